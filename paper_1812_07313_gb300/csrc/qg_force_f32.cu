// FP32 instantiations of the group-force kernel (mixed precision: FP64
// centring and merging, FP32 pairwise arithmetic), scalar FP32 form.
#include "qg_force.cuh"

namespace qg {

template <int R>
static const void *pick_f32(bool quad, bool guard, bool centred) {
  if (centred) {
    if (quad) return guard ? (const void *)force_kernel<float, R, true, true, true, false>
                           : (const void *)force_kernel<float, R, true, false, true, false>;
    return guard ? (const void *)force_kernel<float, R, false, true, true, false>
                 : (const void *)force_kernel<float, R, false, false, true, false>;
  }
  if (quad) return guard ? (const void *)force_kernel<float, R, true, true, false, false>
                         : (const void *)force_kernel<float, R, true, false, false, false>;
  return guard ? (const void *)force_kernel<float, R, false, true, false, false>
               : (const void *)force_kernel<float, R, false, false, false, false>;
}

const void *force_kernel_f32(int R, bool quad, bool guard, bool centred) {
  switch (R) {
    case 2: return pick_f32<2>(quad, guard, centred);
    case 4: return pick_f32<4>(quad, guard, centred);
    case 8: return pick_f32<8>(quad, guard, centred);
    default: return nullptr;
  }
}

}  // namespace qg
