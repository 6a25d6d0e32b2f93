// Paired-FP32 instantiations of the group-force kernel: two sinks per float2
// register and Blackwell's f32x2 FMA / add / multiply, FP64 centring and
// merging as in the scalar form.
#include "qg_force.cuh"

namespace qg {

template <int R>
static const void *pick_f32x2(bool quad, bool guard) {
  if (quad) return guard ? (const void *)force_kernel<float, R, true, true, true, true>
                         : (const void *)force_kernel<float, R, true, false, true, true>;
  return guard ? (const void *)force_kernel<float, R, false, true, true, true>
               : (const void *)force_kernel<float, R, false, false, true, true>;
}

const void *force_kernel_f32x2(int R, bool quad, bool guard) {
  switch (R) {
    case 2: return pick_f32x2<2>(quad, guard);
    case 4: return pick_f32x2<4>(quad, guard);
    case 8: return pick_f32x2<8>(quad, guard);
    default: return nullptr;
  }
}

}  // namespace qg
