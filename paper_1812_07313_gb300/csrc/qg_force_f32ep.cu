// Entry-paired FP32 instantiations of the group-force kernel: two list
// entries per float2 register (each sink's values broadcast to both halves)
// and Blackwell's f32x2 FMA, FP64 centring and merging as in the scalar form.
#include "qg_force.cuh"

namespace qg {

template <int R>
static const void *pick_f32ep(bool quad, bool guard) {
  if (quad) return guard ? (const void *)force_kernel<float, R, true, true, true, kEntryPaired>
                         : (const void *)force_kernel<float, R, true, false, true, kEntryPaired>;
  return guard ? (const void *)force_kernel<float, R, false, true, true, kEntryPaired>
               : (const void *)force_kernel<float, R, false, false, true, kEntryPaired>;
}

const void *force_kernel_f32ep(int R, bool quad, bool guard) {
  switch (R) {
    case 2: return pick_f32ep<2>(quad, guard);
    case 4: return pick_f32ep<4>(quad, guard);
    default: return nullptr;
  }
}

}  // namespace qg
