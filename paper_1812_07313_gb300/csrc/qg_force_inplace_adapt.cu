// In-place instantiations (lists read from host memory, results also written
// there) of the FP32 group-force kernel that chooses the number of sinks per
// thread for every work item, scalar and entry-paired forms.
#include "qg_force.cuh"

namespace qg {

template <int FORM>
static const void *pick_inplace_adapt(bool quad, bool guard) {
  if (quad) return guard ? (const void *)force_kernel<float, 4, true, true, true, FORM, true, true>
                         : (const void *)force_kernel<float, 4, true, false, true, FORM, true, true>;
  return guard ? (const void *)force_kernel<float, 4, false, true, true, FORM, true, true>
               : (const void *)force_kernel<float, 4, false, false, true, FORM, true, true>;
}

const void *force_kernel_inplace_adapt(bool epaired, bool quad, bool guard) {
  return epaired ? pick_inplace_adapt<kEntryPaired>(quad, guard) : pick_inplace_adapt<kScalar>(quad, guard);
}

}  // namespace qg
