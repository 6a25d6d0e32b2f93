// Instantiations of the FP32 group-force kernel (centred) that choose the
// number of sinks per thread for every work item, from 1 to 4, in the scalar
// and entry-paired forms.
#include "qg_force.cuh"

namespace qg {

template <int FORM>
static const void *pick_adapt(bool quad, bool guard) {
  if (quad) return guard ? (const void *)force_kernel<float, 4, true, true, true, FORM, false, true>
                         : (const void *)force_kernel<float, 4, true, false, true, FORM, false, true>;
  return guard ? (const void *)force_kernel<float, 4, false, true, true, FORM, false, true>
               : (const void *)force_kernel<float, 4, false, false, true, FORM, false, true>;
}

const void *force_kernel_adapt(bool epaired, bool quad, bool guard) {
  return epaired ? pick_adapt<kEntryPaired>(quad, guard) : pick_adapt<kScalar>(quad, guard);
}

}  // namespace qg
