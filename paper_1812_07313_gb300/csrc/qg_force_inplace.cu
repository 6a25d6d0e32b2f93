// In-place instantiations of the FP32 group-force kernel (scalar and
// entry-paired forms): the lists are read from page-locked host memory over a
// coherent CPU-GPU link, each index checked and kept on the device as it is
// read, and the results written to host memory as well (a single evaluation
// from host arrays).
#include "qg_force.cuh"

namespace qg {

template <int R, int FORM>
static const void *pick_inplace(bool quad, bool guard) {
  if (quad) return guard ? (const void *)force_kernel<float, R, true, true, true, FORM, true>
                         : (const void *)force_kernel<float, R, true, false, true, FORM, true>;
  return guard ? (const void *)force_kernel<float, R, false, true, true, FORM, true>
               : (const void *)force_kernel<float, R, false, false, true, FORM, true>;
}

const void *force_kernel_inplace(int R, bool quad, bool guard, bool epaired) {
  if (epaired) {
    switch (R) {
      case 2: return pick_inplace<2, kEntryPaired>(quad, guard);
      case 4: return pick_inplace<4, kEntryPaired>(quad, guard);
      default: return nullptr;
    }
  }
  switch (R) {
    case 2: return pick_inplace<2, kScalar>(quad, guard);
    case 4: return pick_inplace<4, kScalar>(quad, guard);
    case 8: return pick_inplace<8, kScalar>(quad, guard);
    default: return nullptr;
  }
}

}  // namespace qg
