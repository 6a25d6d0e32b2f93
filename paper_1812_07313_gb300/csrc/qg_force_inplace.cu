// In-place instantiations of the FP32 group-force kernel (scalar form): the
// lists are read from page-locked host memory over a coherent CPU-GPU link,
// each index checked and kept on the device as it is read, and the results
// written to host memory as well (a single evaluation from host arrays).
#include "qg_force.cuh"

namespace qg {

template <int R>
static const void *pick_inplace(bool quad, bool guard) {
  if (quad) return guard ? (const void *)force_kernel<float, R, true, true, true, false, true>
                         : (const void *)force_kernel<float, R, true, false, true, false, true>;
  return guard ? (const void *)force_kernel<float, R, false, true, true, false, true>
               : (const void *)force_kernel<float, R, false, false, true, false, true>;
}

const void *force_kernel_inplace(int R, bool quad, bool guard) {
  switch (R) {
    case 2: return pick_inplace<2>(quad, guard);
    case 4: return pick_inplace<4>(quad, guard);
    case 8: return pick_inplace<8>(quad, guard);
    default: return nullptr;
  }
}

}  // namespace qg
