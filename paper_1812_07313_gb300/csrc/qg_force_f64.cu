// All-FP64 instantiations of the group-force kernel (comparison path).
#include "qg_force.cuh"

namespace qg {

const void *force_kernel_f64(int R, bool quad, bool guard) {
  if (R != 2) return nullptr;
  if (quad) return guard ? (const void *)force_kernel<double, 2, true, true, true, false>
                         : (const void *)force_kernel<double, 2, true, false, true, false>;
  return guard ? (const void *)force_kernel<double, 2, false, true, true, false>
               : (const void *)force_kernel<double, 2, false, false, true, false>;
}

}  // namespace qg
