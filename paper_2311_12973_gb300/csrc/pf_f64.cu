// pf_f64.cu -- FP64 instantiations of the particle-filter kernel.
#include "pf_impl.cuh"

namespace smc2 {
const void* pf_select_f64(int model, int ppt, bool named) {
  return pf_select_precision<double, false>(model, ppt, named);
}
}  // namespace smc2
