// pf_general_f64.cu -- FP64 instantiations of the particle filter with the paper's own
// resampling variants (multinomial slots, ESS-triggered schedule), in their own
// translation unit so that they compile in parallel with the default ones.
#include "pf_impl.cuh"

namespace smc2 {
const void* pf_select_general_f64(int model, int ppt, bool named) {
  return pf_select_precision<double, true>(model, ppt, named);
}
}  // namespace smc2
