// pf_general_f32.cu -- FP32 instantiations of the particle filter with the paper's own
// resampling variants (multinomial slots, ESS-triggered schedule), in their own
// translation unit so that they compile in parallel with the default ones.
#include "pf_impl.cuh"

namespace smc2 {
const void* pf_select_general_f32(int model, int ppt, bool named) {
  return pf_select_precision<float, true>(model, ppt, named);
}
}  // namespace smc2
