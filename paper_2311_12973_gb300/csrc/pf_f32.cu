// pf_f32.cu -- FP32 instantiations of the particle-filter kernel.
#include "pf_impl.cuh"

namespace smc2 {
const void* pf_select_f32(int model, int ppt, bool named) {
  return pf_select_precision<float, false>(model, ppt, named);
}
}  // namespace smc2
