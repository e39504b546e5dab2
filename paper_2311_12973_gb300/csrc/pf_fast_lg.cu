// The FP32 one-group-per-CTA particle filter for the linear-Gaussian model.
#include "pf_fast.cuh"

namespace smc2 {
const void* pf_fast_select_lg(int ppt, bool trace) {
  return trace ? pf_fast_select<MODEL_LG, true, false>(ppt) : pf_fast_select<MODEL_LG, false, false>(ppt);
}
}  // namespace smc2
