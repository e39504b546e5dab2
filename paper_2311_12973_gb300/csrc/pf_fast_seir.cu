// The FP32 one-group-per-CTA particle filter for the SEIR-type model.
#include "pf_fast.cuh"

namespace smc2 {
const void* pf_fast_select_seir(int ppt, bool trace) {
  return trace ? pf_fast_select<MODEL_SEIR, true, false>(ppt) : pf_fast_select<MODEL_SEIR, false, false>(ppt);
}
}  // namespace smc2
