// The FP32 particle filter with filter groups of unequal width sharing a CTA
// (warps, or several warps on named barriers), for launches over datasets of
// unequal size.
#include "pf_fast.cuh"

namespace smc2 {
const void* pf_fast_select_grouped(int model, int ppt) {
  return model == MODEL_LG ? pf_fast_select<MODEL_LG, false, true>(ppt) : pf_fast_select<MODEL_SEIR, false, true>(ppt);
}
}  // namespace smc2
