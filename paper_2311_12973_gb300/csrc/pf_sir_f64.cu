// pf_sir_f64.cu -- instantiations of the particle filter for the binomial SIR model
// (Sec. V-A) in FP64, default and with the paper's resampling variants.
#include "pf_impl.cuh"

namespace smc2 {
const void* pf_select_sir_f64(int ppt, bool named, bool general) {
  return general ? pf_select_sir<double, true>(ppt, named) : pf_select_sir<double, false>(ppt, named);
}
}  // namespace smc2
