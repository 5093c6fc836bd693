// Pair-sum kernels, FP32 form: objective variant with the first and second lambda-derivative
// sums (Sl, Tx, Ty, Q, Ux, Uy), for the lambda-Hessian of the objective.
#include "pairsum_inst.cuh"

namespace dbie {
KernelRef g1_ref_f32_hess(bool tied, int cfg, bool rows) {
  return tied ? g1_ref_cfg<float, VAR_HESS, true>(cfg, rows) : g1_ref_cfg<float, VAR_HESS, false>(cfg, rows);
}
}  // namespace dbie
