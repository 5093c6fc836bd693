// Pair-sum kernels, FP32 form: objective variant with the lambda-derivative sums (Sl, Tx, Ty).
#include "pairsum_inst.cuh"

namespace dbie {
KernelRef g1_ref_f32_newton(bool tied, int cfg, bool rows) {
  return tied ? g1_ref_cfg<float, VAR_OBJN, true>(cfg, rows) : g1_ref_cfg<float, VAR_OBJN, false>(cfg, rows);
}
}  // namespace dbie
