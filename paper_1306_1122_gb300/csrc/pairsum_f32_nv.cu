// Pair-sum kernels, FP32 form: noise variance (sum of squared weights times pixel variances).
#include "pairsum_inst.cuh"

namespace dbie {
KernelRef g1_ref_f32_nv(bool tied, int cfg, bool rows) {
  return tied ? g1_ref_cfg<float, VAR_NV, true>(cfg, rows) : g1_ref_cfg<float, VAR_NV, false>(cfg, rows);
}
}  // namespace dbie
