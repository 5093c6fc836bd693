// Pair-sum kernels, FP32 form: value variants (B; B and dB/dlambda).
#include "pairsum_inst.cuh"

namespace dbie {
KernelRef g1_ref_f32_val(int var, bool tied, int cfg, bool rows) {
  if (var == VAR_V) return tied ? g1_ref_cfg<float, VAR_V, true>(cfg, rows) : g1_ref_cfg<float, VAR_V, false>(cfg, rows);
  return tied ? g1_ref_cfg<float, VAR_VL, true>(cfg, rows) : g1_ref_cfg<float, VAR_VL, false>(cfg, rows);
}
}  // namespace dbie
