// Pair-sum kernels, FP32 form: objective variant with dB/dlambda (S_lambda).
#include "pairsum_inst.cuh"

namespace dbie {
KernelRef g1_ref_f32_objl(bool tied, int cfg, bool rows) {
  return tied ? g1_ref_cfg<float, VAR_OBJL, true>(cfg, rows) : g1_ref_cfg<float, VAR_OBJL, false>(cfg, rows);
}
}  // namespace dbie
