// Pair-sum kernels, FP32 form: objective variants (B and its gradient; plus dB/dlambda).
#include "pairsum_inst.cuh"

namespace dbie {
KernelRef g1_ref_f32_val(int var, bool tied, int cfg);
KernelRef g1_ref_f32_newton(bool tied, int cfg);
KernelRef g1_ref_f32_hess(bool tied, int cfg);
KernelRef g1_ref_f32_nv(bool tied, int cfg);

KernelRef g1_ref_f32(int var, bool tied, int cfg) {
  if (var == VAR_OBJ)
    return tied ? g1_ref_cfg<float, VAR_OBJ, true>(cfg) : g1_ref_cfg<float, VAR_OBJ, false>(cfg);
  if (var == VAR_OBJL)
    return tied ? g1_ref_cfg<float, VAR_OBJL, true>(cfg) : g1_ref_cfg<float, VAR_OBJL, false>(cfg);
  if (var == VAR_OBJN) return g1_ref_f32_newton(tied, cfg);
  if (var == VAR_HESS) return g1_ref_f32_hess(tied, cfg);
  if (var == VAR_NV) return g1_ref_f32_nv(tied, cfg);
  return g1_ref_f32_val(var, tied, cfg);
}
}  // namespace dbie
