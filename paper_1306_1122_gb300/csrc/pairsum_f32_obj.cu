// Pair-sum kernels, FP32 form: the objective variant (B and its gradient) and the dispatch
// over all FP32 variants.
#include "pairsum_inst.cuh"

namespace dbie {
KernelRef g1_ref_f32_val(int var, bool tied, int cfg, bool rows);
KernelRef g1_ref_f32_newton(bool tied, int cfg, bool rows);
KernelRef g1_ref_f32_hess(bool tied, int cfg, bool rows);
KernelRef g1_ref_f32_nv(bool tied, int cfg, bool rows);
KernelRef g1_ref_f32_objl(bool tied, int cfg, bool rows);

KernelRef g1_ref_f32(int var, bool tied, int cfg, bool rows) {
  if (var == VAR_OBJ)
    return tied ? g1_ref_cfg<float, VAR_OBJ, true>(cfg, rows) : g1_ref_cfg<float, VAR_OBJ, false>(cfg, rows);
  if (var == VAR_OBJL) return g1_ref_f32_objl(tied, cfg, rows);
  if (var == VAR_OBJN) return g1_ref_f32_newton(tied, cfg, rows);
  if (var == VAR_HESS) return g1_ref_f32_hess(tied, cfg, rows);
  if (var == VAR_NV) return g1_ref_f32_nv(tied, cfg, rows);
  return g1_ref_f32_val(var, tied, cfg, rows);
}
}  // namespace dbie
