// Pair-sum kernels, FP64 form (the plain double-precision reference on the GPU).
#include "pairsum_inst.cuh"

namespace dbie {
KernelRef g1_ref_f64(int var, bool tied) {
  switch (var) {
    case VAR_V: return tied ? g1_ref_t<double, VAR_V, true, 0>() : g1_ref_t<double, VAR_V, false, 0>();
    case VAR_VL: return tied ? g1_ref_t<double, VAR_VL, true, 0>() : g1_ref_t<double, VAR_VL, false, 0>();
    case VAR_OBJ: return tied ? g1_ref_t<double, VAR_OBJ, true, 0>() : g1_ref_t<double, VAR_OBJ, false, 0>();
    case VAR_OBJL: return tied ? g1_ref_t<double, VAR_OBJL, true, 0>() : g1_ref_t<double, VAR_OBJL, false, 0>();
    case VAR_OBJN: return tied ? g1_ref_t<double, VAR_OBJN, true, 0>() : g1_ref_t<double, VAR_OBJN, false, 0>();
    case VAR_HESS: return tied ? g1_ref_t<double, VAR_HESS, true, 0>() : g1_ref_t<double, VAR_HESS, false, 0>();
    default: return tied ? g1_ref_t<double, VAR_NV, true, 0>() : g1_ref_t<double, VAR_NV, false, 0>();
  }
}
}  // namespace dbie
