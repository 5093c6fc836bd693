// Pair-sum and adjoint kernels, FP32 form, for element Gauss points (Eq. 15) whose positions are
// float pairs (hi + lo): one launch shape (128 threads, one query per thread).
#include "kernels.h"
#include "pairsum.cuh"

namespace dbie {

template <int VAR, bool TIED>
KernelRef split_ref() {
  return KernelRef{(const void*)&g1_kernel<float, VAR, TIED, 1, 128, NSTAGE, true>, 128, 128,
                   (size_t)NSTAGE * NFIELD_SPLIT * TILE * sizeof(float)};
}

KernelRef g1_ref_f32_split(int var, bool tied) {
  switch (var) {
    case VAR_V: return tied ? split_ref<VAR_V, true>() : split_ref<VAR_V, false>();
    case VAR_VL: return tied ? split_ref<VAR_VL, true>() : split_ref<VAR_VL, false>();
    case VAR_OBJ: return tied ? split_ref<VAR_OBJ, true>() : split_ref<VAR_OBJ, false>();
    case VAR_OBJL: return tied ? split_ref<VAR_OBJL, true>() : split_ref<VAR_OBJL, false>();
    case VAR_OBJN: return tied ? split_ref<VAR_OBJN, true>() : split_ref<VAR_OBJN, false>();
    default: return tied ? split_ref<VAR_HESS, true>() : split_ref<VAR_HESS, false>();
  }
}

KernelRef vjp_ref_split(bool tied) {
  const void* fn = tied ? (const void*)&vjp_kernel<float, true, 1, 128, NSTAGE, true>
                        : (const void*)&vjp_kernel<float, false, 1, 128, NSTAGE, true>;
  return KernelRef{fn, 128, 128, (size_t)NSTAGE * VJP_NFIELD * TILE * sizeof(float)};
}

KernelRef vjp7_ref_split(bool tied) {
  const void* fn = tied ? (const void*)&vjp7_kernel<float, true, 1, 128, NSTAGE, true>
                        : (const void*)&vjp7_kernel<float, false, 1, 128, NSTAGE, true>;
  return KernelRef{fn, 128, 128, (size_t)NSTAGE * VJP7_NFIELD * TILE * sizeof(float)};
}

}  // namespace dbie
