// Pair-sum and adjoint kernels, FP32 form, for element Gauss points (Eq. 15) whose positions are
// float pairs (hi + lo): one launch shape (128 threads, one query per thread).
#include "kernels.h"
#include "pairsum.cuh"

namespace dbie {

template <int VAR, bool TIED, bool ROWS>
KernelRef split_ref_r() {
  return KernelRef{(const void*)&g1_kernel<float, VAR, TIED, 1, 128, NSTAGE, true, ROWS>, 128, 128,
                   (size_t)NSTAGE * NFIELD_SPLIT * TILE * sizeof(float)};
}
template <int VAR, bool TIED>
KernelRef split_ref(bool rows) {
  return rows ? split_ref_r<VAR, TIED, true>() : split_ref_r<VAR, TIED, false>();
}

KernelRef g1_ref_f32_split(int var, bool tied, bool rows) {
  switch (var) {
    case VAR_V: return tied ? split_ref<VAR_V, true>(rows) : split_ref<VAR_V, false>(rows);
    case VAR_VL: return tied ? split_ref<VAR_VL, true>(rows) : split_ref<VAR_VL, false>(rows);
    case VAR_OBJ: return tied ? split_ref<VAR_OBJ, true>(rows) : split_ref<VAR_OBJ, false>(rows);
    case VAR_OBJL: return tied ? split_ref<VAR_OBJL, true>(rows) : split_ref<VAR_OBJL, false>(rows);
    case VAR_OBJN: return tied ? split_ref<VAR_OBJN, true>(rows) : split_ref<VAR_OBJN, false>(rows);
    default: return tied ? split_ref<VAR_HESS, true>(rows) : split_ref<VAR_HESS, false>(rows);
  }
}

KernelRef vjp_ref_split(bool tied) {
  const void* fn = tied ? (const void*)&vjp_kernel<float, true, 1, 128, NSTAGE, true>
                        : (const void*)&vjp_kernel<float, false, 1, 128, NSTAGE, true>;
  return KernelRef{fn, 128, 128, (size_t)NSTAGE * VJP_NFIELD * TILE * sizeof(float)};
}

KernelRef vjp7_ref_split(bool tied) {
  const void* fn = tied ? (const void*)&vjp7_kernel<float, true, 2, 256, NSTAGE, true>
                        : (const void*)&vjp7_kernel<float, false, 2, 256, NSTAGE, true>;
  return KernelRef{fn, 256, 512, (size_t)NSTAGE * VJP7_NFIELD * TILE * sizeof(float)};
}

}  // namespace dbie
