// Adjoint (transpose of Eq. 16) kernels, FP32 and FP64 forms.
#include "kernels.h"
#include "pairsum.cuh"

namespace dbie {

template <typename Real, bool TIED, int CFG>
KernelRef vjp_ref_t() {
  constexpr LaunchCfg c = cfg_of(CFG);
  const void* fn;
  if constexpr (c.minb > 1) fn = (const void*)&vjp_kernel_mb<Real, TIED, c.p, c.nt, NSTAGE, c.minb>;
  else fn = (const void*)&vjp_kernel<Real, TIED, c.p, c.nt, NSTAGE>;
  return KernelRef{fn, c.nt, c.p * c.nt,
                   (size_t)NSTAGE * VJP_NFIELD * TILE * sizeof(Real)};
}

KernelRef vjp_ref(bool fp64, bool tied, int cfg) {
  if (fp64) return tied ? vjp_ref_t<double, true, 0>() : vjp_ref_t<double, false, 0>();
  switch (cfg) {
    case 1: return tied ? vjp_ref_t<float, true, 1>() : vjp_ref_t<float, false, 1>();
    case 2: return tied ? vjp_ref_t<float, true, 2>() : vjp_ref_t<float, false, 2>();
    case 3: return tied ? vjp_ref_t<float, true, 3>() : vjp_ref_t<float, false, 3>();
    case 4: return tied ? vjp_ref_t<float, true, 4>() : vjp_ref_t<float, false, 4>();
    case 5: return tied ? vjp_ref_t<float, true, 5>() : vjp_ref_t<float, false, 5>();
    default: return tied ? vjp_ref_t<float, true, 0>() : vjp_ref_t<float, false, 0>();
  }
}

// The seven-weight adjoint (gradient through the lambda search) runs once per call, after a
// Hessian pass; one launch shape: 256 threads.  FP32: two pixels per thread, each 64-bit read of
// the 27-field point records (two points) serving four pairs, at 121 registers (two CTAs per
// SM; four pixels would need 170).  FP64: four pixels per thread.
template <typename Real, bool TIED>
KernelRef vjp7_ref_t() {
  constexpr int P = sizeof(Real) == 4 ? 2 : 4;
  return KernelRef{(const void*)&vjp7_kernel<Real, TIED, P, 256, NSTAGE>, 256, P * 256,
                   (size_t)NSTAGE * VJP7_NFIELD * TILE * sizeof(Real)};
}

KernelRef vjp7_ref(bool fp64, bool tied) {
  if (fp64) return tied ? vjp7_ref_t<double, true>() : vjp7_ref_t<double, false>();
  return tied ? vjp7_ref_t<float, true>() : vjp7_ref_t<float, false>();
}

}  // namespace dbie
