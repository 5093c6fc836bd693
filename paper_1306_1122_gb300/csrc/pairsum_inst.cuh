// pairsum_inst.cuh -- explicit instantiation helpers for the pair-sum kernels.
#pragma once
#include "kernels.h"
#include "pairsum.cuh"

namespace dbie {

template <typename Real, int VAR, bool TIED, int CFG>
KernelRef g1_ref_t() {
  constexpr LaunchCfg c = cfg_of(CFG);
  const void* fn;
  if constexpr (c.minb > 1) fn = (const void*)&g1_kernel_mb<Real, VAR, TIED, c.p, c.nt, NSTAGE, c.minb>;
  else fn = (const void*)&g1_kernel<Real, VAR, TIED, c.p, c.nt, NSTAGE>;
  return KernelRef{fn, c.nt, c.p * c.nt,
                   (size_t)NSTAGE * NFIELD * TILE * sizeof(Real)};
}

template <typename Real, int VAR, bool TIED>
KernelRef g1_ref_cfg(int cfg) {
  switch (cfg) {
    case 1: return g1_ref_t<Real, VAR, TIED, 1>();
    case 2: return g1_ref_t<Real, VAR, TIED, 2>();
    case 3: return g1_ref_t<Real, VAR, TIED, 3>();
    case 4: return g1_ref_t<Real, VAR, TIED, 4>();
    case 5: return g1_ref_t<Real, VAR, TIED, 5>();
    default: return g1_ref_t<Real, VAR, TIED, 0>();
  }
}

}  // namespace dbie
