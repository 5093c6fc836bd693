// pairsum_inst.cuh -- explicit instantiation helpers for the pair-sum kernels.
#pragma once
#include "kernels.h"
#include "pairsum.cuh"

namespace dbie {

template <typename Real, int VAR, bool TIED, int CFG, bool ROWS = false>
KernelRef g1_ref_t() {
  constexpr LaunchCfg c = cfg_of(CFG, VAR);
  const void* fn;
  if constexpr (c.minb > 1)
    fn = (const void*)&g1_kernel_mb<Real, VAR, TIED, c.p, c.nt, NSTAGE, c.minb, ROWS>;
  else
    fn = (const void*)&g1_kernel<Real, VAR, TIED, c.p, c.nt, NSTAGE, false, ROWS>;
  return KernelRef{fn, c.nt, c.p * c.nt,
                   (size_t)NSTAGE * NFIELD * TILE * sizeof(Real)};
}

template <typename Real, int VAR, bool TIED, bool ROWS>
KernelRef g1_ref_cfg_r(int cfg) {
  switch (cfg) {
    case 1: return g1_ref_t<Real, VAR, TIED, 1, ROWS>();
    case 2: return g1_ref_t<Real, VAR, TIED, 2, ROWS>();
    case 3: return g1_ref_t<Real, VAR, TIED, 3, ROWS>();
    case 4: return g1_ref_t<Real, VAR, TIED, 4, ROWS>();
    case 5: return g1_ref_t<Real, VAR, TIED, 5, ROWS>();
    default: return g1_ref_t<Real, VAR, TIED, 0, ROWS>();
  }
}
// FP32 kernels come in two forms: ROWS (groups of 4 tile pixels on one boundary row) or not.
template <typename Real, int VAR, bool TIED>
KernelRef g1_ref_cfg(int cfg, bool rows) {
  return rows ? g1_ref_cfg_r<Real, VAR, TIED, true>(cfg) : g1_ref_cfg_r<Real, VAR, TIED, false>(cfg);
}

}  // namespace dbie
