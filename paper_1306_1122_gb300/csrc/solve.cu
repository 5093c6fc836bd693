// solve.cu -- per-point objective and the on-device Downhill Simplex search for lambda.
//
// Compiled with -fmad=false: the simplex arithmetic and the objective are evaluated with
// separately rounded operations, as written.
//
//  * objective: B_p = z S0_p, dB_p/dx = z Sx_p, dB_p/dy = z Sy_p, dB_p/dz = S0_p + z^2 S1_p
//    (the fixed-lambda derivatives of Eq. 13), J = curl B (Eq. 14), f = |J x B| / (|J||B|)
//    (Eq. 8), g = |div B| dV/dSigma / |B| (Eq. 9), Phi = f + w_g g.
//  * simplex (Sect. 2.1; Nelder & Mead 1965, reflection 1, expansion 2, contraction 1/2,
//    shrink 1/2, outside/inside contraction as in Lagarias et al. 1998): one thread per active
//    point advances a state machine by one step per round; every round evaluates all pending
//    trial points of all active points in one pair-sum pass.
#include "kernels.h"
#include "solve.cuh"

namespace dbie {

struct Eval {
  double B[3];
  double f, g, phi;
  double s;   // error bound of phi (certified decisions; 0 when not computed)
};

__device__ __forceinline__ void objective(const double B[3], const double G[9], double g_scale,
                                          double w_g, double& f, double& g, double& phi) {
  const double Jx = G[3 * 2 + 1] - G[3 * 1 + 2];
  const double Jy = G[3 * 0 + 2] - G[3 * 2 + 0];
  const double Jz = G[3 * 1 + 0] - G[3 * 0 + 1];
  const double div = G[0] + G[4] + G[8];
  const double cx = Jy * B[2] - Jz * B[1];
  const double cy = Jz * B[0] - Jx * B[2];
  const double cz = Jx * B[1] - Jy * B[0];
  const double nJ = sqrt(Jx * Jx + Jy * Jy + Jz * Jz);
  const double nB = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  const double nC = sqrt(cx * cx + cy * cy + cz * cz);
  f = (nJ * nB > 0.0) ? nC / (nJ * nB) : 0.0;
  g = (nB > 0.0) ? fabs(div) * g_scale / nB : 0.0;
  phi = f + w_g * g;
}

// Sum over the split partials of sum s of the query with local index j in problem pidx
// (near-field corrections were already added to split 0).
__device__ __forceinline__ double gather_sum(const double* out, const PlanHdr& h,
                                             const int32_t* item_off, int pidx, int64_t j,
                                             int nsum, int s) {
  double v = 0.0;
  for (int sp = 0; sp < h.nsplit; ++sp) v += out[out_index(h, item_off, pidx, j, sp, s, nsum)];
  return v;
}

// Pixel-exact near field: add the point's lambda-independent correction of B and grad B
// (corr: dB_p at p, d(dB_p/dx_j) at 3 + 3 p + j).
__device__ __forceinline__ void add_corr(const double* corr, double B[3], double G[9]) {
  if (!corr) return;
  for (int p = 0; p < 3; ++p) B[p] += corr[p];
  for (int j = 0; j < 9; ++j) G[j] += corr[3 + j];
}

// B, gradient and objective from the 12 objective sums of one query (corr: see add_corr).
__device__ __forceinline__ void assemble_obj(const double S[12], double z, double g_scale,
                                             double w_g, Eval& e, double G[9],
                                             const double* corr) {
  for (int p = 0; p < 3; ++p) {
    const double S0 = S[p * 4 + 0], S1 = S[p * 4 + 1], Sx = S[p * 4 + 2], Sy = S[p * 4 + 3];
    e.B[p] = z * S0;
    G[3 * p + 0] = z * Sx;
    G[3 * p + 1] = z * Sy;
    G[3 * p + 2] = S0 + z * z * S1;
  }
  add_corr(corr, e.B, G);
  objective(e.B, G, g_scale, w_g, e.f, e.g, e.phi);
}

// ----------------------------------------------------------------- eval finalize ----
template <int VAR>
__global__ void finalize_eval_kernel(int64_t n, const PlanHdr* __restrict__ plan,
                                     const int32_t* __restrict__ item_off,
                                     const double* __restrict__ out,
                                     const float4* __restrict__ qpos,
                                     const Lam4* __restrict__ qlam, double g_scale, double w_g,
                                     double* B, double* gradB, double* dBdl, const double* gB,
                                     double* fgphi, const double* corr) {
  constexpr int NS = nsum_per_comp(VAR);
  constexpr int NSUM = 3 * NS;
  const PlanHdr h = *plan;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 pos = qpos[i];
    const double z = (double)pos.z;
    double S[NSUM];
    for (int s = 0; s < NSUM; ++s) S[s] = gather_sum(out, h, item_off, 0, i, NSUM, s);
    double Bv[3], G[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = 0; p < 3; ++p) Bv[p] = z * S[p * NS];
    if constexpr (has_grad(VAR)) {
      for (int p = 0; p < 3; ++p) {
        G[3 * p + 0] = z * S[p * NS + 2];
        G[3 * p + 1] = z * S[p * NS + 3];
        G[3 * p + 2] = S[p * NS] + z * z * S[p * NS + 1];
      }
    }
    add_corr(corr ? corr + 12 * i : nullptr, Bv, G);
    if (B)
      for (int p = 0; p < 3; ++p) B[3 * i + p] = Bv[p];
    if constexpr (has_grad(VAR)) {
      if (gradB)
        for (int j = 0; j < 9; ++j) gradB[9 * i + j] = G[j];
      if (fgphi) {
        double f, g, phi;
        objective(Bv, G, g_scale, w_g, f, g, phi);
        fgphi[3 * i + 0] = f;
        fgphi[3 * i + 1] = g;
        fgphi[3 * i + 2] = phi;
      }
    }
    if constexpr (has_dlam(VAR)) {
      const Lam4 l = qlam[i];
      const double lam[3] = {l.x, l.y, l.z};
      for (int p = 0; p < 3; ++p) {
        const double d = z * lam[p] * S[p * NS + idx_sl(VAR)];
        if (gB) {
          if (dBdl) dBdl[3 * i + p] = gB[3 * i + p] * d;
        } else if (dBdl) {
          dBdl[3 * i + p] = d;
        }
      }
    }
  }
}

void launch_finalize_eval(int var, int64_t n, const PlanHdr* plan, const int32_t* item_off,
                          const double* out, const float4* qpos, const Lam4* qlam, double g_scale,
                          double w_g, double* B, double* gradB, double* dBdl, const double* gB,
                          double* fgphi, const double* corr, cudaStream_t s) {
  if (n <= 0) return;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
#define FIN(V)                                                                              \
  finalize_eval_kernel<V><<<grid, 256, 0, s>>>(n, plan, item_off, out, qpos, qlam, g_scale, \
                                               w_g, B, gradB, dBdl, gB, fgphi, corr)
  switch (var) {
    case VAR_V: FIN(VAR_V); break;
    case VAR_VL: FIN(VAR_VL); break;
    case VAR_OBJ: FIN(VAR_OBJ); break;
    default: FIN(VAR_OBJL); break;
  }
#undef FIN
}

// ------------------------------------------------------------------ simplex state ----
// A vertex (or the reflected or trial point) of one point's simplex: lambda, the field and
// objective there, the error bound s of its Phi (0 after a float-float re-evaluation) and its
// identity in the state the step started from (0..n vertex, VID_R reflected, VID_E trial).
struct Vert {
  double l[3];
  double B[3];
  double f, g, phi;
  double s;
  int id;
};

__device__ __forceinline__ double& SD(const SolveArgs& a, int f, int64_t g) {
  return a.sd[(int64_t)f * a.N + g];
}
__device__ __forceinline__ int32_t& SI(const SolveArgs& a, int f, int64_t g) {
  return a.si[(int64_t)f * a.N + g];
}

__device__ __forceinline__ void load_vert(const SolveArgs& a, int64_t g, int v, Vert& x) {
  for (int d = 0; d < 3; ++d) x.l[d] = SD(a, D_VL + v * 3 + d, g);
  for (int p = 0; p < 3; ++p) x.B[p] = SD(a, D_VB + v * 3 + p, g);
  x.f = SD(a, D_VF + v, g);
  x.g = SD(a, D_VG + v, g);
  x.phi = SD(a, D_VPHI + v, g);
  x.s = SD(a, D_VS + v, g);
  x.id = v;
}
__device__ __forceinline__ void store_vert(const SolveArgs& a, int64_t g, int v, const Vert& x) {
  for (int d = 0; d < 3; ++d) SD(a, D_VL + v * 3 + d, g) = x.l[d];
  for (int p = 0; p < 3; ++p) SD(a, D_VB + v * 3 + p, g) = x.B[p];
  SD(a, D_VF + v, g) = x.f;
  SD(a, D_VG + v, g) = x.g;
  SD(a, D_VPHI + v, g) = x.phi;
  SD(a, D_VS + v, g) = x.s;
}
// The reflected point (lambda at D_RL, value at D_RB..D_RPHI, bound at D_RS).
__device__ __forceinline__ void load_r(const SolveArgs& a, int64_t g, Vert& x) {
  for (int d = 0; d < 3; ++d) x.l[d] = SD(a, D_RL + d, g);
  for (int p = 0; p < 3; ++p) x.B[p] = SD(a, D_RB + p, g);
  x.f = SD(a, D_RF, g);
  x.g = SD(a, D_RG, g);
  x.phi = SD(a, D_RPHI, g);
  x.s = SD(a, D_RS, g);
  x.id = VID_R;
}
__device__ __forceinline__ void store_r(const SolveArgs& a, int64_t g, const Vert& x) {
  for (int d = 0; d < 3; ++d) SD(a, D_RL + d, g) = x.l[d];
  for (int p = 0; p < 3; ++p) SD(a, D_RB + p, g) = x.B[p];
  SD(a, D_RF, g) = x.f;
  SD(a, D_RG, g) = x.g;
  SD(a, D_RPHI, g) = x.phi;
  SD(a, D_RS, g) = x.s;
}
// The evaluated single trial point (lambda at D_TL, value at D_EB..D_ES).
__device__ __forceinline__ void load_e(const SolveArgs& a, int64_t g, Vert& x) {
  for (int d = 0; d < 3; ++d) x.l[d] = SD(a, D_TL + d, g);
  for (int p = 0; p < 3; ++p) x.B[p] = SD(a, D_EB + p, g);
  x.f = SD(a, D_EF, g);
  x.g = SD(a, D_EG, g);
  x.phi = SD(a, D_EPHI, g);
  x.s = SD(a, D_ES, g);
  x.id = VID_E;
}
__device__ __forceinline__ void store_e(const SolveArgs& a, int64_t g, const Vert& x) {
  for (int p = 0; p < 3; ++p) SD(a, D_EB + p, g) = x.B[p];
  SD(a, D_EF, g) = x.f;
  SD(a, D_EG, g) = x.g;
  SD(a, D_EPHI, g) = x.phi;
  SD(a, D_ES, g) = x.s;
}
__device__ __forceinline__ void set_value(Vert& x, const Eval& e) {
  for (int p = 0; p < 3; ++p) x.B[p] = e.B[p];
  x.f = e.f;
  x.g = e.g;
  x.phi = e.phi;
  x.s = e.s;
}

// The pixel-exact correction of point g, or null (none, or the point is above its height).
__device__ __forceinline__ const double* corr_of(const SolveArgs& a, const ProbDesc& pd,
                                                 int64_t g, double z) {
  return (a.corr && pd.pxe_z > 0.0 && z <= pd.pxe_z) ? a.corr + 12 * g : nullptr;
}

// ------------------------------------------------------------- certified decisions ----
// Error bound of Phi computed from the mixed form's sums (FP32 pair terms).  Per pair term the
// error of the FP32 evaluation is bounded by the measured accuracy of its operations on GB300:
// SFU sine and cosine within 3.3e-7 absolute on [0, pi] and about 1.1e-7 |theta| beyond (the
// unit's own scaling of the argument), reciprocal square root within 1.25e-7 relative, plus
// FP32 rounding.  With theta = lambda r and u = theta sin(theta) + cos(theta) that gives, for a
// pixel of component p,
//   |d(u b / r^3)|   <= (A0 + A1 theta + A2 theta^2) |b| / r^3,
//   |d(psi b)|       <= [lambda^2 (A0 + A2 theta) + 3 (A3 + A4 theta + A2 theta^2) / r^2] |b| / r^3
// (psi r^3 = lambda^2 cos(theta) - 3 u / r^2; Sx and Sy carry |dx|, |dy| <= r more), and the sum
// over pixels turns these into polynomials in |lambda_p| whose coefficients are the point's
// lambda-independent sums M_j = sum_k |b_pk| / r^j, j = 1..5.  The bounds of B and grad B are
// carried to J = curl B, div B, f (Eq. 8) and g (Eq. 9) to first order:
//   |df| <= |dJ| / |J| + |dB| / |B|  (at most 1),   |dg| <= g_scale |d div B| / |B| + g |dB| / |B|.
// It is a worst case: on the Low & Lou and active-region workloads the measured error of Phi
// stays below 5 % of it.
constexpr double BND_A0 = 9.5e-7, BND_A1 = 1.06e-6, BND_A2 = 1.1e-7, BND_A3 = 1.45e-6,
                 BND_A4 = 1.56e-6;

// First-order bound of Phi's error from the bounds dB (3) and dG (9) of B and grad B.
__device__ __forceinline__ double propagate_bound(const double dB[3], const double dG[9],
                                                  const double B[3], const double G[9],
                                                  double g, double g_scale, double w_g) {
  const double Jx = G[7] - G[5], Jy = G[2] - G[6], Jz = G[3] - G[1];
  const double nJ = sqrt(Jx * Jx + Jy * Jy + Jz * Jz);
  const double nB = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  const double dJx = dG[7] + dG[5], dJy = dG[2] + dG[6], dJz = dG[3] + dG[1];
  const double ndJ = sqrt(dJx * dJx + dJy * dJy + dJz * dJz);
  const double ndB = sqrt(dB[0] * dB[0] + dB[1] * dB[1] + dB[2] * dB[2]);
  if (!(nB > 0.0)) return 2.0;
  double sf = nJ > 0.0 ? ndJ / nJ + ndB / nB : 1.0;
  if (sf > 1.0) sf = 1.0;
  const double sg = g_scale * (dG[0] + dG[4] + dG[8]) / nB + g * ndB / nB;
  return sf + w_g * sg;
}

__device__ __forceinline__ double mixed_phi_bound(const double* M, const double lam[3], int dim,
                                                   double z, const double B[3], const double G[9],
                                                   double g, double g_scale, double w_g) {
  double dB[3], dG[9];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const double L = fabs(dim == 1 ? lam[0] : lam[p]);
    const double* m = M + 5 * p;
    const double L2 = L * L, L3 = L2 * L;
    const double s0 = BND_A0 * m[2] + BND_A1 * L * m[1] + BND_A2 * L2 * m[0];
    const double sx = BND_A0 * L2 * m[1] + BND_A2 * L3 * m[0] +
                      3.0 * (BND_A3 * m[3] + BND_A4 * L * m[2] + BND_A2 * L2 * m[1]);
    const double s1 = BND_A0 * L2 * m[2] + BND_A2 * L3 * m[1] +
                      3.0 * (BND_A3 * m[4] + BND_A4 * L * m[3] + BND_A2 * L2 * m[2]);
    dB[p] = z * s0;
    dG[3 * p + 0] = z * sx;
    dG[3 * p + 1] = z * sx;
    dG[3 * p + 2] = s0 + z * z * s1;
  }
  return propagate_bound(dB, dG, B, G, g, g_scale, w_g);
}

// Error bounds of the difference sums (pairsum_dif.cu) that take a point's float-float
// reference sums at lambda_0 to lambda_a, per component p, with dl = |lambda_a - lambda_0| and
// L = |lambda_a| + |lambda_0|.  Every product of a pixel's difference terms carries a factor
// |delta| = dl r / 2 (or dl).  With the operation accuracies of mixed_phi_bound (SFU sine and
// cosine of sigma within 3.3e-7 + 1.1e-7 |sigma| absolute, sigma, delta and r within 3.2e-7
// relative, the Taylor sine and cosine of delta within 3e-8, FP32 rounding, and sums over blocks
// of 8 pixels in FP32) the changes du of u and dw of psi r^3 are in error by at most
//   dl (2.1e-6 r + 2.6e-6 L r^2 + 1.1e-7 L^2 r^3)                   (du, b / r^3 included)
//   dl (6.3e-6 / r + 1.22e-5 L + 2.6e-6 L^2 r + 1.1e-7 L^3 r^2)     (dw)
// (|du| <= dl L r^2 and |dw| <= dl (5 L + L^2 r) bound the relative roundings), and summed with
// |b| / r^3 they become polynomials in dl and L over the point's sums M_j = sum_k |b_pk| / r^j,
// j = 0..5.  The coefficients below are twice those.  The float-float reference sums add 1e-12
// of their absolute-value sums (their measured error is at most 1.4e-13 of them).
constexpr double DIF_C00 = 4.2e-6, DIF_C01 = 5.2e-6, DIF_C02 = 2.2e-7;
constexpr double DIF_C10 = 1.3e-5, DIF_C11 = 2.4e-5, DIF_C12 = 5.2e-6, DIF_C13 = 2.2e-7;
constexpr double DIF_FF = 1e-12;

// e[4 p + s]: bounds of S0, S1, Sx, Sy of component p (M: M_1..M_5 per component, M0: M_0).
__device__ __forceinline__ void dif_sum_bounds(const double* M, const double* M0,
                                               const double la[3], const double l0[3], int dim,
                                               double e[12]) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int q = dim == 1 ? 0 : p;
    const double dl = fabs(la[q] - l0[q]);
    const double L = fabs(la[q]) + fabs(l0[q]), L2 = L * L, L3 = L2 * L;
    const double R = fabs(l0[q]), R2 = R * R;
    const double* m = M + 5 * p;   // m[j - 1] = M_j
    const double m0 = M0[p];
    const double e0 = dl * (DIF_C00 * m[1] + DIF_C01 * L * m[0] + DIF_C02 * L2 * m0) +
                      DIF_FF * (m[2] + R * m[1]);
    const double e1 = dl * (DIF_C10 * m[3] + DIF_C11 * L * m[2] + DIF_C12 * L2 * m[1] +
                            DIF_C13 * L3 * m[0]) +
                      DIF_FF * (3.0 * m[4] + 3.0 * R * m[3] + R2 * m[2]);
    const double ex = dl * (DIF_C10 * m[2] + DIF_C11 * L * m[1] + DIF_C12 * L2 * m[0] +
                            DIF_C13 * L3 * m0) +
                      DIF_FF * (3.0 * m[3] + 3.0 * R * m[2] + R2 * m[1]);
    e[4 * p + 0] = e0;
    e[4 * p + 1] = e1;
    e[4 * p + 2] = ex;
    e[4 * p + 3] = ex;
  }
}

// Phi bound of a value assembled from reference plus difference sums with sum bounds e.
__device__ __forceinline__ double dif_phi_bound(const double e[12], double z, const double B[3],
                                                const double G[9], double g, double g_scale,
                                                double w_g) {
  double dB[3], dG[9];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    dB[p] = z * e[4 * p];
    dG[3 * p + 0] = z * e[4 * p + 2];
    dG[3 * p + 1] = z * e[4 * p + 3];
    dG[3 * p + 2] = e[4 * p] + z * z * e[4 * p + 1];
  }
  return propagate_bound(dB, dG, B, G, g, g_scale, w_g);
}

// The first near tie of a step: a comparison whose two values differ by no more than the sum of
// their tie radii.  A value's radius is `band` times its bound for a mixed-form value (bound
// s > 0), `band_d` times it for a value re-evaluated by difference (stored as -s), and 0 for a
// value re-evaluated in float-float.
struct TieLog {
  double band;     // 0: decisions are not certified
  double band_d;
  int a, b;        // ids of the first near-tied values (-1: none)
  __device__ __forceinline__ double radius(double s) const {
    return s > 0.0 ? band * s : band_d * (-s);
  }
  __device__ __forceinline__ void note(int ia, double sa, int ib, double sb, double gap) {
    if (band > 0.0 && a < 0) {
      const double r = radius(sa) + radius(sb);
      if (r > 0.0 && fabs(gap) <= r) {
        a = sa != 0.0 ? ia : -1;
        b = sb != 0.0 ? ib : -1;
        if (a < 0) { a = b; b = -1; }
      }
    }
  }
  __device__ __forceinline__ bool lt(const Vert& x, const Vert& y) {
    note(x.id, x.s, y.id, y.s, x.phi - y.phi);
    return x.phi < y.phi;
  }
  __device__ __forceinline__ bool le(const Vert& x, const Vert& y) {
    note(x.id, x.s, y.id, y.s, x.phi - y.phi);
    return x.phi <= y.phi;
  }
};

// Objective of the k-th pending query of point g; its error bound when decisions are certified.
__device__ __forceinline__ void read_eval(const SolveArgs& a, const PlanHdr& h, int pidx,
                                          int64_t slot, double z, Eval& e, int64_t g,
                                          const double lam[3]) {
  const ProbDesc& pd = a.probs[pidx];
  const int64_t j = slot - pd.q_off;
  double S[12], G[9];
#pragma unroll
  for (int s = 0; s < 12; ++s) S[s] = gather_sum(a.out, h, a.item_off, pidx, j, 12, s);
  assemble_obj(S, z, pd.g_scale, a.o.w_g, e, G, corr_of(a, pd, g, z));
  e.s = (a.o.tie > 0.0 && a.msc)
            ? mixed_phi_bound(a.msc + 15 * g, lam, a.o.dim, z, e.B, G, e.g, pd.g_scale, a.o.w_g)
            : 0.0;
}

// Objective of a float-float re-evaluation slot of point g (bound 0) and its 12 sums.
__device__ __forceinline__ void read_eval_ff(const SolveArgs& a, const PlanHdr& hf, int pidx,
                                             int64_t slot, double z, Eval& e, int64_t g,
                                             double S[12]) {
  const ProbDesc& pd = a.probs[pidx];
  const int64_t j = slot - pd.qff_off;
  double G[9];
#pragma unroll
  for (int s = 0; s < 12; ++s) S[s] = gather_sum(a.fout, hf, a.fitem_off, pidx, j, 12, s);
  assemble_obj(S, z, pd.g_scale, a.o.w_g, e, G, corr_of(a, pd, g, z));
  e.s = 0.0;
}

// Objective of a difference re-evaluation slot of point g at lambda lt: the point's float-float
// reference sums plus the difference sums; its bound is stored negated (a difference value).
__device__ __forceinline__ void read_eval_dif(const SolveArgs& a, const PlanHdr& hd, int pidx,
                                              int64_t slot, double z, Eval& e, int64_t g,
                                              const double lt[3]) {
  const ProbDesc& pd = a.probs[pidx];
  const int64_t j = slot - pd.qff_off;
  double S[12], G[9];
#pragma unroll
  for (int s = 0; s < 12; ++s)
    S[s] = SD(a, D_REFS + s, g) + gather_sum(a.dout, hd, a.ditem_off, pidx, j, 12, s);
  assemble_obj(S, z, pd.g_scale, a.o.w_g, e, G, corr_of(a, pd, g, z));
  const double l0[3] = {SD(a, D_REFL, g), SD(a, D_REFL + 1, g), SD(a, D_REFL + 2, g)};
  double eb[12];
  dif_sum_bounds(a.msc + 15 * g, a.msc0 + 3 * g, lt, l0, a.o.dim, eb);
  const double sd = dif_phi_bound(eb, z, e.B, G, e.g, pd.g_scale, a.o.w_g);
  e.s = -(sd > 0.0 ? sd : 1e-300);
}

// atomicAdd(ctr, v) for the lanes of a warp that reach it together (whatever branch they are
// in): lanes with the same counter add their total with one atomic and take consecutive ranges
// in lane order.  Every simplex or quasi-Newton point emits its trial queries through these
// counters each round, so one atomic per lane would serialise N updates of one address.
__device__ __forceinline__ int atomic_add_warp(int* ctr, int v) {
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, reinterpret_cast<unsigned long long>(ctr));
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  const unsigned below = peers & ((1u << lane) - 1u);
  int same = 0;
  __match_all_sync(peers, v, &same);
  int prefix = 0, total = 0;
  if (same) {
    prefix = v * __popc(below);
    total = v * __popc(peers);
  } else {
    for (unsigned m = peers; m; m &= m - 1u) {
      const int l = __ffs(m) - 1;
      const int vl = __shfl_sync(peers, v, l);
      if (l < lane) prefix += vl;
      total += vl;
    }
  }
  int base = 0;
  if (lane == leader) base = atomicAdd(ctr, total);
  base = __shfl_sync(peers, base, leader);
  return base + prefix;
}

// Queue K trial points (lambda rows) of point g for the next round (K fixed at compile time, so
// the rows stay in registers).
template <int K>
__device__ __forceinline__ void emit(const SolveArgs& a, int64_t g, const float4& pos, int pidx,
                                     const double (*lam)[3]) {
  const ProbDesc& pd = a.probs[pidx];
  const int base = atomic_add_warp(a.nxt.q_cnt + pidx, K);
  const int64_t slot0 = pd.q_off + base;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    a.nxt.qpos[slot0 + j] = pos;
    if (a.o.dim == 1) a.nxt.qlam[slot0 + j] = make_lam4(lam[j][0], lam[j][0], lam[j][0]);
    else a.nxt.qlam[slot0 + j] = make_lam4(lam[j][0], lam[j][1], lam[j][2]);
  }
  if (a.o.near_on && (double)pos.z <= pd.near_z) {
    const int nb = atomic_add_warp(a.nxt.near_cnt, K);
#pragma unroll
    for (int j = 0; j < K; ++j) a.nxt.near[nb + j] = (int32_t)(slot0 + j);
  }
  SI(a, I_QSLOT, g) = (int32_t)slot0;
  a.nxt.act[atomic_add_warp(a.nxt.act_cnt, 1)] = (int32_t)g;
}

// Queue the re-evaluation of k (1 or 2) values of point g on side `sd` and put the point on that
// side's waiting list: value j in float-float, or (dif[j]) as the difference from the point's
// float-float reference at lambda lref.  The value ids go to I_RTGT, one per byte (| RT_DIF for
// differences), and the first slot of each kind to I_RSLOT, I_DSLOT.
__device__ __forceinline__ void emit_reeval(const SolveArgs& a, const RoundBuf& sd, int64_t g,
                                            const float4& pos, int pidx, int k,
                                            const double (&l)[2][3], int id0, int id1,
                                            const bool (&dif)[2], const double lref[3]) {
  const ProbDesc& pd = a.probs[pidx];
  const int nd = (dif[0] ? 1 : 0) + (k > 1 && dif[1] ? 1 : 0);
  const int nf = k - nd;
  auto lam4 = [&](const double* x) {
    return a.o.dim == 1 ? make_lam4(x[0], x[0], x[0]) : make_lam4(x[0], x[1], x[2]);
  };
  int64_t fs = 0, ds = 0;
  if (nf > 0) fs = pd.qff_off + atomic_add_warp(sd.fq_cnt + pidx, nf);
  if (nd > 0) ds = pd.qff_off + atomic_add_warp(sd.dq_cnt + pidx, nd);
  SI(a, I_RSLOT, g) = (int32_t)fs;
  SI(a, I_DSLOT, g) = (int32_t)ds;
  int tg = 0xffff;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (j >= k) break;
    const int id = j == 0 ? id0 : id1;
    if (dif[j]) {
      sd.dpos[ds] = pos;
      sd.dlam[ds] = lam4(l[j]);
      sd.dlam0[ds] = lam4(lref);
      ++ds;
    } else {
      sd.fpos[fs] = pos;
      sd.flam[fs] = lam4(l[j]);
      ++fs;
    }
    tg = (tg & ~(0xff << (8 * j))) | (((id | (dif[j] ? RT_DIF : 0)) & 0xff) << (8 * j));
  }
  SI(a, I_RTGT, g) = tg;
  sd.ref[atomic_add_warp(sd.ref_cnt, 1)] = (int32_t)g;
  if (a.stat_ties) atomicAdd(a.stat_ties, 1ull);
  if (nd > 0 && a.stat_difs) atomicAdd(a.stat_difs, (unsigned long long)nd);
}

// N: the number of free lambdas (3, or 1 when the components share one).
template <int N>
__global__ void solve_init_kernel(const SolveArgs a, const double* __restrict__ lam_init) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const float4 pos = a.ppos[g];
    const int pidx = __float_as_int(pos.w);
    constexpr int n = N;
    double lam[N + 1][3];
#pragma unroll
    for (int v = 0; v <= n; ++v)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double l0 = lam_init ? lam_init[3 * g + d] : 0.0;
        lam[v][d] = (d < n) ? l0 + ((v == d + 1) ? a.probs[pidx].step : 0.0) : 0.0;
      }
#pragma unroll
    for (int v = 0; v <= n; ++v)
#pragma unroll
      for (int d = 0; d < 3; ++d) SD(a, D_VL + v * 3 + d, g) = lam[v][d];
    SI(a, I_STAGE, g) = ST_INIT;
    SI(a, I_ITERS, g) = 0;
    SI(a, I_NFEV, g) = 0;
    SI(a, I_STATUS, g) = PT_RUNNING;
    SI(a, I_FLAGS, g) = 0;
    if (a.o.tie_dif > 0.0) SD(a, D_REFS, g) = __longlong_as_double(0x7ff8000000000000LL);  // NaN
    emit<N + 1>(a, g, pos, pidx, lam);
  }
}

void launch_solve_init(const SolveArgs& a, const double* lam_init, int grid, cudaStream_t s) {
  if (a.o.dim == 1) solve_init_kernel<1><<<grid, 256, 0, s>>>(a, lam_init);
  else solve_init_kernel<3><<<grid, 256, 0, s>>>(a, lam_init);
}

// Stable insertion sort of the N+1 vertices by Phi (ties keep their order), unrolled into
// adjacent compare-exchanges so the vertices stay in registers.  Without the early exit of the
// textbook loop the result is the same: after inserting each vertex no adjacent pair of the
// sorted prefix is out of order (v[j].phi < v[j-1].phi false), so the comparisons below the
// insertion point never swap.  The insertion's own comparisons (those down to the insertion
// point) go through the tie log; the ones below it decide nothing.
template <int N>
__device__ __forceinline__ void sort_verts(Vert* v, TieLog& tl) {
#pragma unroll
  for (int i = 1; i <= N; ++i) {
    bool moving = true;
#pragma unroll
    for (int j = i; j > 0; --j) {
      const bool sw = moving ? tl.lt(v[j], v[j - 1]) : v[j].phi < v[j - 1].phi;
      if (sw) {
        const Vert t = v[j];
        v[j] = v[j - 1];
        v[j - 1] = t;
      } else {
        moving = false;
      }
    }
  }
}

// One simplex step per waiting point.  REF = false: the points whose queries the mixed pass of
// this round evaluated (their results are read and their bounds computed); REF = true: the
// points whose near-tied values the float-float pass of this round re-evaluated (the values are
// replaced, bound 0, and the step is decided again).  A step is taken only when none of its
// comparisons is a near tie (TieLog); otherwise the step's inputs stay in the state and the
// near-tied values are queued for float-float re-evaluation, so every decision is the one that
// sums accurate to the float-float level would take.  With a.o.tie == 0 every step is taken as
// evaluated.
template <int N, bool REF>
__global__ void nm_step_kernel(const SolveArgs a) {
  const double rho = 1.0, chi = 2.0, psi = 0.5, sigma = 0.5;
  const int nact = REF ? *a.cur.ref_cnt : *a.cur.act_cnt;
  const int32_t* list = REF ? a.cur.ref : a.cur.act;
  constexpr int n = N;
  const PlanHdr h = *a.plan;
  PlanHdr hf{}, hd{};
  if (REF) {
    hf = *a.fplan;
    if (a.o.tie_dif > 0.0) hd = *a.dplan;
  }
  for (int ia = blockIdx.x * blockDim.x + threadIdx.x; ia < nact; ia += gridDim.x * blockDim.x) {
    const int64_t g = list[ia];
    const float4 pos = a.ppos[g];
    const int pidx = __float_as_int(pos.w);
    const double z = (double)pos.z;
    int stage = SI(a, I_STAGE, g);
    int iters = SI(a, I_ITERS, g);
    int nfev = SI(a, I_NFEV, g);
    int flags = SI(a, I_FLAGS, g);
    const bool single = stage != ST_INIT && stage != ST_SHRINK;

    Vert v[N + 1];
#pragma unroll
    for (int k = 0; k <= n; ++k) load_vert(a, g, k, v[k]);
    Vert e, R;
    e.id = VID_E;
    R.id = VID_R;
    bool vdirty = false, rdirty = false;

    if (!(flags & F_EVAL)) {
      // The pending queries' objectives, evaluated at one site for every stage: a warp whose
      // lanes are in different stages runs the FP64 objective once per query index instead of
      // once per stage.  The initial simplex (n + 1 queries into vertices 0..n) and a shrink
      // (n queries into vertices 1..n) fill vertices by shifting each result in at the top (no
      // run-time vertex index, so they stay in registers); the other stages read one trial point.
      const int64_t slot = SI(a, I_QSLOT, g);
      const int nev = stage == ST_INIT ? n + 1 : (stage == ST_SHRINK ? n : 1);
      const int first = stage == ST_SHRINK ? 1 : 0;
      for (int d = 0; d < 3; ++d) e.l[d] = single ? SD(a, D_TL + d, g) : 0.0;
#pragma unroll 1
      for (int k = 0; k < nev; ++k) {
        double lq[3];   // the query's lambda (read back from the state: a register-array
                        // index that depends on k would move the vertices to local memory)
        for (int d = 0; d < 3; ++d)
          lq[d] = single ? e.l[d] : SD(a, D_VL + 3 * (first + k) + d, g);
        Eval ev;
        read_eval(a, h, pidx, slot + k, z, ev, g, lq);
        if (!single) {
#pragma unroll
          for (int m = 0; m < n; ++m)
            if (m >= first) {
              for (int p = 0; p < 3; ++p) v[m].B[p] = v[m + 1].B[p];
              v[m].f = v[m + 1].f; v[m].g = v[m + 1].g; v[m].phi = v[m + 1].phi;
              v[m].s = v[m + 1].s;
            }
          set_value(v[n], ev);
        } else {
          set_value(e, ev);
        }
      }
      nfev += nev;
      vdirty = !single;
      flags |= F_EVAL;
    } else if (single) {
      load_e(a, g, e);
    }
    if (stage == ST_EXPAND || stage == ST_OCONTRACT) load_r(a, g, R);
    if (REF) {
      // apply the re-evaluated values of this point's targets: the differences first (they
      // were queued against the current reference), then the float-float values, each of which
      // becomes the point's reference
      const int tg = SI(a, I_RTGT, g);
      int64_t slot[2] = {SI(a, I_RSLOT, g), SI(a, I_DSLOT, g)};
#pragma unroll 1
      for (int it = 0; it < 4; ++it) {
        const int t = it & 1;
        const int code = (tg >> (8 * t)) & 0xff;
        if (code == 0xff) continue;
        const bool dif = (code & RT_DIF) != 0;
        if (dif != (it < 2)) continue;
        const int id = code & ~RT_DIF;
        Eval ev;
        double lt[3];
        for (int d = 0; d < 3; ++d)
          lt[d] = id == VID_E ? e.l[d] : (id == VID_R ? R.l[d] : SD(a, D_VL + 3 * id + d, g));
        if (dif) {
          read_eval_dif(a, hd, pidx, slot[1]++, z, ev, g, lt);
        } else {
          double S[12];
          read_eval_ff(a, hf, pidx, slot[0]++, z, ev, g, S);
          if (a.o.tie_dif > 0.0) {
            for (int d = 0; d < 3; ++d) SD(a, D_REFL + d, g) = lt[d];
            for (int s = 0; s < 12; ++s) SD(a, D_REFS + s, g) = S[s];
          }
        }
        if (id == VID_E) {
          set_value(e, ev);
        } else if (id == VID_R) {
          set_value(R, ev);
          rdirty = true;
        } else {
#pragma unroll
          for (int k = 0; k <= n; ++k)
            if (k == id) set_value(v[k], ev);
          vdirty = true;
        }
      }
    }

    // ---- the step.  With certified decisions the vertices the step starts from are in memory
    // first (the step may turn out to wait), and nothing else is written until the step is
    // known to be certain.
    TieLog tl{a.o.tie, a.o.tie_dif, -1, -1};
    if (vdirty && a.o.tie > 0.0)
#pragma unroll
      for (int m = 0; m <= n; ++m) store_vert(a, g, m, v[m]);
    Vert (&w)[N + 1] = v;
    bool to_check = false, accepted = false, store_R = false, emit_shrink = false;
    bool emit_trial = false, mirror = false;
    int next_stage = stage;
    double xt[3] = {0.0, 0.0, 0.0};
    char code = 0;
    int fin = -1;
    auto trial = [&](double coef_c, double coef_w, double out[3]) {  // coef_c c + coef_w w[n]
      double c[3];
#pragma unroll
      for (int d = 0; d < n; ++d) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) s += w[k].l[d];
        c[d] = s / n;
      }
      for (int d = 0; d < 3; ++d) out[d] = (d < n) ? coef_c * c[d] + coef_w * w[n].l[d] : 0.0;
    };

    if (stage == ST_INIT) {
      to_check = true;
    } else if (stage == ST_REFLECT) {
      if (tl.lt(e, w[0])) {
        store_R = true;
        trial(1.0 + rho * chi, -(rho * chi), xt);
        next_stage = ST_EXPAND;
        emit_trial = true;
      } else if (tl.lt(e, w[n - 1])) {
        w[n] = e;
        accepted = true;
        code = 'R';
        to_check = true;
      } else if (tl.lt(e, w[n])) {
        store_R = true;
        trial(1.0 + psi * rho, -(psi * rho), xt);
        next_stage = ST_OCONTRACT;
        emit_trial = true;
      } else {
        trial(1.0 - psi, psi, xt);
        next_stage = ST_ICONTRACT;
        emit_trial = true;
      }
    } else if (stage == ST_EXPAND) {
      if (tl.lt(e, R)) {
        w[n] = e;
        code = 'E';
      } else {
        w[n] = R;
        code = 'R';
      }
      accepted = true;
      to_check = true;
    } else if (stage == ST_OCONTRACT || stage == ST_ICONTRACT) {
      const bool ok = (stage == ST_OCONTRACT) ? tl.le(e, R) : tl.lt(e, w[n]);
      if (ok) {
        w[n] = e;
        accepted = true;
        code = (stage == ST_OCONTRACT) ? 'O' : 'I';
        to_check = true;
      } else {
#pragma unroll
        for (int k = 1; k <= n; ++k)
          for (int d = 0; d < 3; ++d)
            w[k].l[d] = (d < n) ? w[0].l[d] + sigma * (w[k].l[d] - w[0].l[d]) : 0.0;
        next_stage = ST_SHRINK;
        emit_shrink = true;
      }
    } else if (stage == ST_SHRINK) {
      code = 'S';
      to_check = true;
    }
    if (to_check) {
      sort_verts<N>(w, tl);
      // Eq. 12 at the best vertex, then the value spread, then the iteration count
      tl.note(w[0].id, w[0].s, -1, 0.0, w[0].f - a.o.eps_f);
      if (w[0].f <= a.o.eps_f) tl.note(w[0].id, w[0].s, -1, 0.0, w[0].g - a.o.eps_g);
      if (w[0].f <= a.o.eps_f && w[0].g <= a.o.eps_g) {
        fin = PT_CONVERGED;
      } else {
        tl.note(w[n].id, w[n].s, w[0].id, w[0].s, w[n].phi - w[0].phi - a.o.tol);
        if (w[n].phi - w[0].phi <= a.o.tol) fin = PT_CONVERGED;
        else if (iters >= a.o.max_iter) fin = PT_MAXITER;
      }
      if (fin < 0) {
        if (n == 1 && w[0].l[0] == 0.0) {
          // Mirror step: with the best vertex at lambda = 0 the reflection is -w[1], where Phi
          // (even in lambda, Eq. 6) takes w[1]'s value exactly.  Its comparisons are settled
          // (not below w[0], by the sort just done; not below w[1], by equality), so the step
          // goes straight to the inside contraction, and the reflection is counted as the
          // evaluation the search makes.  Every form then decides these exact ties as exact
          // arithmetic does, instead of by the rounding of two sums.
          trial(1.0 - psi, psi, xt);
          next_stage = ST_ICONTRACT;
          mirror = true;
        } else {
          trial(1.0 + rho, -rho, xt);
          next_stage = ST_REFLECT;
        }
        emit_trial = true;
      }
    }

    if (tl.a >= 0) {
      // near tie: keep the step's inputs and re-evaluate the near-tied values in float-float
      // (tl.a >= 0 always; tl.b >= 0 when both values carry a bound).  A vertex target's lambda
      // comes from the stored state the step started from.
      double lt[2][3];
      const int ida = tl.a, idb = tl.b;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        lt[0][d] = ida == VID_E ? e.l[d] : (ida == VID_R ? R.l[d] : SD(a, D_VL + 3 * ida + d, g));
        lt[1][d] = idb < 0 ? 0.0 : idb == VID_E ? e.l[d]
                 : (idb == VID_R ? R.l[d] : SD(a, D_VL + 3 * idb + d, g));
      }
      // A value goes to the difference pass when the point has a float-float reference, the
      // value still carries its mixed-form bound and it lies near the reference (the difference
      // bound, relative to the mixed one, grows as |lambda - lambda_ref| times the point's mean
      // pixel distance sum |b| / sum |b| / r: estimated below about 0.5 here); otherwise to
      // float-float.  Without a reference only the value with the larger bound goes to
      // float-float: it becomes the reference, and the other value, if still near-tied, goes
      // to the difference pass in the next round.
      int k = idb >= 0 ? 2 : 1;
      int id0 = ida, id1 = idb;
      bool dif[2] = {false, false};
      double lref[3] = {0.0, 0.0, 0.0};
      if (a.o.tie_dif > 0.0) {
        const double sv[2] = {
            ida == VID_E ? e.s : (ida == VID_R ? R.s : SD(a, D_VS + ida, g)),
            idb < 0 ? 0.0 : idb == VID_E ? e.s : (idb == VID_R ? R.s : SD(a, D_VS + idb, g))};
        if (!isnan(SD(a, D_REFS, g))) {
#pragma unroll
          for (int d = 0; d < 3; ++d) lref[d] = SD(a, D_REFL + d, g);
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            bool near = j < k && sv[j] > 0.0;
#pragma unroll
            for (int p = 0; p < 3; ++p) {
              const int q = n == 1 ? 0 : p;
              const double m1 = a.msc[15 * g + 5 * p];
              const double reach = m1 > 0.0 ? a.msc0[3 * g + p] / m1 : 0.0;
              near = near && fabs(lt[j][q] - lref[q]) * reach < 0.25;
            }
            dif[j] = near;
          }
        } else if (k == 2 && sv[0] > 0.0 && sv[1] > 0.0) {
          k = 1;
          if (sv[1] > sv[0]) {
            id0 = idb;
#pragma unroll
            for (int d = 0; d < 3; ++d) lt[0][d] = lt[1][d];
          }
        }
      }
      emit_reeval(a, REF ? a.nxt : a.cur, g, pos, pidx, k, lt, id0, id1, dif, lref);
      if (single) store_e(a, g, e);
      if (rdirty) store_r(a, g, R);
      SI(a, I_FLAGS, g) = flags;
      SI(a, I_NFEV, g) = nfev;
      continue;
    }

    // ---- the step is certain: take it
    if (rdirty && !store_R) store_r(a, g, R);
    if (store_R) {
      Vert r = e;
      store_r(a, g, r);
    }
    if (code && a.codes && iters >= 1 && iters <= a.codes_stride)
      a.codes[g * a.codes_stride + (iters - 1)] = code;
    if (fin >= 0) {
      for (int p = 0; p < 3; ++p) {
        a.res_B[3 * g + p] = w[0].B[p];
        a.res_lam[3 * g + p] = fabs(n == 1 ? w[0].l[0] : w[0].l[p]);
      }
      a.res_f[g] = w[0].f;
      a.res_g[g] = w[0].g;
      a.res_iters[g] = iters;
      a.res_status[g] = fin;
      a.res_nfev[g] = nfev;
      stage = ST_DONE;
      SI(a, I_STATUS, g) = fin;
    } else {
      if (to_check) iters += 1;
      if (mirror) nfev += 1;
      if (emit_trial) {
        double rows[1][3] = {{xt[0], xt[1], xt[2]}};
        for (int d = 0; d < 3; ++d) SD(a, D_TL + d, g) = xt[d];
        emit<1>(a, g, pos, pidx, rows);
      } else if (emit_shrink) {
        double rows[N][3];
#pragma unroll
        for (int k = 1; k <= n; ++k)
          for (int d = 0; d < 3; ++d) rows[k - 1][d] = w[k].l[d];
        emit<N>(a, g, pos, pidx, rows);
      }
      stage = next_stage;
      // a finished point's vertices are not read again; otherwise store what changed
      if (vdirty || to_check || accepted || emit_shrink)
#pragma unroll
        for (int k = 0; k <= n; ++k) store_vert(a, g, k, w[k]);
    }
    SI(a, I_STAGE, g) = stage;
    SI(a, I_ITERS, g) = iters;
    SI(a, I_NFEV, g) = nfev;
    SI(a, I_FLAGS, g) = 0;
  }
}

void launch_nm_step(const SolveArgs& a, int grid, cudaStream_t s) {
  if (a.o.dim == 1) nm_step_kernel<1, false><<<grid, 128, 0, s>>>(a);
  else nm_step_kernel<3, false><<<grid, 128, 0, s>>>(a);
}
void launch_nm_refine(const SolveArgs& a, int grid, cudaStream_t s) {
  if (a.o.dim == 1) nm_step_kernel<1, true><<<grid, 128, 0, s>>>(a);
  else nm_step_kernel<3, true><<<grid, 128, 0, s>>>(a);
}

// --------------------------------------------------------------- per-round plan ----
__global__ void plan_round_kernel(const PlanArgs a) {
  __shared__ long long s_blocks;
  __shared__ int s_minTiles;
  if (threadIdx.x == 0) {
    s_blocks = 0;
    s_minTiles = 1 << 30;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < a.nprob; p += blockDim.x) {
    const int q = a.q_cnt_cur[p];
    a.q_cnt_pass[p] = q;
    if (q > 0) {
      atomicAdd((unsigned long long*)&s_blocks, (unsigned long long)((q + a.qper - 1) / a.qper));
      atomicMin(&s_minTiles, a.probs[p].ntiles);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long blocks = s_blocks;
    int nsplit = 1;
    if (blocks > 0 && blocks < a.target_items) {
      nsplit = (int)((a.target_items + blocks - 1) / blocks);
      if (nsplit > a.nsplit_cap) nsplit = a.nsplit_cap;
      if (nsplit > s_minTiles) nsplit = s_minTiles;
      if (nsplit < 1) nsplit = 1;
    }
    int acc = 0;
    double pairs = 0.0;
    unsigned long long queries = 0;
    for (int p = 0; p < a.nprob; ++p) {
      a.item_off[p] = acc;
      const int q = a.q_cnt_pass[p];
      acc += ((q + a.qper - 1) / a.qper) * nsplit;
      pairs += (double)q * (double)(a.probs[p].nx) * (double)(a.probs[p].ny);
      queries += (unsigned long long)q;
    }
    a.item_off[a.nprob] = acc;
    PlanHdr h;
    h.nitems = acc;
    h.nsplit = nsplit;
    h.qper = a.qper;
    h.pad0 = 0;
    *a.plan = h;
    *a.work = 0;
    // the plan of a float-float re-evaluation pass leaves the next round's counters alone
    if (a.act_cnt_nxt) *a.act_cnt_nxt = 0;
    if (a.near_cnt_nxt) *a.near_cnt_nxt = 0;
    if (a.ref_cnt_nxt) *a.ref_cnt_nxt = 0;
    if (a.round_ctr) *a.round_ctr += 1;
    if (a.stat_queries) *a.stat_queries += queries;
    if (a.stat_pairs) *a.stat_pairs += pairs;
  }
  for (int p = threadIdx.x; p < a.nprob; p += blockDim.x) {
    if (a.q_cnt_nxt) a.q_cnt_nxt[p] = 0;
    if (a.fq_cnt_nxt) a.fq_cnt_nxt[p] = 0;
    if (a.dq_cnt_nxt) a.dq_cnt_nxt[p] = 0;
  }
}

void launch_plan_round(const PlanArgs& a, cudaStream_t s) { plan_round_kernel<<<1, 256, 0, s>>>(a); }

// The lambda-independent absolute-value sums of every point, the coefficients of the mixed
// form's error bound: msc[15 g + 5 p + j - 1] = sum_k |b_pk| / r_gk^j, j = 1..5, over the
// quadrature points of the point's problem.  FP32 terms summed per tile, tiles summed in FP64
// (relative error below 1e-4: a scale, not a result).
__global__ void msc_kernel(const ProbDesc* __restrict__ probs, int64_t N,
                           const float4* __restrict__ ppos, double* __restrict__ msc,
                           double* __restrict__ msc0) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const float4 pos = ppos[g];
    const ProbDesc& pd = probs[__float_as_int(pos.w)];
    const float z2 = __fmul_rn(pos.z, pos.z);
    double tot[15], tot0[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 15; ++i) tot[i] = 0.0;
    for (int t = 0; t < pd.ntiles; ++t) {
      const float* T = pd.tiles32 + (int64_t)t * pd.nf32 * TILE;
      float acc[15], acc0[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < 15; ++i) acc[i] = 0.f;
#pragma unroll 2
      for (int e = 0; e < TILE; ++e) {
        const float dx = pos.x - __ldg(T + e), dy = pos.y - __ldg(T + TILE + e);
        const float ri = rsqrtf(dx * dx + dy * dy + z2);
        const float b[3] = {fabsf(__ldg(T + 2 * TILE + e)), fabsf(__ldg(T + 3 * TILE + e)),
                            fabsf(__ldg(T + 4 * TILE + e))};
#pragma unroll
        for (int p = 0; p < 3; ++p) acc0[p] += b[p];
        float wj = ri;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
#pragma unroll
          for (int p = 0; p < 3; ++p) acc[5 * p + j] += b[p] * wj;
          wj *= ri;
        }
      }
#pragma unroll
      for (int i = 0; i < 15; ++i) tot[i] += (double)acc[i];
#pragma unroll
      for (int p = 0; p < 3; ++p) tot0[p] += (double)acc0[p];
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) msc[15 * g + i] = tot[i];
    if (msc0)
#pragma unroll
      for (int p = 0; p < 3; ++p) msc0[3 * g + p] = tot0[p];
  }
}

void launch_msc(const ProbDesc* probs, int64_t N, const float4* ppos, double* msc, double* msc0,
                int grid, cudaStream_t s) {
  if (N > 0) msc_kernel<<<grid, 128, 0, s>>>(probs, N, ppos, msc, msc0);
}

// Difference sums of n queries of one problem (slots 0..n-1) and their bounds (debug entry).
__global__ void dif_debug_kernel(int64_t n, const PlanHdr* __restrict__ plan,
                                 const int32_t* __restrict__ item_off,
                                 const double* __restrict__ out, const Lam4* __restrict__ qlam,
                                 const Lam4* __restrict__ qlam0, const double* __restrict__ msc,
                                 const double* __restrict__ msc0, int dim, double* dS,
                                 double* dS_bound) {
  const PlanHdr h = *plan;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int s = 0; s < 12; ++s) dS[12 * i + s] = gather_sum(out, h, item_off, 0, i, 12, s);
    if (dS_bound) {
      const double la[3] = {qlam[i].x, qlam[i].y, qlam[i].z};
      const double l0[3] = {qlam0[i].x, qlam0[i].y, qlam0[i].z};
      double e[12];
      dif_sum_bounds(msc + 15 * i, msc0 + 3 * i, la, l0, dim, e);
      for (int s = 0; s < 12; ++s) dS_bound[12 * i + s] = e[s];
    }
  }
}

void launch_dif_debug(int64_t n, const PlanHdr* plan, const int32_t* item_off, const double* out,
                      const Lam4* qlam, const Lam4* qlam0, const double* msc, const double* msc0,
                      int dim, double* dS, double* dS_bound, cudaStream_t s) {
  const int64_t nb = (n + 127) / 128;
  if (n > 0)
    dif_debug_kernel<<<(int)(nb < 1024 ? nb : 1024), 128, 0, s>>>(
        n, plan, item_off, out, qlam, qlam0, msc, msc0, dim, dS, dS_bound);
}

// ------------------------------------------------------------------ certified B ----
// Worst-case error of the mixed form's B at lambda (the B part of mixed_phi_bound): per
// component z (A0 M3 + A1 |lambda| M2 + A2 lambda^2 M1); returns the Euclidean norm.
__device__ __forceinline__ double mixed_b_bound(const double* M, const double lam[3], int dim,
                                                double z) {
  double s = 0.0;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const double L = fabs(dim == 1 ? lam[0] : lam[p]);
    const double* m = M + 5 * p;
    const double d = z * (BND_A0 * m[2] + BND_A1 * L * m[1] + BND_A2 * L * L * m[0]);
    s += d * d;
  }
  return sqrt(s);
}

// After a certified search: every point whose final B the bound does not certify to `rel`
// relative (the cancellation-dominated points) queues a float-float value query at lambda* on
// side cur and joins cur's waiting list.
__global__ void certb_flag_kernel(const SolveArgs a, double rel) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const float4 pos = a.ppos[g];
    const int pidx = __float_as_int(pos.w);
    const double lam[3] = {a.res_lam[3 * g], a.res_lam[3 * g + 1], a.res_lam[3 * g + 2]};
    const double* B = a.res_B + 3 * g;
    const double nB = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    if (!(mixed_b_bound(a.msc + 15 * g, lam, a.o.dim, (double)pos.z) > rel * nB)) continue;
    const ProbDesc& pd = a.probs[pidx];
    const int base = atomic_add_warp(a.cur.fq_cnt + pidx, 1);
    const int64_t slot = pd.qff_off + base;
    a.cur.fpos[slot] = pos;
    a.cur.flam[slot] = make_lam4(lam[0], lam[1], lam[2]);
    SI(a, I_RSLOT, g) = (int32_t)slot;
    a.cur.ref[atomic_add_warp(a.cur.ref_cnt, 1)] = (int32_t)g;
  }
}

// B of the queued points from the float-float value sums (3 per query).
__global__ void certb_apply_kernel(const SolveArgs a) {
  const int n = *a.cur.ref_cnt;
  const PlanHdr hf = *a.fplan;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int64_t g = a.cur.ref[i];
    const float4 pos = a.ppos[g];
    const int pidx = __float_as_int(pos.w);
    const ProbDesc& pd = a.probs[pidx];
    const double z = (double)pos.z;
    const int64_t j = (int64_t)SI(a, I_RSLOT, g) - pd.qff_off;
    const double* corr = corr_of(a, pd, g, z);
    for (int p = 0; p < 3; ++p)
      a.res_B[3 * g + p] = z * gather_sum(a.fout, hf, a.fitem_off, pidx, j, 3, p) +
                           (corr ? corr[p] : 0.0);
  }
}

void launch_certb_flag(const SolveArgs& a, double rel, int grid, cudaStream_t s) {
  certb_flag_kernel<<<grid, 128, 0, s>>>(a, rel);
}
void launch_certb_apply(const SolveArgs& a, int grid, cudaStream_t s) {
  certb_apply_kernel<<<grid, 128, 0, s>>>(a);
}

}  // namespace dbie

// ======================================================= objective gradient, quasi-Newton ----
namespace dbie {

// Phi and dPhi/dlambda_q from the 21 sums of VAR_OBJN (per component: S0, S1, Sx, Sy, Sl, Tx, Ty).
// lambda_q moves only component q: dB_q = z lambda Sl, d(dB_q/dx) = -z lambda Tx,
// d(dB_q/dy) = -z lambda Ty, d(dB_q/dz) = lambda Sl - z^2 lambda S0; the rest is the chain rule
// through J = curl B, div B and the norms (kinks of f and g contribute 0).
__device__ void objective_grad(const double* S, double z, const double lam[3], double g_scale,
                               double w_g, Eval& e, double dphi[3], const double* corr) {
  double G[9], dBdl[3], dGdl[9];
  for (int p = 0; p < 3; ++p) {
    const double* s = S + 7 * p;
    e.B[p] = z * s[0];
    G[3 * p + 0] = z * s[2];
    G[3 * p + 1] = z * s[3];
    G[3 * p + 2] = s[0] + z * z * s[1];
    dBdl[p] = z * lam[p] * s[4];
    dGdl[3 * p + 0] = -(z * lam[p] * s[5]);
    dGdl[3 * p + 1] = -(z * lam[p] * s[6]);
    dGdl[3 * p + 2] = lam[p] * s[4] - z * z * lam[p] * s[0];
  }
  add_corr(corr, e.B, G);
  objective(e.B, G, g_scale, w_g, e.f, e.g, e.phi);
  const double* B = e.B;
  const double J[3] = {G[3 * 2 + 1] - G[3 * 1 + 2], G[3 * 0 + 2] - G[3 * 2 + 0],
                       G[3 * 1 + 0] - G[3 * 0 + 1]};
  const double D = G[0] + G[4] + G[8];
  const double C[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2],
                       J[0] * B[1] - J[1] * B[0]};
  const double nJ = sqrt(J[0] * J[0] + J[1] * J[1] + J[2] * J[2]);
  const double nB = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  const double nC = sqrt(C[0] * C[0] + C[1] * C[1] + C[2] * C[2]);
  for (int q = 0; q < 3; ++q) {
    double dB[3] = {0, 0, 0}, dG[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    dB[q] = dBdl[q];
    for (int j = 0; j < 3; ++j) dG[3 * q + j] = dGdl[3 * q + j];
    const double dJ[3] = {dG[3 * 2 + 1] - dG[3 * 1 + 2], dG[3 * 0 + 2] - dG[3 * 2 + 0],
                          dG[3 * 1 + 0] - dG[3 * 0 + 1]};
    const double dD = dG[0] + dG[4] + dG[8];
    const double dC[3] = {dJ[1] * B[2] - dJ[2] * B[1] + J[1] * dB[2] - J[2] * dB[1],
                          dJ[2] * B[0] - dJ[0] * B[2] + J[2] * dB[0] - J[0] * dB[2],
                          dJ[0] * B[1] - dJ[1] * B[0] + J[0] * dB[1] - J[1] * dB[0]};
    double df = 0.0, dg = 0.0;
    if (nJ * nB > 0.0) {
      const double JdJ = J[0] * dJ[0] + J[1] * dJ[1] + J[2] * dJ[2];
      const double BdB = B[0] * dB[0] + B[1] * dB[1] + B[2] * dB[2];
      const double CdC = C[0] * dC[0] + C[1] * dC[1] + C[2] * dC[2];
      df = (nC > 0.0 ? CdC / (nC * nJ * nB) : 0.0) - e.f * (JdJ / (nJ * nJ) + BdB / (nB * nB));
    }
    if (nB > 0.0) {
      const double BdB = B[0] * dB[0] + B[1] * dB[1] + B[2] * dB[2];
      const double sgn = D > 0.0 ? 1.0 : (D < 0.0 ? -1.0 : 0.0);
      dg = g_scale * (sgn * dD / nB - fabs(D) * BdB / (nB * nB * nB));
    }
    dphi[q] = df + w_g * dg;
  }
}

__global__ void finalize_objective_kernel(int64_t n, const PlanHdr* __restrict__ plan,
                                          const int32_t* __restrict__ item_off,
                                          const double* __restrict__ out,
                                          const float4* __restrict__ qpos,
                                          const Lam4* __restrict__ qlam, double g_scale,
                                          double w_g, double* fgphi, double* dphi, double* B,
                                          const double* corr) {
  const PlanHdr h = *plan;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double S[21];
#pragma unroll
    for (int s = 0; s < 21; ++s) S[s] = gather_sum(out, h, item_off, 0, i, 21, s);
    const Lam4 l = qlam[i];
    const double lam[3] = {l.x, l.y, l.z};
    Eval e;
    double dp[3];
    objective_grad(S, (double)qpos[i].z, lam, g_scale, w_g, e, dp, corr ? corr + 12 * i : nullptr);
    if (fgphi) {
      fgphi[3 * i] = e.f;
      fgphi[3 * i + 1] = e.g;
      fgphi[3 * i + 2] = e.phi;
    }
    if (dphi)
      for (int q = 0; q < 3; ++q) dphi[3 * i + q] = dp[q];
    if (B)
      for (int p = 0; p < 3; ++p) B[3 * i + p] = e.B[p];
  }
}

void launch_finalize_objective(int64_t n, const PlanHdr* plan, const int32_t* item_off,
                               const double* out, const float4* qpos, const Lam4* qlam,
                               double g_scale, double w_g, double* fgphi, double* dphi, double* B,
                               const double* corr, cudaStream_t s) {
  if (n <= 0) return;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  finalize_objective_kernel<<<grid, 256, 0, s>>>(n, plan, item_off, out, qpos, qlam, g_scale,
                                                 w_g, fgphi, dphi, B, corr);
}

// ----------------------------------------------------------------------- quasi-Newton ----
// Same algorithm, same order of operations as the oracle's orc_bfgs (this file is compiled
// without FMA contraction): one line-search trial per point per round.

__global__ void bfgs_init_kernel(const SolveArgs a, const double* __restrict__ lam_init) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const float4 pos = a.ppos[g];
    const int pidx = __float_as_int(pos.w);
    const int n = a.o.dim;
    // Phi is even in every lambda_p, so lambda = 0 is a stationary point: start one step away
    // from the initial lambda along (1, 1, 1).
    double x[1][3];
    for (int d = 0; d < 3; ++d) {
      x[0][d] = d < n ? (lam_init ? lam_init[3 * g + d] : 0.0) + a.probs[pidx].step : 0.0;
      SD(a, B_X + d, g) = x[0][d];
    }
    SI(a, I_STAGE, g) = ST_BF_INIT;
    SI(a, I_ITERS, g) = 0;
    SI(a, I_NFEV, g) = 0;
    SI(a, I_STATUS, g) = PT_RUNNING;
    emit<1>(a, g, pos, pidx, x);
  }
}

void launch_bfgs_init(const SolveArgs& a, const double* lam_init, int grid, cudaStream_t s) {
  bfgs_init_kernel<<<grid, 256, 0, s>>>(a, lam_init);
}

// N: the number of free lambdas (3, or 1 when the components share one); fixed at compile time
// so the per-point state stays in registers.
template <int N>
__global__ void bfgs_step_kernel(const SolveArgs a) {
  const int nact = *a.cur.act_cnt;
  constexpr int n = N;
  const PlanHdr h = *a.plan;
  for (int ia = blockIdx.x * blockDim.x + threadIdx.x; ia < nact; ia += gridDim.x * blockDim.x) {
    const int64_t g = a.cur.act[ia];
    const float4 pos = a.ppos[g];
    const int pidx = __float_as_int(pos.w);
    const ProbDesc& pd = a.probs[pidx];
    const double z = (double)pos.z;
    const int stage = SI(a, I_STAGE, g);
    int iters = SI(a, I_ITERS, g);
    int nfev = SI(a, I_NFEV, g) + 1;
    double x[3], gr[3], H[9], dv[3], B[3];
    for (int i = 0; i < 3; ++i) {
      x[i] = SD(a, B_X + i, g);
      gr[i] = SD(a, B_GR + i, g);
      dv[i] = SD(a, B_D + i, g);
      B[i] = SD(a, B_B + i, g);
    }
    for (int i = 0; i < 9; ++i) H[i] = SD(a, B_H + i, g);
    double F = SD(a, B_PHI, g), fv = SD(a, B_F, g), gv = SD(a, B_G, g);
    double alpha = SD(a, B_ALPHA, g), gd = SD(a, B_GD, g), gn = SD(a, B_GN, g);

    // the pending trial's objective and gradient
    double xt[3] = {0, 0, 0};
    if (stage == ST_BF_INIT) {
      for (int i = 0; i < n; ++i) xt[i] = x[i];
    } else {
      for (int i = 0; i < n; ++i) xt[i] = x[i] + alpha * dv[i];
    }
    const double lamt[3] = {xt[0], n == 1 ? xt[0] : xt[1], n == 1 ? xt[0] : xt[2]};
    double S[21];
    const int64_t j = (int64_t)SI(a, I_QSLOT, g) - pd.q_off;
#pragma unroll
    for (int s = 0; s < 21; ++s) S[s] = gather_sum(a.out, h, a.item_off, pidx, j, 21, s);
    Eval e;
    double dp[3], gt[3] = {0, 0, 0};
    objective_grad(S, z, lamt, pd.g_scale, a.o.w_g, e, dp, corr_of(a, pd, g, z));
    if (n == 1) gt[0] = dp[0] + dp[1] + dp[2];
    else { gt[0] = dp[0]; gt[1] = dp[1]; gt[2] = dp[2]; }
    const bool flagt = e.f <= a.o.eps_f && e.g <= a.o.eps_g;

    int fin = -1;  // final status, or -1 to continue
    bool flag = false;
    bool need_dir = false;
    if (stage == ST_BF_INIT) {
      for (int i = 0; i < 3; ++i) { gr[i] = gt[i]; B[i] = e.B[i]; }
      F = e.phi; fv = e.f; gv = e.g; flag = flagt;
      gn = 0.0;
      for (int i = 0; i < n; ++i) gn += gr[i] * gr[i];
      gn = sqrt(gn);
      for (int i = 0; i < 9; ++i) H[i] = 0.0;
      if (gn > 0.0)
        for (int i = 0; i < n; ++i) H[3 * i + i] = pd.step / gn;
      need_dir = true;
    } else if (e.phi <= F + 1e-4 * alpha * gd) {  // Armijo: accept the trial
      iters += 1;
      double sv[3] = {0, 0, 0}, yv[3] = {0, 0, 0}, sy = 0.0, ss = 0.0, yy = 0.0;
      for (int i = 0; i < n; ++i) {
        sv[i] = xt[i] - x[i];
        yv[i] = gt[i] - gr[i];
        sy += sv[i] * yv[i];
        ss += sv[i] * sv[i];
        yy += yv[i] * yv[i];
      }
      if (sy > 1e-12 * sqrt(ss) * sqrt(yy)) {
        const double rho = 1.0 / sy;
        double Hy[3] = {0, 0, 0}, yHy = 0.0;
        for (int i = 0; i < n; ++i) {
          double t = 0.0;
          for (int k = 0; k < n; ++k) t += H[3 * i + k] * yv[k];
          Hy[i] = t;
        }
        for (int i = 0; i < n; ++i) yHy += yv[i] * Hy[i];
        const double c2 = rho * rho * yHy + rho;
        for (int i = 0; i < n; ++i)
          for (int k = 0; k < n; ++k)
            H[3 * i + k] = H[3 * i + k] - rho * (sv[i] * Hy[k] + Hy[i] * sv[k]) + c2 * sv[i] * sv[k];
      }
      const double dec = F - e.phi;
      for (int i = 0; i < n; ++i) { x[i] = xt[i]; gr[i] = gt[i]; }
      for (int i = 0; i < 3; ++i) B[i] = e.B[i];
      F = e.phi; fv = e.f; gv = e.g; flag = flagt;
      gn = 0.0;
      for (int i = 0; i < n; ++i) gn += gr[i] * gr[i];
      gn = sqrt(gn);
      if (dec <= a.o.tol) fin = PT_CONVERGED;
      else need_dir = true;
    } else {  // reject: halve the step (at most 31 trials per line search)
      alpha = 0.5 * alpha;
      if (alpha < 9.313225746154785e-10) fin = PT_CONVERGED;  // 2^-30
      else {
        double row[1][3] = {{0, 0, 0}};
        for (int i = 0; i < n; ++i) row[0][i] = x[i] + alpha * dv[i];
        SD(a, B_ALPHA, g) = alpha;
        SI(a, I_NFEV, g) = nfev;
        emit<1>(a, g, pos, pidx, row);
        continue;
      }
    }
    if (need_dir) {
      if (flag) fin = PT_CONVERGED;
      else if (!(gn > 0.0)) fin = PT_CONVERGED;
      else if (iters >= a.o.max_iter) fin = PT_MAXITER;
      else {
        for (int i = 0; i < n; ++i) {
          double s = 0.0;
          for (int k = 0; k < n; ++k) s += H[3 * i + k] * gr[k];
          dv[i] = -s;
        }
        gd = 0.0;
        for (int i = 0; i < n; ++i) gd += gr[i] * dv[i];
        if (!(gd < 0.0)) {
          for (int i = 0; i < 9; ++i) H[i] = 0.0;
          for (int i = 0; i < n; ++i) H[3 * i + i] = pd.step / gn;
          gd = 0.0;
          for (int i = 0; i < n; ++i) { dv[i] = -(H[3 * i + i] * gr[i]); gd += gr[i] * dv[i]; }
        }
        alpha = 1.0;
        double row[1][3] = {{0, 0, 0}};
        for (int i = 0; i < n; ++i) row[0][i] = x[i] + alpha * dv[i];
        emit<1>(a, g, pos, pidx, row);
      }
    }
    if (fin >= 0) {
      for (int p = 0; p < 3; ++p) {
        a.res_B[3 * g + p] = B[p];
        a.res_lam[3 * g + p] = fabs(n == 1 ? x[0] : x[p]);
      }
      a.res_f[g] = fv;
      a.res_g[g] = gv;
      a.res_iters[g] = iters;
      a.res_status[g] = fin;
      a.res_nfev[g] = nfev;
      SI(a, I_STATUS, g) = fin;
    }
    for (int i = 0; i < 3; ++i) {
      SD(a, B_X + i, g) = x[i];
      SD(a, B_GR + i, g) = gr[i];
      SD(a, B_D + i, g) = dv[i];
      SD(a, B_B + i, g) = B[i];
    }
    for (int i = 0; i < 9; ++i) SD(a, B_H + i, g) = H[i];
    SD(a, B_PHI, g) = F;
    SD(a, B_F, g) = fv;
    SD(a, B_G, g) = gv;
    SD(a, B_ALPHA, g) = alpha;
    SD(a, B_GD, g) = gd;
    SD(a, B_GN, g) = gn;
    SI(a, I_STAGE, g) = fin >= 0 ? ST_DONE : ST_BF_LS;
    SI(a, I_ITERS, g) = iters;
    SI(a, I_NFEV, g) = nfev;
  }
}

void launch_bfgs_step(const SolveArgs& a, int grid, cudaStream_t s) {
  if (a.o.dim == 1) bfgs_step_kernel<1><<<grid, 128, 0, s>>>(a);
  else bfgs_step_kernel<3><<<grid, 128, 0, s>>>(a);
}

}  // namespace dbie
