// second_order.cu -- lambda-Hessian of the objective, the gradient of a loss through the lambda
// search, and the noise variance of B (none of them in the paper).
//
// Compiled with -fmad=false: every operation is rounded as written.
//
// From the ten sums of the Hessian pass (per component p, lambda = lambda_p):
//   q       : B = z S0, Gx = z Sx, Gy = z Sy, Gz = S0 + z^2 S1            (Eq. 16, Eq. 13)
//   dq/dl   : z l Sl, -z l Tx, -z l Ty, l Sl - z^2 l S0
//   d2q/dl2 : z (Sl - l Q), -z (Tx + l^2 Ux), -z (Ty + l^2 Uy), (Sl - l Q) - z^2 (S0 + l^2 Sl)
// (dS0/dl = l Sl, dS1/dl = -l S0, dSx/dl = -l Tx, dSl/dl = -Q, dTx/dl = l Ux).  Phi = f + w_g g
// (Eq. 8, 9, 14) depends on lambda only through the twelve q, and q_m only on the lambda of its
// own component, so with F = dPhi/dq, P = d2Phi/dq2 and the 12 x dim matrix D of dq/dlambda,
//   grad_l Phi = D^T F,   H = D^T P D + diag_j(sum over q of component j of F d2q/dl_j^2).
// F comes from the closed-form gradient of Phi (reverse mode, written out below), and P D from
// the same gradient evaluated once on dual numbers that carry one tangent of q per column of D
// (three tangents, or one for a shared lambda).
//
// Gradient through the search: lambda* is a stationary point, grad_l Phi(lambda*; B0) = 0, so
// d(lambda*)/dB0 = -H^-1 d(grad_l Phi)/dB0 and
//   dL/dB0 = A^T gB - d/dB0 [v . grad_l Phi],  v = H^-1 dL/dl,  dL/dl_p = gB_p dB_p/dl_p.
// The second term is a transposed sum over points of seven kernel functions per component with
// per-point weights (vjp7_kernel); the weights need F and P (D v) = sum_k v_k (P D)_k, which the
// Hessian's columns already hold.
#include "kernels.h"
#include "solve.cuh"

namespace dbie {

namespace {

// Dual number with K tangents, v + sum_k d_k e_k (e_j e_k = 0): a value and its derivatives
// along K directions at once (the value arithmetic, square roots and divisions done once).
template <int K>
struct Du {
  double v, d[K];
};
template <int K>
__device__ __forceinline__ Du<K> operator+(const Du<K>& x, const Du<K>& y) {
  Du<K> r{x.v + y.v, {}};
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = x.d[k] + y.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Du<K> operator-(const Du<K>& x, const Du<K>& y) {
  Du<K> r{x.v - y.v, {}};
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = x.d[k] - y.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Du<K> operator*(const Du<K>& x, const Du<K>& y) {
  Du<K> r{x.v * y.v, {}};
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = fma(x.v, y.d[k], x.d[k] * y.v);
  return r;
}
template <int K>
__device__ __forceinline__ Du<K> operator*(const Du<K>& x, double s) {
  Du<K> r{x.v * s, {}};
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = x.d[k] * s;
  return r;
}
template <int K>
__device__ __forceinline__ Du<K> dsqrt(const Du<K>& x) {
  const double r = sqrt(x.v), h = 0.5 / r;
  Du<K> o{r, {}};
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = x.d[k] * h;
  return o;
}
template <int K>
__device__ __forceinline__ Du<K> drecip(const Du<K>& x) {
  const double r = 1.0 / x.v, m = -(r * r);
  Du<K> o{r, {}};
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = x.d[k] * m;
  return o;
}
template <int K>
__device__ __forceinline__ Du<K> dzero() {
  Du<K> o{0.0, {}};
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = 0.0;
  return o;
}

// Phi = f + w_g g of Eq. 8, 9 (J = curl B, Eq. 14) and its gradient F with respect to
// q = (B (3), G (9, G[3p+j] = dB_p/dx_j)).  With C = J x B:
//   f = |C| / (|J| |B|) (0 when |J||B| = 0),   g = g_scale |D| / |B| (0 when |B| = 0),
//   df/dJ = B x C / (|C| |J| |B|) - f J / |J|^2,   df/dB = C x J / (|C| |J| |B|) - f B / |B|^2
// (the |C| term 0 when |C| = 0), dg/dB = -g B / |B|^2, dg/dD = g_scale sign(D) / |B| (sign(0) =
// +1), and J, D linear in G.  Evaluated on dual numbers (branches taken on the values): the
// value parts are Phi and F, the derivative parts their derivatives along the tangents of q.
template <int K>
__device__ void objective_grad_q(const Du<K>* q, double g_scale, double w_g, Du<K>& phi,
                                 Du<K>* F) {
  using T = Du<K>;
  const T* B = q;
  const T* G = q + 3;
  const T Jx = G[7] - G[5], Jy = G[2] - G[6], Jz = G[3] - G[1];
  const T D = G[0] + G[4] + G[8];
  const T Cx = Jy * B[2] - Jz * B[1];
  const T Cy = Jz * B[0] - Jx * B[2];
  const T Cz = Jx * B[1] - Jy * B[0];
  const T sJ = Jx * Jx + Jy * Jy + Jz * Jz, sB = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  const T sC = Cx * Cx + Cy * Cy + Cz * Cz;
  const T z0 = dzero<K>();
  const T nJ = sJ.v > 0.0 ? dsqrt(sJ) : z0;
  const T nB = sB.v > 0.0 ? dsqrt(sB) : z0;
  const T nC = sC.v > 0.0 ? dsqrt(sC) : z0;
  T gB[3] = {z0, z0, z0}, gJ[3] = {z0, z0, z0}, gD = z0;
  phi = z0;
  if (nJ.v * nB.v > 0.0) {
    const T inv = drecip(nJ * nB);
    const T f = nC * inv;
    phi = f;
    if (nC.v > 0.0) {
      const T k = inv * drecip(nC);
      gJ[0] = (B[1] * Cz - B[2] * Cy) * k;
      gJ[1] = (B[2] * Cx - B[0] * Cz) * k;
      gJ[2] = (B[0] * Cy - B[1] * Cx) * k;
      gB[0] = (Cy * Jz - Cz * Jy) * k;
      gB[1] = (Cz * Jx - Cx * Jz) * k;
      gB[2] = (Cx * Jy - Cy * Jx) * k;
    }
    const T fJ = f * drecip(sJ), fB = f * drecip(sB);
    gJ[0] = gJ[0] - Jx * fJ;
    gJ[1] = gJ[1] - Jy * fJ;
    gJ[2] = gJ[2] - Jz * fJ;
    for (int i = 0; i < 3; ++i) gB[i] = gB[i] - B[i] * fB;
  }
  if (nB.v > 0.0) {
    const double gs = g_scale * w_g;
    const T rB = drecip(nB);
    const T aD = D.v < 0.0 ? D * -1.0 : D;
    const T g = (aD * rB) * gs;
    phi = phi + g;
    gD = rB * (D.v < 0.0 ? -gs : gs);
    const T gb = g * drecip(sB);
    for (int i = 0; i < 3; ++i) gB[i] = gB[i] - B[i] * gb;
  }
  for (int i = 0; i < 3; ++i) F[i] = gB[i];
  // G index 3p + j: Jx = G7 - G5, Jy = G2 - G6, Jz = G3 - G1, D = G0 + G4 + G8
  F[3 + 0] = gD;
  F[3 + 1] = z0 - gJ[2];
  F[3 + 2] = gJ[1];
  F[3 + 3] = gJ[2];
  F[3 + 4] = gD;
  F[3 + 5] = z0 - gJ[0];
  F[3 + 6] = z0 - gJ[1];
  F[3 + 7] = gJ[0];
  F[3 + 8] = gD;
}

// q (value), dq/dlambda_p and d2q/dlambda_p^2 of one query from its 30 Hessian-pass sums;
// q index: 0..2 B_p, 3 + 3p + j dB_p/dx_j.
__device__ void q_derivs(const double* S, double z, const double lam[3], double q[12],
                         double d1[12], double d2[12]) {
  for (int p = 0; p < 3; ++p) {
    const double* s = S + 10 * p;
    const double l = lam[p], l2 = l * l;
    const double S0 = s[0], S1 = s[1], Sx = s[2], Sy = s[3], Sl = s[4], Tx = s[5], Ty = s[6];
    const double Qs = s[7], Ux = s[8], Uy = s[9];
    q[p] = z * S0;
    q[3 + 3 * p] = z * Sx;
    q[4 + 3 * p] = z * Sy;
    q[5 + 3 * p] = S0 + z * z * S1;
    d1[p] = z * l * Sl;
    d1[3 + 3 * p] = -(z * l * Tx);
    d1[4 + 3 * p] = -(z * l * Ty);
    d1[5 + 3 * p] = l * Sl - z * z * l * S0;
    const double e = Sl - l * Qs;   // d2S0/dl2 = Sl + l dSl/dl
    d2[p] = z * e;
    d2[3 + 3 * p] = -(z * (Tx + l2 * Ux));
    d2[4 + 3 * p] = -(z * (Ty + l2 * Uy));
    d2[5 + 3 * p] = e - z * z * (S0 + l2 * Sl);
  }
}

__device__ __forceinline__ int comp_of(int m) { return m < 3 ? m : (m - 3) / 3; }

// Phi, its lambda-gradient and lambda-Hessian (DIM 3: per component; DIM 1: one shared lambda,
// entry 0 only), with F = dPhi/dq and the columns P D of the Hessian's first term (PD[12 k + m]).
template <int DIM>
__device__ void hessian_cols(const double q[12], const double d1[12], const double d2[12],
                             double g_scale, double w_g, double& phi, double grad[3], double H[9],
                             double F[12], double PD[12 * DIM]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) H[i] = 0.0;
  grad[0] = grad[1] = grad[2] = 0.0;
  // one evaluation, tangent k = column k of D (dq/dlambda_k)
  Du<DIM> x[12], ph, Fd[12];
#pragma unroll
  for (int m = 0; m < 12; ++m) {
    x[m].v = q[m];
#pragma unroll
    for (int k = 0; k < DIM; ++k) x[m].d[k] = (DIM == 1 || comp_of(m) == k) ? d1[m] : 0.0;
  }
  objective_grad_q<DIM>(x, g_scale, w_g, ph, Fd);
  phi = ph.v;
#pragma unroll
  for (int m = 0; m < 12; ++m) {
    F[m] = Fd[m].v;
#pragma unroll
    for (int k = 0; k < DIM; ++k) PD[12 * k + m] = Fd[m].d[k];
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    double gj = 0.0, cj = 0.0;
#pragma unroll
    for (int m = 0; m < 12; ++m)
      if (DIM == 1 || comp_of(m) == j) {
        gj += d1[m] * F[m];
        cj += d2[m] * F[m];
      }
    grad[j] = gj;
#pragma unroll
    for (int k = j; k < DIM; ++k) {
      double h = j == k ? cj : 0.0;
#pragma unroll
      for (int m = 0; m < 12; ++m)
        if (DIM == 1 || comp_of(m) == j) h += d1[m] * PD[12 * k + m];
      H[3 * j + k] = h;
      H[3 * k + j] = h;
    }
  }
}

// Cholesky solve of H v = r (m <= 3); false when H is not positive definite.
__device__ bool chol3(int m, const double* H, const double* r, double* v) {
  double L[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, y[3] = {0, 0, 0};
  for (int j = 0; j < m; ++j) {
    double d = H[3 * j + j];
    for (int k = 0; k < j; ++k) d -= L[3 * j + k] * L[3 * j + k];
    if (!(d > 0.0)) return false;
    L[3 * j + j] = sqrt(d);
    for (int i = j + 1; i < m; ++i) {
      double e = H[3 * i + j];
      for (int k = 0; k < j; ++k) e -= L[3 * i + k] * L[3 * j + k];
      L[3 * i + j] = e / L[3 * j + j];
    }
  }
  for (int i = 0; i < m; ++i) {
    double e = r[i];
    for (int k = 0; k < i; ++k) e -= L[3 * i + k] * y[k];
    y[i] = e / L[3 * i + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double e = y[i];
    for (int k = i + 1; k < m; ++k) e -= L[3 * k + i] * v[k];
    v[i] = e / L[3 * i + i];
  }
  return true;
}

__device__ __forceinline__ double gsum(const double* out, const PlanHdr& h,
                                       const int32_t* item_off, int64_t j, int nsum, int s) {
  double v = 0.0;
  for (int sp = 0; sp < h.nsplit; ++sp) v += out[out_index(h, item_off, 0, j, sp, s, nsum)];
  return v;
}

__global__ void finalize_hessian_kernel(int64_t n, const PlanHdr* __restrict__ plan,
                                        const int32_t* __restrict__ item_off,
                                        const double* __restrict__ out,
                                        const float4* __restrict__ qpos,
                                        const Lam4* __restrict__ qlam, int dim, double g_scale,
                                        double w_g, double* phi_out, double* grad_out,
                                        double* hess_out, const double* __restrict__ corr) {
  constexpr int NSUM = 3 * nsum_per_comp(VAR_HESS);
  const PlanHdr h = *plan;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double S[NSUM];
    for (int s = 0; s < NSUM; ++s) S[s] = gsum(out, h, item_off, i, NSUM, s);
    const Lam4 l = qlam[i];
    // one shared lambda: lambda_x for every component, as the tied pair-sum pass used
    const double lam[3] = {l.x, dim == 1 ? l.x : l.y, dim == 1 ? l.x : l.z};
    double q[12], d1[12], d2[12], phi = 0.0, grad[3], H[9];
    q_derivs(S, (double)qpos[i].z, lam, q, d1, d2);
    if (corr)   // pixel-exact near field: B and grad B move, their lambda-derivatives do not
      for (int m = 0; m < 12; ++m) q[m] += corr[12 * i + m];
    double F[12], PD[36];
    if (dim == 1) hessian_cols<1>(q, d1, d2, g_scale, w_g, phi, grad, H, F, PD);
    else hessian_cols<3>(q, d1, d2, g_scale, w_g, phi, grad, H, F, PD);
    if (phi_out) phi_out[i] = phi;
    if (grad_out)
      for (int j = 0; j < 3; ++j) grad_out[3 * i + j] = grad[j];
    if (hess_out)
      for (int j = 0; j < 9; ++j) hess_out[9 * i + j] = H[j];
  }
}

// Per point: H, v = H^-1 dL/dlambda and the 21 adjoint weights, written as the point's record of
// the seven-weight adjoint sweep (plus padding records up to the tile multiple).
__global__ void implicit_weights_kernel(int64_t n, int nptiles, const PlanHdr* __restrict__ plan,
                                        const int32_t* __restrict__ item_off,
                                        const double* __restrict__ out,
                                        const float4* __restrict__ qpos,
                                        const Lam4* __restrict__ qlam,
                                        const double* __restrict__ gB, int dim, double g_scale,
                                        double w_g, float* p32, double* p64, int fp64,
                                        double* v_out, int32_t* flags,
                                        const double* __restrict__ corr, double* pxe_w) {
  constexpr int NSUM = 3 * nsum_per_comp(VAR_HESS);
  const PlanHdr h = *plan;
  const int64_t total = (int64_t)nptiles * TILE;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    double x = 0.0, y = 0.0, z = 1.0, lam[3] = {0.0, 0.0, 0.0}, W[21];
    float zf = 1.f;
    for (int m = 0; m < 21; ++m) W[m] = 0.0;
    if (i < n) {
      const float4 pos = qpos[i];
      x = pos.x;
      y = pos.y;
      zf = pos.z;
      z = zf;
      const Lam4 l = qlam[i];
      lam[0] = l.x;
      lam[1] = dim == 1 ? l.x : l.y;
      lam[2] = dim == 1 ? l.x : l.z;
      double S[NSUM];
      for (int s = 0; s < NSUM; ++s) S[s] = gsum(out, h, item_off, i, NSUM, s);
      double q[12], d1[12], d2[12], phi = 0.0, grad[3], H[9];
      q_derivs(S, z, lam, q, d1, d2);
      if (corr)
        for (int m = 0; m < 12; ++m) q[m] += corr[12 * i + m];
      double F[12], PD[36];
      if (dim == 1) hessian_cols<1>(q, d1, d2, g_scale, w_g, phi, grad, H, F, PD);
      else hessian_cols<3>(q, d1, d2, g_scale, w_g, phi, grad, H, F, PD);
      const double g[3] = {gB[3 * i], gB[3 * i + 1], gB[3 * i + 2]};
      double gl[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0};
      if (dim == 1) gl[0] = g[0] * d1[0] + g[1] * d1[1] + g[2] * d1[2];
      else for (int p = 0; p < 3; ++p) gl[p] = g[p] * d1[p];
      const bool pd = chol3(dim, H, gl, v);
      if (!pd) v[0] = v[1] = v[2] = 0.0;
      double vp[3];
      for (int p = 0; p < 3; ++p) vp[p] = dim == 1 ? v[0] : v[p];
      if (v_out)
        for (int p = 0; p < 3; ++p) v_out[3 * i + p] = vp[p];
      if (flags) flags[i] = pd ? 0 : 1;
      // Phi's first derivatives dPhi/dq and w = (d2 Phi / dq dq) . (dq along v) = sum_k v_k (P D)_k
      double Fq[12], wq[12];
#pragma unroll
      for (int m = 0; m < 12; ++m) {
        double w = v[0] * PD[m];
        if (dim == 3) w = (w + v[1] * PD[12 + m]) + v[2] * PD[24 + m];
        Fq[m] = pd ? F[m] : 0.0;
        wq[m] = pd ? w : 0.0;
      }
      for (int p = 0; p < 3; ++p) {
        const double lp = lam[p], vl = vp[p] * lp;
        const double wB = wq[p], wx = wq[3 + 3 * p], wy = wq[4 + 3 * p], wz = wq[5 + 3 * p];
        const double FB = Fq[p], Fx = Fq[3 + 3 * p], Fy = Fq[4 + 3 * p], Fz = Fq[5 + 3 * p];
        double* w = W + 7 * p;
        w[0] = g[p] * z - (z * wB + wz - vl * z * z * Fz);   // phi
        w[1] = -(z * z * wz);                                 // psi
        w[2] = -(z * wx);                                     // psi dx
        w[3] = -(z * wy);                                     // psi dy
        w[4] = -(vl * (z * FB + Fz));                         // cos(lambda r) / r
        w[5] = vl * z * Fx;                                   // phi dx
        w[6] = vl * z * Fy;                                   // phi dy
        if (pxe_w) {
          // the correction moves B_p and grad B_p only (linear in B0, lambda-independent)
          double* o = pxe_w + 12 * i + 4 * p;
          o[0] = g[p] - wB;
          o[1] = -wx;
          o[2] = -wy;
          o[3] = -wz;
        }
      }
    }
    const int64_t base = (i / TILE) * (int64_t)(VJP7_NFIELD * TILE) + (i % TILE);
    if (fp64) {
      p64[base] = x;
      p64[base + TILE] = y;
      p64[base + 2 * TILE] = z * z;
      for (int p = 0; p < 3; ++p) p64[base + (3 + p) * TILE] = lam[p];
      for (int m = 0; m < 21; ++m) p64[base + (6 + m) * TILE] = W[m];
    } else {
      p32[base] = (float)x;
      p32[base + TILE] = (float)y;
      p32[base + 2 * TILE] = __fmul_rn(zf, zf);
      for (int p = 0; p < 3; ++p) p32[base + (3 + p) * TILE] = (float)lam[p];
      for (int m = 0; m < 21; ++m) p32[base + (6 + m) * TILE] = (float)W[m];
    }
  }
}

__global__ void finalize_nv_kernel(int64_t n, const PlanHdr* __restrict__ plan,
                                   const int32_t* __restrict__ item_off,
                                   const double* __restrict__ out,
                                   const float4* __restrict__ qpos, double* var) {
  const PlanHdr h = *plan;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double z = (double)qpos[i].z;
    for (int p = 0; p < 3; ++p) var[3 * i + p] = z * z * gsum(out, h, item_off, i, 3, p);
  }
}

// Variance tiles: positions as the boundary's, and s_p = (sigma_p (dA / 2 pi))^2 (sigma_p from
// the array, or sigma0 where the array is NULL); padding pixels carry s = 0.
__global__ void stage_variance_kernel(const float* __restrict__ sx, const float* __restrict__ sy,
                                      const float* __restrict__ sz, double sigma0, int nx, int ny,
                                      double x0, double y0, double hx, double hy, double w,
                                      int ntiles, float* __restrict__ t32,
                                      double* __restrict__ t64) {
  const int64_t npix = (int64_t)nx * ny;
  const int64_t total = (int64_t)ntiles * TILE;
  const float* sg[3] = {sx, sy, sz};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const bool real = k < npix;
    const int64_t kk = real ? k : npix - 1;
    const int i = (int)(kk % nx), j = (int)(kk / nx);
    const double x = x0 + i * hx, y = y0 + j * hy;
    const int64_t base = (k / TILE) * (int64_t)(NFIELD * TILE) + (k % TILE);
    t64[base] = x;
    t64[base + TILE] = y;
    t32[base] = (float)x;
    t32[base + TILE] = (float)y;
    for (int p = 0; p < 3; ++p) {
      const double sd = real ? (sg[p] ? (double)sg[p][kk] : sigma0) * w : 0.0;
      t64[base + (2 + p) * TILE] = sd * sd;
      t32[base + (2 + p) * TILE] = (float)(sd * sd);
    }
  }
}

int grid_for(int64_t n, int cap) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g < cap ? g : cap));
}

}  // namespace

void launch_finalize_hessian(int64_t n, const PlanHdr* plan, const int32_t* item_off,
                             const double* out, const float4* qpos, const Lam4* qlam, int dim,
                             double g_scale, double w_g, double* phi, double* grad, double* hess,
                             const double* corr, cudaStream_t s) {
  if (n <= 0) return;
  finalize_hessian_kernel<<<grid_for(n, 4096), 256, 0, s>>>(n, plan, item_off, out, qpos, qlam,
                                                            dim, g_scale, w_g, phi, grad, hess,
                                                            corr);
}

void launch_implicit_weights(int64_t n, int nptiles, const PlanHdr* plan, const int32_t* item_off,
                             const double* out, const float4* qpos, const Lam4* qlam,
                             const double* gB, int dim, double g_scale, double w_g, float* p32,
                             double* p64, int fp64, double* v_out, int32_t* flags,
                             const double* corr, double* pxe_w, cudaStream_t s) {
  const int64_t total = (int64_t)nptiles * TILE;
  if (total <= 0) return;
  implicit_weights_kernel<<<grid_for(total, 4096), 128, 0, s>>>(
      n, nptiles, plan, item_off, out, qpos, qlam, gB, dim, g_scale, w_g, p32, p64, fp64, v_out,
      flags, corr, pxe_w);
}

void launch_finalize_nv(int64_t n, const PlanHdr* plan, const int32_t* item_off, const double* out,
                        const float4* qpos, double* var, cudaStream_t s) {
  if (n <= 0) return;
  finalize_nv_kernel<<<grid_for(n, 4096), 256, 0, s>>>(n, plan, item_off, out, qpos, var);
}

void launch_stage_variance(const float* sx, const float* sy, const float* sz, double sigma0,
                           int nx, int ny, double x0, double y0, double hx, double hy, double w,
                           int ntiles, float* t32, double* t64, cudaStream_t s) {
  const int64_t total = (int64_t)ntiles * TILE;
  stage_variance_kernel<<<grid_for(total, 8192), 256, 0, s>>>(sx, sy, sz, sigma0, nx, ny, x0, y0,
                                                              hx, hy, w, ntiles, t32, t64);
}

}  // namespace dbie
