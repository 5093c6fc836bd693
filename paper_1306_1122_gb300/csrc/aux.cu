// aux.cu -- staging, packing, near-field correction and adjoint finalisation kernels.
#include "ff_math.cuh"
#include "kernels.h"

namespace dbie {

// Boundary staging (Eq. 3 / Eq. 16): row-major (ny, nx) components -> tile-blocked SoA in FP32
// and FP64, with b_p = B_p0 * dA / (2 pi).  Padding pixels repeat the last pixel's position
// with b = 0.
__global__ void stage_boundary_kernel(const float* __restrict__ Bx, const float* __restrict__ By,
                                      const float* __restrict__ Bz, int nx, int ny, double x0,
                                      double y0, double hx, double hy, double scale, int ntiles,
                                      float* __restrict__ t32, double* __restrict__ t64) {
  const int64_t npix = (int64_t)nx * ny;
  const int64_t total = (int64_t)ntiles * TILE;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const bool real = k < npix;
    const int64_t kk = real ? k : npix - 1;
    const int i = (int)(kk % nx), j = (int)(kk / nx);
    const double x = x0 + i * hx, y = y0 + j * hy;
    const double b[3] = {real ? (double)Bx[kk] * scale : 0.0, real ? (double)By[kk] * scale : 0.0,
                         real ? (double)Bz[kk] * scale : 0.0};
    const int64_t base = (k / TILE) * (int64_t)(NFIELD * TILE) + (k % TILE);
    t64[base] = x;
    t64[base + TILE] = y;
    t32[base] = (float)x;
    t32[base + TILE] = (float)y;
    for (int p = 0; p < 3; ++p) {
      t64[base + (2 + p) * TILE] = b[p];
      t32[base + (2 + p) * TILE] = (float)b[p];
    }
  }
}

void launch_stage_boundary(const float* Bx, const float* By, const float* Bz, int nx, int ny,
                           double x0, double y0, double hx, double hy, double scale, int ntiles,
                           float* t32, double* t64, cudaStream_t s) {
  const int64_t total = (int64_t)ntiles * TILE;
  const int grid = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  stage_boundary_kernel<<<grid, 256, 0, s>>>(Bx, By, Bz, nx, ny, x0, y0, hx, hy, scale, ntiles,
                                             t32, t64);
}

// Quadratic Lagrange polynomials on the nodes -1, 0, +1 (index 0, 1, 2).
__device__ __forceinline__ double lagrange3(int a, double t) {
  return a == 0 ? 0.5 * t * (t - 1.0) : (a == 1 ? 1.0 - t * t : 0.5 * t * (t + 1.0));
}

// Eq. 15 staging: quadrature point k = J * qnx + I of element (I / g, J / g), Gauss indices
// (I % g, J % g), at xc + xi hx, yc + eta hy, carrying the nine-node interpolant of B0 times the
// Gauss weights, the Jacobian hx hy and 1 / (2 pi).  Padding points carry b = 0.  FP32 tiles
// have NFIELD_SPLIT fields (positions as hi + lo float pairs), FP64 tiles NFIELD.
__global__ void stage_q9_kernel(const float* __restrict__ B0, int nx, int ny, double x0, double y0,
                                double hx, double hy, QuadInfo qi, int ntiles,
                                float* __restrict__ t32, double* __restrict__ t64) {
  const int g = qi.g;
  const int qnx = (nx - 1) / 2 * g, qny = (ny - 1) / 2 * g;
  const int64_t nq = (int64_t)qnx * qny;
  const int64_t npix = (int64_t)nx * ny;
  const int64_t total = (int64_t)ntiles * TILE;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const bool real = k < nq;
    const int64_t kk = real ? k : nq - 1;
    const int I = (int)(kk % qnx), J = (int)(kk / qnx);
    const int ex = I / g, a = I % g, ey = J / g, b = J % g;
    const double xi = qi.gx[a], eta = qi.gx[b];
    const double x = x0 + (2 * ex + 1) * hx + xi * hx;
    const double y = y0 + (2 * ey + 1) * hy + eta * hy;
    const double w = qi.gw[a] * qi.gw[b] * hx * hy / TWO_PI;
    double v[3] = {0.0, 0.0, 0.0};
    if (real)
      for (int jb = 0; jb < 3; ++jb)
        for (int ia = 0; ia < 3; ++ia) {
          const double sf = lagrange3(ia, xi) * lagrange3(jb, eta);
          const int64_t node = (int64_t)(2 * ey + jb) * nx + (2 * ex + ia);
          for (int p = 0; p < 3; ++p) v[p] += sf * (double)B0[p * npix + node];
        }
    const int64_t base = (k / TILE) * (int64_t)(NFIELD * TILE) + (k % TILE);
    const int64_t base32 = (k / TILE) * (int64_t)(NFIELD_SPLIT * TILE) + (k % TILE);
    t64[base] = x;
    t64[base + TILE] = y;
    const float xh = (float)x, yh = (float)y;
    t32[base32] = xh;
    t32[base32 + TILE] = yh;
    t32[base32 + 5 * TILE] = (float)(x - (double)xh);
    t32[base32 + 6 * TILE] = (float)(y - (double)yh);
    for (int p = 0; p < 3; ++p) {
      const double bv = real ? v[p] * w : 0.0;
      t64[base + (2 + p) * TILE] = bv;
      t32[base32 + (2 + p) * TILE] = (float)bv;
    }
  }
}

void launch_stage_q9(const float* B0, int nx, int ny, double x0, double y0, double hx, double hy,
                     const QuadInfo& qi, int ntiles, float* t32, double* t64, cudaStream_t s) {
  const int64_t total = (int64_t)ntiles * TILE;
  const int grid = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  stage_q9_kernel<<<grid, 256, 0, s>>>(B0, nx, ny, x0, y0, hx, hy, qi, ntiles, t32, t64);
}

// Adjoint of the Eq. 15 staging: per node, the sum over the elements that hold it and over their
// Gauss points of shape function x Gauss weights x hx hy / (2 pi) x the per-point adjoint T.
__global__ void q9_gather_kernel(const double* __restrict__ T, int nx, int ny, double hx,
                                 double hy, QuadInfo qi, double* gB0, int accumulate) {
  const int g = qi.g;
  const int nex = (nx - 1) / 2, ney = (ny - 1) / 2, qnx = nex * g;
  const int64_t npix = (int64_t)nx * ny;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < npix;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(k % nx), j = (int)(k / nx);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int ey = (j - 1) / 2 - 1; ey <= j / 2; ++ey) {
      if (ey < 0 || ey >= ney) continue;
      const int jb = j - 2 * ey;
      if (jb < 0 || jb > 2) continue;
      for (int ex = (i - 1) / 2 - 1; ex <= i / 2; ++ex) {
        if (ex < 0 || ex >= nex) continue;
        const int ia = i - 2 * ex;
        if (ia < 0 || ia > 2) continue;
        for (int b = 0; b < g; ++b)
          for (int a = 0; a < g; ++a) {
            const double c = lagrange3(ia, qi.gx[a]) * lagrange3(jb, qi.gx[b]) * qi.gw[a] *
                             qi.gw[b] * hx * hy / TWO_PI;
            const int64_t q = (int64_t)(ey * g + b) * qnx + (ex * g + a);
            for (int p = 0; p < 3; ++p) acc[p] += c * T[3 * q + p];
          }
      }
    }
    for (int p = 0; p < 3; ++p) gB0[3 * k + p] = accumulate ? gB0[3 * k + p] + acc[p] : acc[p];
  }
}

void launch_q9_gather(const double* T, int nx, int ny, double hx, double hy, const QuadInfo& qi,
                      double* gB0, int accumulate, cudaStream_t s) {
  const int64_t npix = (int64_t)nx * ny;
  const int grid = (int)((npix + 255) / 256 < 8192 ? (npix + 255) / 256 : 8192);
  q9_gather_kernel<<<grid, 256, 0, s>>>(T, nx, ny, hx, hy, qi, gB0, accumulate);
}

// Queries of a single evaluation: one per point, lambda from float or double input.
__global__ void pack_eval_kernel(int64_t n, const float* __restrict__ xyz,
                                 const float* __restrict__ lam_f, const double* __restrict__ lam_d,
                                 float4* __restrict__ qpos, Lam4* __restrict__ qlam,
                                 int32_t* near_list, int32_t* near_cnt, int near_on, double near_z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    qpos[i] = make_float4(x, y, z, __int_as_float(0));
    if (lam_d)
      qlam[i] = make_lam4(lam_d[3 * i], lam_d[3 * i + 1], lam_d[3 * i + 2]);
    else
      qlam[i] = make_lam4((double)lam_f[3 * i], (double)lam_f[3 * i + 1], (double)lam_f[3 * i + 2]);
    if (near_on && (double)z <= near_z) near_list[atomicAdd(near_cnt, 1)] = (int32_t)i;
  }
}

void launch_pack_eval(int64_t n, const float* xyz, const float* lam_f, const double* lam_d,
                      float4* qpos, Lam4* qlam, int32_t* near_list, int32_t* near_cnt,
                      int near_on, double near_z, cudaStream_t s) {
  if (n <= 0) return;
  const int grid = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
  pack_eval_kernel<<<grid, 256, 0, s>>>(n, xyz, lam_f, lam_d, qpos, qlam, near_list, near_cnt,
                                        near_on, near_z);
}

__global__ void plan_single_kernel(PlanHdr* plan, int32_t* item_off, int32_t* q_cnt,
                                   int32_t* work, int nitems, int nsplit, int qper, int qcount) {
  PlanHdr h;
  h.nitems = nitems;
  h.nsplit = nsplit;
  h.qper = qper;
  h.pad0 = 0;
  *plan = h;
  item_off[0] = 0;
  item_off[1] = nitems;
  q_cnt[0] = qcount;
  *work = 0;
}

void launch_plan_single(PlanHdr* plan, int32_t* item_off, int32_t* q_cnt, int32_t* work,
                        int nitems, int nsplit, int qper, int qcount, cudaStream_t s) {
  plan_single_kernel<<<1, 1, 0, s>>>(plan, item_off, q_cnt, work, nitems, nsplit, qper, qcount);
}

// Near-field correction (mixed precision, points with z <= near_z): over the (2W+1)^2 pixels
// around the point, replace the FP32 pair terms that the pair-sum kernel added by FP64 ones.
// The FP32 terms are recomputed with the same explicitly rounded code (pair_terms32), so the
// correction sum_k (t64 - t32) removes exactly what was added.  Eight lanes per query; the
// correction is added in place to the query's split-0 partial sums (run after the pair sums).
// Index (along one axis) of the quadrature point nearest to coordinate x: the pixel for the
// midpoint rule; for nine-node elements of width 2h with g Gauss points, element e and the
// nearest abscissa a give e * g + a.
__device__ __forceinline__ long near_index(double x, double x0, double h, int nq,
                                           const ProbDesc& pd) {
  if (pd.quad_g == 0) return lrint((x - x0) / h);
  const int g = pd.quad_g;
  const long ne = nq / g;
  long e = (long)floor((x - x0) / (2.0 * h));
  e = e < 0 ? 0 : (e > ne - 1 ? ne - 1 : e);
  const double xi = (x - x0) / h - (double)(2 * e + 1);
  int best = 0;
  double bd = fabs(xi - pd.gx[0]);
  for (int a = 1; a < g; ++a) {
    const double d = fabs(xi - pd.gx[a]);
    if (d < bd) { bd = d; best = a; }
  }
  return e * g + best;
}

template <int VAR, bool TIED>
__global__ void nearfield_kernel(const ProbDesc* __restrict__ probs,
                                 const int32_t* __restrict__ near_list,
                                 const int32_t* __restrict__ near_cnt,
                                 const float4* __restrict__ qpos, const Lam4* __restrict__ qlam,
                                 const PlanHdr* __restrict__ plan,
                                 const int32_t* __restrict__ item_off, double* __restrict__ out) {
  constexpr int NS = nsum_per_comp(VAR);
  constexpr int NSUM = 3 * NS;
  // Eight lanes per query, four queries per warp: a 7 x 7 window takes 7 passes of 8 lanes
  // (49 of 56 lane slots busy) instead of 2 of 32 (49 of 64).  The loop runs warp-uniformly so
  // the shuffles see every lane.
  constexpr int GL = 8;
  // sin and cos of lambda r in float-float on the FP32 pipe (absolute error ~1e-13 + 5e-15 |lambda
  // r|, far below the FP32 terms' error that the correction removes) instead of FP64 sincos,
  // which cost most of this kernel's FP64-pipe time
  __shared__ float4 s_tab[ff::SC_TABLE];
  ff::fill_sincos_table(s_tab, threadIdx.x);
  __syncthreads();
  auto sincos_ff = [&](double th, double& s, double& c) {
    ff::ds S, C;
    ff::sincos_ds_any(ff::from_double(th), s_tab, S, C);
    s = ff::to_double(S);
    c = ff::to_double(C);
  };
  const int lane = threadIdx.x & 31, sub = lane & (GL - 1), grp = lane / GL;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int cnt = *near_cnt;
  for (int64_t wb = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * (32 / GL); wb < cnt;
       wb += nwarps * (32 / GL)) {
    const int64_t w = wb + grp;
    const bool valid = w < cnt;
    const int64_t slot = near_list[valid ? w : wb];
    const float4 pos = qpos[slot];
    const Lam4 lam = qlam[slot];
    const int pidx = __float_as_int(pos.w);
    const ProbDesc& pd = probs[pidx];
    const Query<float, TIED> q32 = make_query<float, TIED>(pos, lam);
    const Query<double, TIED> q64 = make_query<double, TIED>(pos, lam);
    const int W = pd.near_w > 0 ? pd.near_w : NEAR_W;
    const long ix = near_index((double)pos.x, pd.x0, pd.hx, pd.nx, pd);
    const long iy = near_index((double)pos.y, pd.y0, pd.hy, pd.ny, pd);
    const long i0 = ix - W < 0 ? 0 : ix - W;
    const long i1 = ix + W > pd.nx - 1 ? pd.nx - 1 : ix + W;
    const long j0 = iy - W < 0 ? 0 : iy - W;
    const long j1 = iy + W > pd.ny - 1 ? pd.ny - 1 : iy + W;
    const long wi = i1 - i0 + 1, wj = j1 - j0 + 1;
    double c[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) c[s] = 0.0;
    if (valid && wi > 0 && wj > 0 && wi <= 2 * W + 1 && wj <= 2 * W + 1) {
      const int nwin = (int)(wi * wj);
      for (int e = sub; e < nwin; e += GL) {
        const int64_t k = (j0 + e / wi) * (int64_t)pd.nx + (i0 + e % wi);
        const int nf = pd.nf32 > 0 ? pd.nf32 : NFIELD;
        const float b32[3] = {*tile_field(pd.tiles32, k, 2, nf), *tile_field(pd.tiles32, k, 3, nf),
                              *tile_field(pd.tiles32, k, 4, nf)};
        const double b64[3] = {*tile_field(pd.tiles64, k, 2), *tile_field(pd.tiles64, k, 3),
                               *tile_field(pd.tiles64, k, 4)};
        Terms32<VAR, TIED> t32;
        Terms64<VAR, TIED> t64;
        if (nf == NFIELD_SPLIT)
          pair_terms32_split<VAR, TIED>(q32, *tile_field(pd.tiles32, k, 0, nf),
                                        *tile_field(pd.tiles32, k, 1, nf),
                                        *tile_field(pd.tiles32, k, 5, nf),
                                        *tile_field(pd.tiles32, k, 6, nf), b32, t32);
        else
          pair_terms32<VAR, TIED>(q32, *tile_field(pd.tiles32, k, 0), *tile_field(pd.tiles32, k, 1),
                                  b32, t32);
        pair_terms64_sc<VAR, TIED>(q64, *tile_field(pd.tiles64, k, 0),
                                   *tile_field(pd.tiles64, k, 1), b64, t64, sincos_ff);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const int lp = TIED ? 0 : p;
          // FP32 contributions as the scalar FP32 code computes them (products of two FP32
          // factors, exact in FP64; the packed kernel's can differ by a rounding of a factor),
          // replaced by the FP64 terms.
          if constexpr (has_hess(VAR)) c[p * NS] += t64.t0[p] - (double)t32.t0[p];
          else c[p * NS] += t64.t0[p] - (double)t32.u[lp] * (double)t32.rb[p];
          if constexpr (has_grad(VAR)) {
            c[p * NS + 1] += t64.t1[p] - (double)t32.t1[p];
            c[p * NS + 2] += t64.t1[p] * t64.dx - (double)t32.t1[p] * (double)t32.dx;
            c[p * NS + 3] += t64.t1[p] * t64.dy - (double)t32.t1[p] * (double)t32.dy;
          }
          if constexpr (has_hess(VAR))
            c[p * NS + idx_sl(VAR)] += t64.tl[p] - (double)t32.tl[p];
          else if constexpr (has_dlam(VAR))
            c[p * NS + idx_sl(VAR)] += t64.tl[p] - (double)t32.cr[lp] * (double)b32[p];
          if constexpr (has_newton(VAR)) {
            c[p * NS + IDX_TX] += t64.t0[p] * t64.dx - (double)t32.t0[p] * (double)t32.dx;
            c[p * NS + IDX_TY] += t64.t0[p] * t64.dy - (double)t32.t0[p] * (double)t32.dy;
          }
          if constexpr (has_hess(VAR)) {
            c[p * NS + IDX_Q] += t64.tq[p] - (double)t32.sn[lp] * (double)b32[p];
            c[p * NS + IDX_UX] += t64.tl[p] * t64.dx - (double)t32.tl[p] * (double)t32.dx;
            c[p * NS + IDX_UY] += t64.tl[p] * t64.dy - (double)t32.tl[p] * (double)t32.dy;
          }
        }
      }
    }
    const PlanHdr h = *plan;
#pragma unroll
    for (int s = 0; s < NSUM; ++s) {
      double v = c[s];
      for (int off = GL / 2; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (sub == 0 && valid) out[out_index(h, item_off, pidx, slot - pd.q_off, 0, s, NSUM)] += v;
    }
  }
}

void launch_nearfield(int var, bool tied, const ProbDesc* probs, const int32_t* near_list,
                      const int32_t* near_cnt, const float4* qpos, const Lam4* qlam,
                      const PlanHdr* plan, const int32_t* item_off, double* out, int grid,
                      cudaStream_t s) {
#define NF(V, T)                                                                            \
  nearfield_kernel<V, T><<<grid, 256, 0, s>>>(probs, near_list, near_cnt, qpos, qlam, plan, \
                                              item_off, out)
  if (tied) {
    switch (var) {
      case VAR_V: NF(VAR_V, true); break;
      case VAR_VL: NF(VAR_VL, true); break;
      case VAR_OBJ: NF(VAR_OBJ, true); break;
      case VAR_OBJL: NF(VAR_OBJL, true); break;
      case VAR_OBJN: NF(VAR_OBJN, true); break;
      case VAR_HESS: NF(VAR_HESS, true); break;
      default: break;  // VAR_NV: sums of positive terms, no near-field correction
    }
  } else {
    switch (var) {
      case VAR_V: NF(VAR_V, false); break;
      case VAR_VL: NF(VAR_VL, false); break;
      case VAR_OBJ: NF(VAR_OBJ, false); break;
      case VAR_OBJL: NF(VAR_OBJL, false); break;
      case VAR_OBJN: NF(VAR_OBJN, false); break;
      case VAR_HESS: NF(VAR_HESS, false); break;
      default: break;
    }
  }
#undef NF
}

// Point records for the adjoint sweep: x, y, z^2, lambda (3), w_p = gB_p * z (3).
__global__ void pack_vjp_kernel(int64_t n, const float* __restrict__ xyz,
                                const double* __restrict__ lam, const double* __restrict__ gB,
                                int tied, int nptiles, float* __restrict__ p32,
                                double* __restrict__ p64, int fp64) {
  const int64_t total = (int64_t)nptiles * TILE;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool real = i < n;
    double x = 0.0, y = 0.0, z = 1.0, l[3] = {0, 0, 0}, w[3] = {0, 0, 0};
    float zf = 1.f;
    if (real) {
      x = xyz[3 * i];
      y = xyz[3 * i + 1];
      zf = xyz[3 * i + 2];
      z = zf;
      for (int p = 0; p < 3; ++p) {
        l[p] = lam[3 * i + (tied ? 0 : p)];
        w[p] = gB[3 * i + p] * z;
      }
    }
    const int64_t base = (i / TILE) * (int64_t)(VJP_NFIELD * TILE) + (i % TILE);
    if (fp64) {
      p64[base] = x;
      p64[base + TILE] = y;
      p64[base + 2 * TILE] = z * z;
      for (int p = 0; p < 3; ++p) {
        p64[base + (3 + p) * TILE] = l[p];
        p64[base + (6 + p) * TILE] = w[p];
      }
    } else {
      p32[base] = (float)x;
      p32[base + TILE] = (float)y;
      p32[base + 2 * TILE] = __fmul_rn(zf, zf);
      for (int p = 0; p < 3; ++p) {
        p32[base + (3 + p) * TILE] = (float)l[p];
        p32[base + (6 + p) * TILE] = (float)w[p];
      }
    }
  }
}

void launch_pack_vjp(int64_t n, const float* xyz, const double* lam, const double* gB, int tied,
                     int nptiles, float* p32, double* p64, int fp64, cudaStream_t s) {
  const int64_t total = (int64_t)nptiles * TILE;
  const int grid = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  pack_vjp_kernel<<<grid, 256, 0, s>>>(n, xyz, lam, gB, tied, nptiles, p32, p64, fp64);
}

__global__ void finalize_vjp_kernel(int64_t npix, const PlanHdr* __restrict__ plan,
                                    const double* __restrict__ out, double scale, double* gB0,
                                    int accumulate) {
  const PlanHdr h = *plan;
  const int32_t zero = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < npix;
       k += (int64_t)gridDim.x * blockDim.x) {
    for (int p = 0; p < 3; ++p) {
      double v = 0.0;
      for (int sp = 0; sp < h.nsplit; ++sp) v += out[out_index(h, &zero, 0, k, sp, p, 3)];
      v *= scale;
      gB0[3 * k + p] = accumulate ? gB0[3 * k + p] + v : v;
    }
  }
}

void launch_finalize_vjp(int64_t npix, const PlanHdr* plan, const double* out, double scale,
                         double* gB0, int accumulate, cudaStream_t s) {
  const int grid = (int)((npix + 255) / 256 < 8192 ? (npix + 255) / 256 : 8192);
  finalize_vjp_kernel<<<grid, 256, 0, s>>>(npix, plan, out, scale, gB0, accumulate);
}

}  // namespace dbie

namespace dbie {

// Input validation on the device: counts non-finite values (mode 0) or, for (n, 3) point
// arrays, points with a non-finite coordinate or z <= 0 (mode 1).
__global__ void count_bad_kernel(const float* __restrict__ a, int64_t n, int mode, int32_t* cnt) {
  int local = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mode == 0) {
      local += isfinite(a[i]) ? 0 : 1;
    } else {
      const float x = a[3 * i], y = a[3 * i + 1], z = a[3 * i + 2];
      local += (isfinite(x) && isfinite(y) && isfinite(z) && z > 0.f) ? 0 : 1;
    }
  }
  if (local) atomicAdd(cnt, local);
}

void launch_count_bad(const float* a, int64_t n, int mode, int32_t* cnt, cudaStream_t s) {
  if (n <= 0) return;
  const int grid = (int)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048);
  count_bad_kernel<<<grid, 256, 0, s>>>(a, n, mode, cnt);
}

// Evaluation points of problem pidx -> float4 (x, y, z, problem) at the global offset.
__global__ void pack_points_kernel(int64_t n, const float* __restrict__ xyz, int pidx,
                                   float4* __restrict__ ppos) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    ppos[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], __int_as_float(pidx));
}

void launch_pack_points(int64_t n, const float* xyz, int pidx, float4* ppos, cudaStream_t s) {
  if (n <= 0) return;
  const int grid = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
  pack_points_kernel<<<grid, 256, 0, s>>>(n, xyz, pidx, ppos);
}

}  // namespace dbie
