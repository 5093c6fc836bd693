// pxe.cu -- pixel-exact near field (the exact near-field integration of the lambda = 0 kernel).
//
// For a point with z <= near_z the magnetogram is read as constant on each pixel rectangle
// (hx x hy around the pixel centre).  The lambda = 0 part of the DBIE kernel (Eq. 6),
// K0 = z / (2 pi r^3), is integrated exactly over every pixel; the lambda-dependent remainder
// z [lambda r sin(lambda r) + cos(lambda r) - 1] / (2 pi r^3) stays on the midpoint rule of
// Eq. 16.  This removes the midpoint rule's lattice error of K0 (8e-3 of B at z = 1 pixel, 0.24
// at z = 0.5); the remainder's is ~lambda^2 z smaller.  The correction
//   c_ik = int_pixel K0 - dA K0(r_ik)   (and its derivatives with respect to the point)
// does not depend on lambda: a solve computes sum_k c_ik B0_k once per point and every round adds
// it to B and grad B; the lambda-derivatives are those of the midpoint sums.
//
// Evaluation.  The integral over a rectangle is the solid angle over 2 pi: with
// F(a, b) = arctan(a b / (z R)), R = |(a, b, z)|, corners a = x_c - x_i, b = y_c - y_i,
//   int K0 = [F(a1, b1) - F(a0, b1) - F(a1, b0) + F(a0, b0)] / 2 pi,
//   dF/da = b z / (R (a^2 + z^2)),  dF/db = a z / (R (b^2 + z^2)),
//   dF/dz = -a b (R^2 + z^2) / (R (a^2 + z^2) (b^2 + z^2)),  a corner moving as -x_i.
// Far from the point the four arctangents nearly cancel (the pixel's share is ~dA z / r^3 while
// each F is ~pi / 2), which FP32 cannot resolve.  So the mixed form integrates the (2W+1)^2
// pixels around the point exactly in FP64 and every other pixel by a 3 x 3 Gauss-Legendre rule
// in FP32 (its error there is below 1e-7 of the absolute-value sum, beyond W = 3); the FP64 form
// integrates every pixel exactly in FP64.
//
// The exact rectangle integral is evaluated as one atan2 of the product of the four corner
// factors z R + i a b (pixel_exact).
//
// Kernels.  Correction: pxe_window (FP64 window sums, one warp per point) and pxe_gauss (the other
// pixels' FP32 Gauss sums, one CTA per near point, added to it), or pxe_exact in the FP64 form.
// Transpose: pxe_compact (stable list of the near points); pxe_adj (the Gauss-rule pairs, one
// thread per pixel and chunk of near points, the points through shared memory); pxe_bin_* and
// pxe_adj_window (the window pairs, pixel-major over the near points binned by nearest pixel);
// pxe_adj_reduce (the parts summed in order into dL/dB0).
#include <type_traits>

#include "kernels.h"

namespace dbie {

constexpr int PXE_NT = 128;

// Per-pixel correction in units of b = B0 dA / 2 pi:  w = [int_pixel z / r^3 - dA z / r^3] / dA
// and its derivatives with respect to the point (x_i, y_i, z); dx = x_i - x_k, dy = y_i - y_k.
// The pixel is the hx x hy rectangle; dA is the midpoint rule's pixel area (usually hx hy).

// Exactly, in FP64 (the solid angle).  The four corner terms s_c arctan(a_c b_c / (z R_c)) are
// summed as one argument: arctan(ab / (zR)) is the argument of zR + i ab, so their signed sum is
// the argument of the product of the factors zR + i s_c a_c b_c (one atan2 instead of four
// arctangents and their divisions).  The sum is 2 pi times the pixel's weight, in (0, 2 pi), so a
// negative atan2 is taken modulo 2 pi.  The derivatives share 1 / (R (a^2 + z^2) (b^2 + z^2)).
__device__ __forceinline__ void pixel_exact(double dx, double dy, double z, double hx, double hy,
                                            double inv_dA, double w[4]) {
  const double ca[2] = {-dx - 0.5 * hx, -dx + 0.5 * hx}, cb[2] = {-dy - 0.5 * hy, -dy + 0.5 * hy};
  const double zz = z * z;
  double pr = 1.0, pim = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int u = c >> 1, t = c & 1;
    const double s = (u == t) ? 1.0 : -1.0;
    const double a = ca[u], b = cb[t];
    const double a2 = a * a + zz, b2 = b * b + zz, R2 = a2 + b * b, R = sqrt(R2);
    const double fr = z * R, fi = s * (a * b);
    const double nr = pr * fr - pim * fi;
    pim = pr * fi + pim * fr;
    pr = nr;
    const double inv = 1.0 / (R * a2 * b2);
    gx -= s * (b * z * b2 * inv);
    gy -= s * (a * z * a2 * inv);
    gz -= s * (a * b * (R2 + zz) * inv);
  }
  double v = atan2(pim, pr);
  if (v < 0.0) v += TWO_PI;
  const double r2 = dx * dx + dy * dy + zz, ri = 1.0 / sqrt(r2), ri2 = ri * ri, ri3 = ri2 * ri;
  const double u5 = -3.0 * z * ri3 * ri2;
  w[0] = v * inv_dA - z * ri3;
  w[1] = gx * inv_dA - u5 * dx;
  w[2] = gy * inv_dA - u5 * dy;
  w[3] = gz * inv_dA - (ri3 + u5 * z);
}

// z / r^3 and its derivatives with respect to the point, FP32.
__device__ __forceinline__ void k0_terms(float dx, float dy, float z, float zz, float t[4]) {
  const float ri = rsqrtf(dx * dx + dy * dy + zz);
  const float ri2 = ri * ri, ri3 = ri2 * ri;
  const float u = -3.0f * z * ri3 * ri2;   // -3 z / r^5
  t[0] = z * ri3;
  t[1] = u * dx;
  t[2] = u * dy;
  t[3] = ri3 + u * z;
}

// By the 3 x 3 Gauss-Legendre rule on the pixel, FP32 (pixels away from the point);
// ga = hx hy / dA.
__device__ __forceinline__ void pixel_gauss(float dx, float dy, float z, float zz, float hx,
                                            float hy, float ga, float w[4]) {
  const float gxi = 0.3872983346207417f;        // sqrt(3/5) / 2: abscissae on a unit pixel
  const float gw[3] = {0.2777777777777778f, 0.4444444444444444f, 0.2777777777777778f};  // (5,8,5)/18
  const float ox[3] = {-gxi * hx, 0.0f, gxi * hx}, oy[3] = {-gxi * hy, 0.0f, gxi * hy};
  float t[4];
  k0_terms(dx, dy, z, zz, t);
  // the centre Gauss point coincides with the midpoint: weight ga (4/9)^2 - 1
  const float wc = ga * gw[1] * gw[1] - 1.0f;
#pragma unroll
  for (int m = 0; m < 4; ++m) w[m] = wc * t[m];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (a == 1 && b == 1) continue;
      k0_terms(dx - ox[a], dy - oy[b], z, zz, t);
      const float wab = ga * gw[a] * gw[b];
#pragma unroll
      for (int m = 0; m < 4; ++m) w[m] += wab * t[m];
    }
}

// Height below which point i is corrected: zmax >= 0 for every problem, else the problem's own.
__device__ __forceinline__ bool pxe_near(const ProbDesc& pd, float z, double zmax) {
  const double lim = zmax >= 0.0 ? zmax : pd.pxe_z;
  return lim > 0.0 && (double)z <= lim;
}

__device__ __forceinline__ int64_t tile_base(int64_t k) {
  return (k / TILE) * (int64_t)(NFIELD * TILE) + (k % TILE);
}

// Window of the mixed form: pixels within W of the pixel nearest to the point (clipped).
struct Win {
  long i0, i1, j0, j1;
  __device__ bool has(long i, long j) const { return i >= i0 && i <= i1 && j >= j0 && j <= j1; }
};
__device__ __forceinline__ Win window_of(const ProbDesc& pd, double x, double y) {
  const long ix = lrint((x - pd.x0) / pd.hx), iy = lrint((y - pd.y0) / pd.hy);
  const long W = NEAR_W;
  Win w;
  w.i0 = ix - W < 0 ? 0 : ix - W;
  w.i1 = ix + W > pd.nx - 1 ? pd.nx - 1 : ix + W;
  w.j0 = iy - W < 0 ? 0 : iy - W;
  w.j1 = iy + W > pd.ny - 1 ? pd.ny - 1 : iy + W;
  return w;
}

// corr[12 i ..]: dB_p (3), then d(dB_p/dx_j) at 3 + 3 p + j; zero for points above the height.
// Mixed form, in two kernels with their own register budgets: pxe_window_kernel sums the window
// pixels exactly in FP64 (one warp per point) and writes corr; pxe_gauss_kernel then adds the FP32
// Gauss-rule sum over the other pixels (one CTA per near point).  FP64 form: pxe_exact_kernel,
// every pixel exactly.

__device__ __forceinline__ void add_exact12(const ProbDesc& pd, int64_t k, double xd, double yd,
                                            double zd, double inv_dA, double acc[12]) {
  const int64_t base = tile_base(k);
  double w[4];
  pixel_exact(xd - pd.tiles64[base], yd - pd.tiles64[base + TILE], zd, pd.hx, pd.hy, inv_dA, w);
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const double b = pd.tiles64[base + (2 + p) * TILE];
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[4 * p + m] += b * w[m];
  }
}

__device__ __forceinline__ void store12(double* out, int m, double v) {
  const int p = m >> 2, e = m & 3;
  out[e == 0 ? p : 3 + 3 * p + (e - 1)] = v;
}

__global__ void pxe_window_kernel(const ProbDesc* __restrict__ probs, int64_t n,
                                  const float4* __restrict__ pos, double zmax,
                                  double* __restrict__ corr) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
    const float4 p4 = pos[i];
    const ProbDesc& pd = probs[__float_as_int(p4.w)];
    double acc[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) acc[m] = 0.0;
    if (pxe_near(pd, p4.z, zmax)) {
      const double xd = p4.x, yd = p4.y, zd = p4.z, inv_dA = 1.0 / pd.area;
      const Win win = window_of(pd, xd, yd);
      const long wi = win.i1 - win.i0 + 1, wj = win.j1 - win.j0 + 1;
      if (wi > 0 && wj > 0)
        for (long e = lane; e < wi * wj; e += 32)
          add_exact12(pd, (win.j0 + e / wi) * (int64_t)pd.nx + (win.i0 + e % wi), xd, yd, zd,
                      inv_dA, acc);
    }
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      double v = acc[m];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) store12(corr + 12 * i, m, v);
    }
  }
}

// Block sum of v[12] (every thread of the block calls it); thread t < 12 gets entry t.
__device__ __forceinline__ double block_sum12(double (*red)[12], const double v[12], int lane,
                                              int warp) {
#pragma unroll
  for (int m = 0; m < 12; ++m) {
    double x = v[m];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) red[warp][m] = x;
  }
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 12)
    for (int w = 0; w < PXE_NT / 32; ++w) t += red[w][threadIdx.x];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(PXE_NT, 8) pxe_gauss_kernel(const ProbDesc* __restrict__ probs,
                                                               int64_t n,
                                                               const float4* __restrict__ pos,
                                                               double zmax,
                                                               double* __restrict__ corr) {
  __shared__ double red[PXE_NT / 32][12];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const float4 p4 = pos[i];
    const ProbDesc& pd = probs[__float_as_int(p4.w)];
    if (!pxe_near(pd, p4.z, zmax)) continue;   // the same branch for the whole block
    const Win win = window_of(pd, (double)p4.x, (double)p4.y);
    const int64_t npix = (int64_t)pd.nx * pd.ny;
    const float xf = p4.x, yf = p4.y, z = p4.z, zz = z * z;
    const float hx = (float)pd.hx, hy = (float)pd.hy, ga = (float)(pd.hx * pd.hy / pd.area);
    float acc[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) acc[m] = 0.0f;
    // column and row of pixel k, advanced with k (no integer division in the loop)
    int ci = (int)(threadIdx.x % pd.nx), cj = (int)(threadIdx.x / pd.nx);
    const int step_i = PXE_NT % pd.nx, step_j = PXE_NT / pd.nx;
    for (int64_t k = threadIdx.x; k < npix; k += PXE_NT) {
      const bool in_win = win.has(ci, cj);
      ci += step_i;
      cj += step_j;
      if (ci >= pd.nx) {
        ci -= pd.nx;
        ++cj;
      }
      if (in_win) continue;
      const int64_t base = tile_base(k);
      float w[4];
      pixel_gauss(xf - pd.tiles32[base], yf - pd.tiles32[base + TILE], z, zz, hx, hy, ga, w);
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const float b = pd.tiles32[base + (2 + p) * TILE];
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[4 * p + m] += b * w[m];
      }
    }
    double accd[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) accd[m] = (double)acc[m];
    const double v = block_sum12(red, accd, lane, warp);
    if (threadIdx.x < 12) {
      const int p = threadIdx.x >> 2, e = threadIdx.x & 3;
      corr[12 * i + (e == 0 ? p : 3 + 3 * p + (e - 1))] += v;   // after the window's sum
    }
  }
}

__global__ void __launch_bounds__(PXE_NT) pxe_exact_kernel(const ProbDesc* __restrict__ probs,
                                                           int64_t n,
                                                           const float4* __restrict__ pos,
                                                           double zmax,
                                                           double* __restrict__ corr) {
  __shared__ double red[PXE_NT / 32][12];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const float4 p4 = pos[i];
    const ProbDesc& pd = probs[__float_as_int(p4.w)];
    double* out = corr + 12 * i;
    if (!pxe_near(pd, p4.z, zmax)) {   // the same branch for the whole block
      if (threadIdx.x < 12) out[threadIdx.x] = 0.0;
      continue;
    }
    const double xd = p4.x, yd = p4.y, zd = p4.z, inv_dA = 1.0 / pd.area;
    const int64_t npix = (int64_t)pd.nx * pd.ny;
    double acc[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) acc[m] = 0.0;
    for (int64_t k = threadIdx.x; k < npix; k += PXE_NT) add_exact12(pd, k, xd, yd, zd, inv_dA, acc);
    const double v = block_sum12(red, acc, lane, warp);
    if (threadIdx.x < 12) store12(out, threadIdx.x, v);
  }
}

void launch_pxe_corr(bool fp64, const ProbDesc* probs, int64_t n, const float4* pos, double zmax,
                     double* corr, int grid, cudaStream_t s) {
  if (n <= 0) return;
  const int g = (int)(n < grid ? n : grid);
  if (fp64) {
    pxe_exact_kernel<<<g, PXE_NT, 0, s>>>(probs, n, pos, zmax, corr);
  } else {
    const int64_t gw = (n * 32 + 255) / 256;
    pxe_window_kernel<<<(int)(gw < grid ? gw : grid), 256, 0, s>>>(probs, n, pos, zmax, corr);
    pxe_gauss_kernel<<<g, PXE_NT, 0, s>>>(probs, n, pos, zmax, corr);
  }
}

// Stable list of the points with z <= zmax (one block: each thread counts a contiguous range,
// a block scan gives the offsets, then each thread writes its range in order).
constexpr int PXE_SCAN = 1024;
__global__ void __launch_bounds__(PXE_SCAN) pxe_compact_kernel(int64_t n,
                                                               const float4* __restrict__ pos,
                                                               double zmax,
                                                               int32_t* __restrict__ list,
                                                               int32_t* __restrict__ cnt) {
  __shared__ int32_t s[PXE_SCAN];
  const int t = threadIdx.x;
  const int64_t per = (n + PXE_SCAN - 1) / PXE_SCAN;
  const int64_t lo = t * per, hi = lo + per < n ? lo + per : n;
  int32_t c = 0;
  for (int64_t i = lo; i < hi; ++i) c += ((double)pos[i].z <= zmax) ? 1 : 0;
  s[t] = c;
  __syncthreads();
  for (int off = 1; off < PXE_SCAN; off <<= 1) {
    const int32_t v = t >= off ? s[t - off] : 0;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  int32_t o = s[t] - c;
  for (int64_t i = lo; i < hi; ++i)
    if ((double)pos[i].z <= zmax) list[o++] = (int32_t)i;
  if (t == PXE_SCAN - 1) *cnt = s[t];
}

// Transpose of one problem's correction: sum_i sum_m w_ipm c^m_ik over the listed points
// (c^m: the per-pixel correction and its derivatives, as pxe_corr uses them), for chunk
// blockIdx.y of the list, into part[(chunk * npix + k) * 3 + p]; pxe_adj_reduce_kernel adds the
// chunks in order (times dA / 2 pi) to gB0.  Weights: FULL, 12 per point at 4 p + m; otherwise
// 3 per point (gB_p, m = 0 only).
template <bool FP64, bool FULL>
__global__ void __launch_bounds__(PXE_NT) pxe_adj_kernel(const ProbDesc* __restrict__ prob,
                                                         const int32_t* __restrict__ list,
                                                         const int32_t* __restrict__ cnt,
                                                         const float4* __restrict__ pos,
                                                         const double* __restrict__ w,
                                                         double* __restrict__ part) {
  constexpr int NW = FULL ? 12 : 3;
  // weights in the working precision (the mixed form converts once per point, not per pair:
  // FP64-to-FP32 conversions run on GB300's narrow FP64 pipe)
  using WT = typename std::conditional<FP64, double, float>::type;
  __shared__ float sx[PXE_NT], sy[PXE_NT], sz[PXE_NT];
  __shared__ int32_t sw0[PXE_NT];   // window origin of each point (packed i0, j0), mixed form
  __shared__ WT sw[NW][PXE_NT];
  const ProbDesc& pd = *prob;
  const int64_t npix = (int64_t)pd.nx * pd.ny;
  const int64_t k = blockIdx.x * (int64_t)PXE_NT + threadIdx.x;
  const bool live = k < npix;
  const int64_t base = tile_base(live ? k : 0);
  const long ki = live ? (long)(k % pd.nx) : 0, kj = live ? (long)(k / pd.nx) : 0;
  const double xk = pd.tiles64[base], yk = pd.tiles64[base + TILE];
  const float xkf = pd.tiles32[base], ykf = pd.tiles32[base + TILE];
  const float hx = (float)pd.hx, hy = (float)pd.hy, ga = (float)(pd.hx * pd.hy / pd.area);
  const double inv_dA = 1.0 / pd.area;
  double hi[3] = {0.0, 0.0, 0.0};
  const int m_all = *cnt;
  const int jb = (int)(((int64_t)m_all * blockIdx.y) / gridDim.y);
  const int m = (int)(((int64_t)m_all * (blockIdx.y + 1)) / gridDim.y);
  for (int j0 = jb; j0 < m; j0 += PXE_NT) {
    __syncthreads();
    const int j = j0 + threadIdx.x;
    if (j < m) {
      const int64_t q = list[j];
      const float4 p4 = pos[q];
      sx[threadIdx.x] = p4.x;
      sy[threadIdx.x] = p4.y;
      sz[threadIdx.x] = p4.z;
      const long ix = lrint(((double)p4.x - pd.x0) / pd.hx), iy = lrint(((double)p4.y - pd.y0) / pd.hy);
      // nearest pixel, clamped to a range that keeps the packing exact
      const long cx = ix < -32768 ? -32768 : (ix > 32767 ? 32767 : ix);
      const long cy = iy < -32768 ? -32768 : (iy > 32767 ? 32767 : iy);
      sw0[threadIdx.x] = (int32_t)(((cy + 32768) << 16) | (cx + 32768));
#pragma unroll
      for (int e = 0; e < NW; ++e) sw[e][threadIdx.x] = (WT)w[NW * q + e];
    }
    __syncthreads();
    if (!live) continue;
    const int len = m - j0 < PXE_NT ? m - j0 : PXE_NT;
    float acc[3] = {0.0f, 0.0f, 0.0f};
    for (int jj = 0; jj < len; ++jj) {
      if constexpr (!FP64) {
        // window pairs are summed exactly by pxe_adj_window_kernel
        const int32_t pk = sw0[jj];
        const long ix = (long)(pk & 0xffff) - 32768, iy = (long)((pk >> 16) & 0xffff) - 32768;
        if (ki >= ix - NEAR_W && ki <= ix + NEAR_W && kj >= iy - NEAR_W && kj <= iy + NEAR_W)
          continue;
      }
      if constexpr (FP64) {
        double c[4];
        pixel_exact((double)sx[jj] - xk, (double)sy[jj] - yk, (double)sz[jj], pd.hx, pd.hy,
                    inv_dA, c);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          if constexpr (FULL)
            hi[p] += (double)sw[4 * p][jj] * c[0] + (double)sw[4 * p + 1][jj] * c[1] +
                     (double)sw[4 * p + 2][jj] * c[2] + (double)sw[4 * p + 3][jj] * c[3];
          else
            hi[p] += (double)sw[p][jj] * c[0];
        }
      } else {
        const float z = sz[jj];
        float c[4];
        pixel_gauss(sx[jj] - xkf, sy[jj] - ykf, z, z * z, hx, hy, ga, c);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          if constexpr (FULL)
            acc[p] += sw[4 * p][jj] * c[0] + sw[4 * p + 1][jj] * c[1] + sw[4 * p + 2][jj] * c[2] +
                      sw[4 * p + 3][jj] * c[3];
          else
            acc[p] += sw[p][jj] * c[0];
        }
      }
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) hi[p] += (double)acc[p];
  }
  if (!live) return;
  double* o = part + ((int64_t)blockIdx.y * npix + k) * 3;
#pragma unroll
  for (int p = 0; p < 3; ++p) o[p] = hi[p];
}

// ---- the window pairs of the transpose (mixed form), pixel-major without divergence ----------
// Near points are binned by their nearest pixel (ix, iy) on the lattice extended by W on every
// side; pixel (i, j) then takes the points of the (2W+1)^2 bins around it, in bin order and, within
// a bin, in near-list order (a stable counting sort), so the sums do not depend on the schedule.
__device__ __forceinline__ int64_t bin_of(const ProbDesc& pd, float4 p4) {
  const long bx = pd.nx + 2 * NEAR_W, by = pd.ny + 2 * NEAR_W;
  const long ix = lrint(((double)p4.x - pd.x0) / pd.hx) + NEAR_W;
  const long iy = lrint(((double)p4.y - pd.y0) / pd.hy) + NEAR_W;
  return (ix >= 0 && ix < bx && iy >= 0 && iy < by) ? (int64_t)iy * bx + ix : -1;
}

__global__ void pxe_bin_count_kernel(const ProbDesc* __restrict__ prob,
                                     const int32_t* __restrict__ list,
                                     const int32_t* __restrict__ cnt,
                                     const float4* __restrict__ pos, int32_t* __restrict__ bcount) {
  const int m = *cnt;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = bin_of(*prob, pos[list[j]]);
    if (b >= 0) atomicAdd(bcount + b, 1);
  }
}

// Exclusive prefix of bcount[0 .. nb) into boff[0 .. nb] (one block).
__global__ void __launch_bounds__(PXE_SCAN) pxe_bin_scan_kernel(int64_t nb,
                                                                const int32_t* __restrict__ bcount,
                                                                int32_t* __restrict__ boff) {
  __shared__ int32_t s[PXE_SCAN];
  const int t = threadIdx.x;
  const int64_t per = (nb + PXE_SCAN - 1) / PXE_SCAN;
  const int64_t lo = t * per, hi = lo + per < nb ? lo + per : nb;
  int32_t c = 0;
  for (int64_t i = lo; i < hi; ++i) c += bcount[i];
  s[t] = c;
  __syncthreads();
  for (int off = 1; off < PXE_SCAN; off <<= 1) {
    const int32_t v = t >= off ? s[t - off] : 0;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  int32_t o = s[t] - c;
  for (int64_t i = lo; i < hi; ++i) {
    boff[i] = o;
    o += bcount[i];
  }
  if (t == PXE_SCAN - 1) boff[nb] = s[t];
}

__global__ void pxe_bin_fill_kernel(const ProbDesc* __restrict__ prob,
                                    const int32_t* __restrict__ list,
                                    const int32_t* __restrict__ cnt,
                                    const float4* __restrict__ pos,
                                    const int32_t* __restrict__ boff, int32_t* __restrict__ bfill,
                                    int32_t* __restrict__ entries) {
  const int m = *cnt;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = bin_of(*prob, pos[list[j]]);
    if (b >= 0) entries[boff[b] + atomicAdd(bfill + b, 1)] = (int32_t)j;
  }
}

// Near-list order within each bin (insertion sort; bins hold a few points).
__global__ void pxe_bin_sort_kernel(int64_t nb, const int32_t* __restrict__ boff,
                                    int32_t* __restrict__ entries) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int32_t lo = boff[b], hi = boff[b + 1];
    for (int32_t i = lo + 1; i < hi; ++i) {
      const int32_t v = entries[i];
      int32_t j = i - 1;
      while (j >= lo && entries[j] > v) {
        entries[j + 1] = entries[j];
        --j;
      }
      entries[j + 1] = v;
    }
  }
}

template <bool FULL>
__global__ void __launch_bounds__(PXE_NT) pxe_adj_window_kernel(
    const ProbDesc* __restrict__ prob, const int32_t* __restrict__ list,
    const int32_t* __restrict__ boff, const int32_t* __restrict__ entries,
    const float4* __restrict__ pos, const double* __restrict__ w, double* __restrict__ part) {
  constexpr int NW = FULL ? 12 : 3;
  const ProbDesc& pd = *prob;
  const int64_t npix = (int64_t)pd.nx * pd.ny;
  const int64_t k = blockIdx.x * (int64_t)PXE_NT + threadIdx.x;
  if (k >= npix) return;
  const long ki = (long)(k % pd.nx), kj = (long)(k / pd.nx);
  const int64_t base = tile_base(k);
  const double xk = pd.tiles64[base], yk = pd.tiles64[base + TILE];
  const double inv_dA = 1.0 / pd.area;
  const long bx = pd.nx + 2 * NEAR_W;
  double acc[3] = {0.0, 0.0, 0.0};
  for (long dj = -NEAR_W; dj <= NEAR_W; ++dj)
    for (long di = -NEAR_W; di <= NEAR_W; ++di) {
      const int64_t b = (kj + dj + NEAR_W) * bx + (ki + di + NEAR_W);
      for (int32_t e = boff[b]; e < boff[b + 1]; ++e) {
        const int64_t q = list[entries[e]];
        const float4 p4 = pos[q];
        double c[4];
        pixel_exact((double)p4.x - xk, (double)p4.y - yk, (double)p4.z, pd.hx, pd.hy, inv_dA, c);
        const double* wq = w + NW * q;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          if constexpr (FULL)
            acc[p] += wq[4 * p] * c[0] + wq[4 * p + 1] * c[1] + wq[4 * p + 2] * c[2] +
                      wq[4 * p + 3] * c[3];
          else
            acc[p] += wq[p] * c[0];
        }
      }
    }
#pragma unroll
  for (int p = 0; p < 3; ++p) part[3 * k + p] = acc[p];
}

__global__ void pxe_adj_reduce_kernel(const ProbDesc* __restrict__ prob, int nchunk,
                                      const double* __restrict__ part, double* __restrict__ gB0) {
  const int64_t npix = (int64_t)prob->nx * prob->ny;
  const double sc = prob->area / TWO_PI;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * npix;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int y = 0; y < nchunk; ++y) v += part[y * 3 * npix + e];
    gB0[e] += sc * v;
  }
}

int pxe_adjoint_chunks(int64_t n, int64_t npix, int sm_count) {
  const int64_t gx = (npix + PXE_NT - 1) / PXE_NT;
  int64_t c = (4LL * sm_count + gx - 1) / gx;          // about four CTAs per SM
  const int64_t cmax = (n + PXE_NT - 1) / PXE_NT;       // at least one shared-memory batch each
  c = c < cmax ? c : cmax;
  return (int)(c < 1 ? 1 : (c > 65535 ? 65535 : c));
}

int64_t pxe_bins(int nx, int ny) { return (int64_t)(nx + 2 * NEAR_W) * (ny + 2 * NEAR_W); }

cudaError_t launch_pxe_adjoint(bool fp64, bool full, const ProbDesc* prob, int64_t n, int nx,
                               int ny, const float4* pos, double zmax, const double* w,
                               int32_t* list, int32_t* cnt, int32_t* bins, int nchunk,
                               double* part, double* gB0, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t npix = (int64_t)nx * ny;
  pxe_compact_kernel<<<1, PXE_SCAN, 0, s>>>(n, pos, zmax, list, cnt);
  const int nparts = nchunk + (fp64 ? 0 : 1);
  if (!fp64) {
    // bins: count [nb], offsets [nb + 1], fill [nb], entries [n]
    const int64_t nb = pxe_bins(nx, ny);
    int32_t* bcount = bins;
    int32_t* boff = bins + nb;
    int32_t* bfill = boff + nb + 1;
    int32_t* entries = bfill + nb;
    cudaError_t e = cudaMemsetAsync(bcount, 0, sizeof(int32_t) * nb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bfill, 0, sizeof(int32_t) * nb, s);
    if (e != cudaSuccess) return e;
    const int gn = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    pxe_bin_count_kernel<<<gn, 256, 0, s>>>(prob, list, cnt, pos, bcount);
    pxe_bin_scan_kernel<<<1, PXE_SCAN, 0, s>>>(nb, bcount, boff);
    pxe_bin_fill_kernel<<<gn, 256, 0, s>>>(prob, list, cnt, pos, boff, bfill, entries);
    const int gb = (int)((nb + 255) / 256 < 4096 ? (nb + 255) / 256 : 4096);
    pxe_bin_sort_kernel<<<gb, 256, 0, s>>>(nb, boff, entries);
    const int gp = (int)((npix + PXE_NT - 1) / PXE_NT);
    double* wpart = part + (int64_t)nchunk * 3 * npix;
    if (full)
      pxe_adj_window_kernel<true><<<gp, PXE_NT, 0, s>>>(prob, list, boff, entries, pos, w, wpart);
    else
      pxe_adj_window_kernel<false><<<gp, PXE_NT, 0, s>>>(prob, list, boff, entries, pos, w, wpart);
  }
  const dim3 grid((unsigned)((npix + PXE_NT - 1) / PXE_NT), (unsigned)nchunk);
#define ADJ(D, F) pxe_adj_kernel<D, F><<<grid, PXE_NT, 0, s>>>(prob, list, cnt, pos, w, part)
  if (fp64) {
    if (full) ADJ(true, true); else ADJ(true, false);
  } else {
    if (full) ADJ(false, true); else ADJ(false, false);
  }
#undef ADJ
  const int64_t e = 3 * npix;
  const int g2 = (int)((e + 255) / 256 < 8192 ? (e + 255) / 256 : 8192);
  pxe_adj_reduce_kernel<<<g2, 256, 0, s>>>(prob, nparts, part, gB0);
  return cudaGetLastError();
}

}  // namespace dbie
