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
// Kernels: pxe_corr (one CTA per near point; the window in FP64, one pixel per thread, then the
// other pixels strided over the CTA; FP64 block reduction), pxe_compact (stable list of the near
// points), pxe_adj (the transpose, one thread per pixel and chunk of near points, the points
// through shared memory) and pxe_adj_reduce (the chunks in order, added into dL/dB0).
#include "kernels.h"

namespace dbie {

constexpr int PXE_NT = 128;

// Per-pixel correction in units of b = B0 dA / 2 pi:  w = [int_pixel z / r^3 - dA z / r^3] / dA
// and its derivatives with respect to the point (x_i, y_i, z); dx = x_i - x_k, dy = y_i - y_k.
// The pixel is the hx x hy rectangle; dA is the midpoint rule's pixel area (usually hx hy).

// Exactly, in FP64 (the solid angle).
__device__ __forceinline__ void pixel_exact(double dx, double dy, double z, double hx, double hy,
                                            double inv_dA, double w[4]) {
  const double ca[2] = {-dx - 0.5 * hx, -dx + 0.5 * hx}, cb[2] = {-dy - 0.5 * hy, -dy + 0.5 * hy};
  const double zz = z * z;
  double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const double s = (u == t) ? 1.0 : -1.0;
      const double a = ca[u], b = cb[t];
      const double a2 = a * a + zz, b2 = b * b + zz, R2 = a2 + b * b, R = sqrt(R2);
      v += s * atan(a * b / (z * R));
      gx -= s * (b * z / (R * a2));
      gy -= s * (a * z / (R * b2));
      gz -= s * (a * b * (R2 + zz) / (R * a2 * b2));
    }
  const double r2 = dx * dx + dy * dy + zz, r = sqrt(r2), ri3 = 1.0 / (r2 * r);
  const double u5 = -3.0 * z * ri3 / r2;
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
template <bool FP64>
__global__ void __launch_bounds__(PXE_NT) pxe_corr_kernel(const ProbDesc* __restrict__ probs,
                                                          int64_t n,
                                                          const float4* __restrict__ pos,
                                                          double zmax, double* __restrict__ corr) {
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
    double accd[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) accd[m] = 0.0;
    auto add_exact = [&](int64_t k) {
      const int64_t base = tile_base(k);
      double w[4];
      pixel_exact(xd - pd.tiles64[base], yd - pd.tiles64[base + TILE], zd, pd.hx, pd.hy, inv_dA, w);
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const double b = pd.tiles64[base + (2 + p) * TILE];
#pragma unroll
        for (int m = 0; m < 4; ++m) accd[4 * p + m] += b * w[m];
      }
    };
    if constexpr (FP64) {
      for (int64_t k = threadIdx.x; k < npix; k += PXE_NT) add_exact(k);
    } else {
      const Win win = window_of(pd, xd, yd);
      const long wi = win.i1 - win.i0 + 1, wj = win.j1 - win.j0 + 1;
      if (wi > 0 && wj > 0)
        for (long e = threadIdx.x; e < wi * wj; e += PXE_NT)
          add_exact((win.j0 + e / wi) * (int64_t)pd.nx + (win.i0 + e % wi));
      const float xf = p4.x, yf = p4.y, z = p4.z, zz = z * z;
      const float hx = (float)pd.hx, hy = (float)pd.hy, ga = (float)(pd.hx * pd.hy / pd.area);
      float acc[12];
#pragma unroll
      for (int m = 0; m < 12; ++m) acc[m] = 0.0f;
      for (int64_t k = threadIdx.x; k < npix; k += PXE_NT) {
        if (win.has((long)(k % pd.nx), (long)(k / pd.nx))) continue;
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
#pragma unroll
      for (int m = 0; m < 12; ++m) accd[m] += (double)acc[m];
    }
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      double v = accd[m];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][m] = v;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
      double v = 0.0;
      for (int w = 0; w < PXE_NT / 32; ++w) v += red[w][threadIdx.x];
      const int p = threadIdx.x >> 2, m = threadIdx.x & 3;
      out[m == 0 ? p : 3 + 3 * p + (m - 1)] = v;
    }
    __syncthreads();
  }
}

void launch_pxe_corr(bool fp64, const ProbDesc* probs, int64_t n, const float4* pos, double zmax,
                     double* corr, int grid, cudaStream_t s) {
  if (n <= 0) return;
  const int g = (int)(n < grid ? n : grid);
  if (fp64) pxe_corr_kernel<true><<<g, PXE_NT, 0, s>>>(probs, n, pos, zmax, corr);
  else pxe_corr_kernel<false><<<g, PXE_NT, 0, s>>>(probs, n, pos, zmax, corr);
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
  __shared__ float sx[PXE_NT], sy[PXE_NT], sz[PXE_NT];
  __shared__ int32_t sw0[PXE_NT];   // window origin of each point (packed i0, j0), mixed form
  __shared__ double sw[NW][PXE_NT];
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
      for (int e = 0; e < NW; ++e) sw[e][threadIdx.x] = w[NW * q + e];
    }
    __syncthreads();
    if (!live) continue;
    const int len = m - j0 < PXE_NT ? m - j0 : PXE_NT;
    float acc[3] = {0.0f, 0.0f, 0.0f};
    for (int jj = 0; jj < len; ++jj) {
      bool exact = FP64;
      if constexpr (!FP64) {
        const int32_t pk = sw0[jj];
        const long ix = (long)(pk & 0xffff) - 32768, iy = (long)((pk >> 16) & 0xffff) - 32768;
        exact = ki >= ix - NEAR_W && ki <= ix + NEAR_W && kj >= iy - NEAR_W && kj <= iy + NEAR_W;
      }
      if (exact) {
        double c[4];
        pixel_exact((double)sx[jj] - xk, (double)sy[jj] - yk, (double)sz[jj], pd.hx, pd.hy,
                    inv_dA, c);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          if constexpr (FULL)
            hi[p] += sw[4 * p][jj] * c[0] + sw[4 * p + 1][jj] * c[1] + sw[4 * p + 2][jj] * c[2] +
                     sw[4 * p + 3][jj] * c[3];
          else
            hi[p] += sw[p][jj] * c[0];
        }
      } else {
        const float z = sz[jj];
        float c[4];
        pixel_gauss(sx[jj] - xkf, sy[jj] - ykf, z, z * z, hx, hy, ga, c);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          if constexpr (FULL)
            acc[p] += (float)sw[4 * p][jj] * c[0] + (float)sw[4 * p + 1][jj] * c[1] +
                      (float)sw[4 * p + 2][jj] * c[2] + (float)sw[4 * p + 3][jj] * c[3];
          else
            acc[p] += (float)sw[p][jj] * c[0];
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

void launch_pxe_adjoint(bool fp64, bool full, const ProbDesc* prob, int64_t n, int64_t npix,
                        const float4* pos, double zmax, const double* w, int32_t* list,
                        int32_t* cnt, int nchunk, double* part, double* gB0, cudaStream_t s) {
  if (n <= 0) return;
  pxe_compact_kernel<<<1, PXE_SCAN, 0, s>>>(n, pos, zmax, list, cnt);
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
  pxe_adj_reduce_kernel<<<g2, 256, 0, s>>>(prob, nchunk, part, gB0);
}

}  // namespace dbie
