// pairsum_dif.cu -- difference sums: the change of the objective sums of Eq. 16 (and of the
// fixed-lambda derivatives of Eq. 13) between two lambdas of one point, from FP32 terms whose
// error is proportional to the change.
//
// Per pixel and component, with theta = lambda r, sigma = (lambda_a + lambda_0) r / 2 and
// delta = (lambda_a - lambda_0) r / 2, the angle-sum identities give
//   cos(theta_a) - cos(theta_0)                     = -2 sin(sigma) sin(delta)
//   theta_a sin(theta_a) - theta_0 sin(theta_0)     =  2 [delta sin(sigma) cos(delta)
//                                                         + sigma cos(sigma) sin(delta)]
//   lambda_a^2 cos(theta_a) - lambda_0^2 cos(theta_0) = (lambda_a^2 - lambda_0^2) cos(sigma) cos(delta)
//                                                     - (lambda_a^2 + lambda_0^2) sin(sigma) sin(delta)
// so the change of u = theta sin(theta) + cos(theta) and of w = lambda^2 cos(theta) - 3 u / r^2
// is a sum of products that each carry a factor delta (or lambda_a - lambda_0).  Evaluated in FP32
// (SFU sine and cosine of sigma; sin and cos of delta by their Taylor polynomials for |delta| <= 1),
// every rounding and every SFU error is relative to that factor: the error of a difference sum is
// a bound times |lambda_a - lambda_0|, where the error of the plain FP32 sums is a bound times 1.
// Added to float-float sums at lambda_0, the differences give the sums at lambda_a with an error
// that shrinks with the distance between the two lambdas.  The lambda search uses them to
// re-decide near-tied comparisons against a float-float reference value of the same point.
//
// Work distribution is that of the float-float pass (pairsum_ff.cu): persistent CTAs take items
// (problem, block of 128 queries, tile range) from a device counter and read the float-float
// tiles (pixel positions as hi + lo pairs) through the same TMA / mbarrier ring.  One query per
// thread; the 12 sums are summed in FP32 over blocks of 8 pixels and the block sums in
// float-float.
#include "ff_math.cuh"
#include "kernels.h"
#include "pairsum.cuh"

namespace dbie {

constexpr int DIF_NT = 128;
constexpr int DIF_NF = 2 * NFIELD;   // floats per pixel in a float-float tile (hi, lo)
constexpr int DIF_BLK = 8;           // pixels per FP32 block sum

__device__ __forceinline__ float dif_load(const float* sx, int f, int part, int k) {
  return sx[f * 2 * TILE + part * TILE + k];
}

// sin(d), cos(d): Taylor polynomials through d^9 and d^10 for |d| <= 1 (truncation below 3e-8
// relative), the SFU beyond.
__device__ __forceinline__ void sincos_delta(float d, float& s, float& c) {
  if (fabsf(d) <= 1.0f) {
    const float d2 = d * d;
    s = d * fmaf(d2, fmaf(d2, fmaf(d2, fmaf(d2, 1.0f / 362880.0f, -1.0f / 5040.0f),
                                   1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
    c = fmaf(d2, fmaf(d2, fmaf(d2, fmaf(d2, fmaf(d2, -1.0f / 3628800.0f, 1.0f / 40320.0f),
                                        -1.0f / 720.0f), 1.0f / 24.0f), -0.5f), 1.0f);
  } else {
    s = sin_mufu(d);
    c = cos_mufu(d);
  }
}

template <bool TIED>
__global__ void __launch_bounds__(DIF_NT) g1_dif_kernel(const G1Args a) {
  using ff::ds;
  constexpr int NL = TIED ? 1 : 3;
  constexpr int NSUM = 12;
  constexpr int NWARP = DIF_NT / 32;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[NSTAGE];
  __shared__ __align__(8) uint64_t empty_bar[NSTAGE];
  __shared__ int s_item;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x;
  TileRing<float, NSTAGE, NWARP> ring{reinterpret_cast<float*>(smem_raw), full_bar, empty_bar,
                                      &s_abort, a.err, (uint32_t)(DIF_NF * TILE), 0u, 0u};
  if (tid == 0) {
    ring.init_barriers();
    s_abort = 0;
  }
  __syncthreads();
  const PlanHdr plan = *a.plan;

  for (;;) {
    if (tid == 0) s_item = s_abort ? plan.nitems : atomicAdd(a.work, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= plan.nitems) break;
    const int pidx = find_problem(a.item_off, a.nprob, it);
    const ProbDesc& pd = a.probs[pidx];
    const int local = it - __ldg(a.item_off + pidx);
    const int blk = local / plan.nsplit;
    const int sp = local - blk * plan.nsplit;
    const int qtotal = __ldg(a.q_cnt + pidx);
    const int t0 = (int)(((int64_t)sp * pd.ntiles) / plan.nsplit);
    const int t1 = (int)(((int64_t)(sp + 1) * pd.ntiles) / plan.nsplit);

    const int j = blk * DIF_NT + tid;
    const bool valid = j < qtotal;
    float4 pos = make_float4(0.f, 0.f, 1.f, 0.f);
    Lam4 la = make_lam4(0.0, 0.0, 0.0), l0 = make_lam4(0.0, 0.0, 0.0);
    if (valid) {   // slots of problem p start at its qff_off, as in the float-float pass
      pos = a.qpos[pd.qff_off + j];
      la = a.qlam[pd.qff_off + j];
      l0 = a.qlam0[pd.qff_off + j];
    }
    const float z2 = pos.z * pos.z;
    // per lambda: (la + l0) / 2, (la - l0) / 2, la^2 - l0^2 and la^2 + l0^2, formed in FP64
    float hs[NL], hd[NL], pq[NL], qq[NL];
    {
      const double a3[3] = {la.x, la.y, la.z}, b3[3] = {l0.x, l0.y, l0.z};
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        hs[l] = (float)(0.5 * (a3[l] + b3[l]));
        hd[l] = (float)(0.5 * (a3[l] - b3[l]));
        pq[l] = (float)((a3[l] - b3[l]) * (a3[l] + b3[l]));
        qq[l] = (float)(a3[l] * a3[l] + b3[l] * b3[l]);
      }
    }
    ds acc[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = ds{0.f, 0.f};

    const bool warp_busy = __any_sync(0xffffffffu, valid);
    sweep_tiles(ring, pd.tilesff, t0, t1, tid, [&](const float* sx) {
      if (!warp_busy) return;
#pragma unroll 1
      for (int k0 = 0; k0 < TILE; k0 += DIF_BLK) {
        float bs[NSUM];
#pragma unroll
        for (int s = 0; s < NSUM; ++s) bs[s] = 0.f;
#pragma unroll 2
        for (int k = k0; k < k0 + DIF_BLK; ++k) {
          const float dx = (pos.x - dif_load(sx, 0, 0, k)) - dif_load(sx, 0, 1, k);
          const float dy = (pos.y - dif_load(sx, 1, 0, k)) - dif_load(sx, 1, 1, k);
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, z2));
          const float ri = rsqrt_mufu(r2);
          const float r = r2 * ri;
          const float ri2 = ri * ri;
          const float ri3 = ri2 * ri;
          float du[NL], dw[NL];
#pragma unroll
          for (int l = 0; l < NL; ++l) {
            const float sg = hs[l] * r, dl = hd[l] * r;
            const float ss = sin_mufu(sg), cs = cos_mufu(sg);
            float sd, cd;
            sincos_delta(dl, sd, cd);
            const float cs_sd = cs * sd, ss_sd = ss * sd;
            du[l] = 2.0f * (fmaf(dl, ss * cd, sg * cs_sd) - ss_sd);
            dw[l] = fmaf(pq[l], cs * cd, fmaf(-qq[l], ss_sd, -3.0f * du[l] * ri2));
          }
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            const int lp = TIED ? 0 : p;
            const float rb = ri3 * dif_load(sx, 2 + p, 0, k);
            const float t1 = dw[lp] * rb;
            bs[4 * p + 0] = fmaf(du[lp], rb, bs[4 * p + 0]);
            bs[4 * p + 1] += t1;
            bs[4 * p + 2] = fmaf(t1, dx, bs[4 * p + 2]);
            bs[4 * p + 3] = fmaf(t1, dy, bs[4 * p + 3]);
          }
        }
#pragma unroll
        for (int s = 0; s < NSUM; ++s) {
          const ds t = ff::two_sum(acc[s].hi, bs[s]);
          acc[s] = ds{t.hi, __fadd_rn(acc[s].lo, t.lo)};
        }
      }
    });

    if (valid) {
#pragma unroll
      for (int s = 0; s < NSUM; ++s)
        a.out[((int64_t)it * NSUM + s) * DIF_NT + tid] = (double)acc[s].hi + (double)acc[s].lo;
    }
  }
  if (tid == 0) ring.drain();
}

template <bool TIED>
static KernelRef dif_ref_t() {
  return KernelRef{(const void*)&g1_dif_kernel<TIED>, DIF_NT, DIF_NT,
                   (size_t)NSTAGE * DIF_NF * TILE * sizeof(float)};
}

KernelRef g1_ref_dif(bool tied) { return tied ? dif_ref_t<true>() : dif_ref_t<false>(); }

}  // namespace dbie
