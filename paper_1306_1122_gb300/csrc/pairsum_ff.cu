// pairsum_ff.cu -- the pair sums of Eq. 16 (and the fixed-lambda derivatives of Eq. 13) in
// float-float arithmetic: the "FF" form.
//
// Every pair term is carried as hi + lo float pairs (ff_math.cuh): the point-pixel offsets, r and
// 1/r from the SFU reciprocal square root with Newton corrections, sin and cos of lambda r by a
// Cody-Waite reduction and a table, the products of the terms and the running sums.  The result
// agrees with the FP64 sums to about 1e-13 of the absolute-value sum, at the FP32 pipe's issue
// rate: on GB300 about ten times faster than the same sweep in native FP64.  The lambda search
// uses it to re-evaluate the queries whose simplex decision the FP32-term sums cannot certify;
// dbie_eval offers it as DBIE_PREC_FLOAT_FLOAT.
//
// Work distribution is that of the other pair-sum kernels: persistent CTAs take items
// (problem, block of 128 queries, tile range) from a device counter and stream the problem's
// boundary tiles through an mbarrier-guarded ring filled by TMA bulk copies.  One query per
// thread.  Tiles hold, per field (x, y, bx, by, bz), TILE float pairs (hi, lo) converted from the
// FP64 tiles, so the pixel positions and b = B0 dA / 2 pi enter at FP64 accuracy.
#include <type_traits>

#include "ff_math.cuh"
#include "kernels.h"
#include "pairsum.cuh"

namespace dbie {

using ff::ds;
using ff::dsv;

constexpr int FF_NT = 128;
constexpr int FF_NF = 2 * NFIELD;   // floats per pixel in a float-float tile

// Float-float tiles: per field (x, y, bx, by, bz) TILE hi parts, then TILE lo parts.
__global__ void stage_ff_kernel(const double* __restrict__ t64, int ntiles,
                                float* __restrict__ tff) {
  const int64_t total = (int64_t)ntiles * TILE;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tile = k / TILE;
    const int e = (int)(k % TILE);
    for (int f = 0; f < NFIELD; ++f) {
      const ds d = ff::from_double(t64[tile * (NFIELD * TILE) + f * TILE + e]);
      float* dst = tff + tile * (int64_t)(FF_NF * TILE) + f * 2 * TILE + e;
      dst[0] = d.hi;
      dst[TILE] = d.lo;
    }
  }
}

void launch_stage_ff(const double* t64, int ntiles, float* tff, cudaStream_t s) {
  const int64_t total = (int64_t)ntiles * TILE;
  const int grid = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  stage_ff_kernel<<<grid, 256, 0, s>>>(t64, ntiles, tff);
}

// Hi or lo part of field f for pixel k of a float-float tile.
__device__ __forceinline__ float ff_load(const float* sx, int f, int part, int k) {
  return sx[f * 2 * TILE + part * TILE + k];
}

template <int VAR, bool TIED>
__global__ void __launch_bounds__(FF_NT) g1_ff_kernel(const G1Args a) {
  static_assert(VAR == VAR_V || VAR == VAR_OBJ, "float-float form: value and objective sums");
  using D = ds;
  constexpr int NS = nsum_per_comp(VAR);
  constexpr int NSUM = 3 * NS;
  constexpr int NL = TIED ? 1 : 3;
  constexpr int NWARP = FF_NT / 32;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[NSTAGE];
  __shared__ __align__(8) uint64_t empty_bar[NSTAGE];
  __shared__ int s_item;
  __shared__ volatile int s_abort;
  __shared__ float4 s_tab[ff::SC_TABLE];

  const int tid = threadIdx.x;
  TileRing<float, NSTAGE, NWARP> ring{reinterpret_cast<float*>(smem_raw), full_bar, empty_bar,
                                      &s_abort, a.err, (uint32_t)(FF_NF * TILE), 0u, 0u};
  if (tid == 0) {
    ring.init_barriers();
    s_abort = 0;
  }
  ff::fill_sincos_table(s_tab, tid);
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

    const int j = blk * FF_NT + tid;
    const bool valid = j < qtotal;
    float4 pos = make_float4(0.f, 0.f, 1.f, 0.f);
    Lam4 lam4 = make_lam4(0.0, 0.0, 0.0);
    if (valid) {   // float-float queries of problem p start at its qff_off (0 for one problem)
      pos = a.qpos[pd.qff_off + j];
      lam4 = a.qlam[pd.qff_off + j];
    }
    const D xq = D{pos.x, 0.f}, yq = D{pos.y, 0.f};
    const D z2 = ff::two_prod(pos.z, pos.z);
    D lam[NL], lam2[NL];
    const double lamd[3] = {lam4.x, lam4.y, lam4.z};
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      lam[l] = ff::from_double(lamd[l]);
      lam2[l] = ff::mul(lam[l], lam[l]);
    }
    D acc[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = D{0.f, 0.f};

    // re-evaluation passes are often sparse (a few queries of a problem per block): a warp
    // without a valid query only keeps the tile ring's protocol (wait, release) and skips the
    // arithmetic
    const bool warp_busy = __any_sync(0xffffffffu, valid);
    // lambda r below the reduction range of sincos_ds for every pixel: |lambda| times the
    // largest distance to the quadrature grid's box (pixel centres, or Gauss points of elements
    // two node spacings wide, all inside [x0 - |hx|, x0 + 2 nx |hx|] with nx quadrature points
    // per row); otherwise (rare: a far-out trial lambda) the warp takes the path with the FP64
    // fallback, so the common path stays branch-free
    double lmax = 0.0;
#pragma unroll
    for (int l = 0; l < NL; ++l) lmax = fmax(lmax, fabs(lamd[l]));
    const double ax = fabs(pd.hx), ay = fabs(pd.hy);
    const double ex = fmax(fabs(pos.x - (pd.x0 - ax)), fabs(pos.x - (pd.x0 + 2.0 * pd.nx * ax)));
    const double ey = fmax(fabs(pos.y - (pd.y0 - ay)), fabs(pos.y - (pd.y0 + 2.0 * pd.ny * ay)));
    const double rmax = sqrt(ex * ex + ey * ey + (double)pos.z * pos.z);
    const bool warp_fast =
        __all_sync(0xffffffffu, !valid || lmax * rmax < 0.9 * (double)ff::SC_MAX_ARG);
    auto tile_body = [&](const float* sx, auto any_angle) {
#pragma unroll 1
      for (int k = 0; k < TILE; ++k) {
        const D X = D{ff_load(sx, 0, 0, k), ff_load(sx, 0, 1, k)};
        const D Y = D{ff_load(sx, 1, 0, k), ff_load(sx, 1, 1, k)};
        const D dx = ff::sub(xq, X);
        const D dy = ff::sub(yq, Y);
        // (products that feed a further float-float operation stay unnormalised: mul_nr)
        const D r2 = ff::add(ff::add(ff::mul_nr(dx, dx), ff::mul_nr(dy, dy)), z2);
        D r, ri;
        ff::sqrt_rsqrt(r2, r, ri);
        const D ri2 = ff::mul_nr(ri, ri);
        const D ri3 = ff::mul_nr(ri2, ri);
        D u[NL], c[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          const D th = ff::mul_nr(lam[l], r);
          D s;
          if constexpr (decltype(any_angle)::value) ff::sincos_ds_any(th, s_tab, s, c[l]);
          else ff::sincos_ds<float>(th, s_tab, s, c[l]);
          u[l] = ff::add(ff::mul_nr(th, s), c[l]);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const int lp = TIED ? 0 : p;
          const D rb = ff::mul_nr(ri3, D{ff_load(sx, 2 + p, 0, k), ff_load(sx, 2 + p, 1, k)});
          ff::acc_add(acc[p * NS], ff::mul_nr(u[lp], rb));
          if constexpr (has_grad(VAR)) {
            // psi b = (lambda^2 cos(lambda r) - 3 u / r^2) b / r^3
            const D w = ff::sub(ff::mul_nr(lam2[lp], c[lp]),
                                ff::mul_f_nr(ff::mul_nr(u[lp], ri2), 3.0f));
            const D t1 = ff::mul_nr(w, rb);
            ff::acc_add(acc[p * NS + 1], t1);
            ff::acc_add(acc[p * NS + 2], ff::mul_nr(t1, dx));
            ff::acc_add(acc[p * NS + 3], ff::mul_nr(t1, dy));
          }
        }
      }
    };
    sweep_tiles(ring, pd.tilesff, t0, t1, tid, [&](const float* sx) {
      if (!warp_busy) return;
      if (warp_fast) tile_body(sx, std::false_type{});
      else tile_body(sx, std::true_type{});
    });

    if (valid) {
#pragma unroll
      for (int s = 0; s < NSUM; ++s)
        a.out[((int64_t)it * NSUM + s) * FF_NT + tid] = ff::to_double(acc[s]);
    }
  }
  if (tid == 0) ring.drain();
}

template <int VAR, bool TIED>
static KernelRef ff_ref_t() {
  return KernelRef{(const void*)&g1_ff_kernel<VAR, TIED>, FF_NT, FF_NT,
                   (size_t)NSTAGE * FF_NF * TILE * sizeof(float)};
}

KernelRef g1_ref_ff(int var, bool tied) {
  if (var == VAR_V) return tied ? ff_ref_t<VAR_V, true>() : ff_ref_t<VAR_V, false>();
  return tied ? ff_ref_t<VAR_OBJ, true>() : ff_ref_t<VAR_OBJ, false>();
}

}  // namespace dbie
