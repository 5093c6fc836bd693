// pairsum.cuh -- the DBIE pair-sum kernels, N-body style.
//
// g1_kernel: Eq. 6 / Eq. 16 and the fixed-lambda derivatives of Eq. 13.  Each CTA holds a
//   block of queries (evaluation point + lambda triple) in registers and streams boundary tiles
//   through shared memory.
// vjp_kernel: the transpose of Eq. 16 (dL/dB0 = A^T gB): each CTA holds a block of pixels in
//   registers and streams tiles of points (with their lambda and upstream gradient), recomputing
//   a_ik instead of storing the point-by-pixel matrix.
//
//  * Work: persistent CTAs take items (problem, register block, tile range) from a device
//    counter, so many magnetograms of uneven size share one launch and small sets can be split
//    over tile ranges; each item writes FP64 partial sums for its split.
//  * Staging: one elected thread moves each tile with one cp.async.bulk (TMA bulk copy, no
//    multicast) into an NSTAGE-deep ring of shared-memory buffers guarded by mbarriers (full:
//    transaction bytes; empty: one arrival per warp).  Every wait is bounded in time.
//  * Arithmetic (mixed form): FP32 pair terms (rsqrt, sin, cos on the SFU), plain FP32 sums
//    over SUB elements, folded by an error-free two-sum (its error carried into the next
//    block) and converted to FP64 at the end of the item.  FP64 form: the same sweep in double precision.
#pragma once
#include "dbie_internal.cuh"

namespace dbie {

#ifndef DBIE_FOLD_PIXELS
#define DBIE_FOLD_PIXELS 64   // packed: each f32x2 lane sums 32 of them between folds
#endif
#ifndef DBIE_STAGED
#define DBIE_STAGED 0
#endif
#ifndef DBIE_GROUP_UNROLL
#define DBIE_GROUP_UNROLL 16
#endif
#ifndef DBIE_TRACE_ITEMS
#define DBIE_TRACE_ITEMS 0   // 1: g1 work items record their start, end and SM (G1Args::trace)
#endif
#ifndef DBIE_PACKED
#define DBIE_PACKED 1     // FP32 pair sums on pixel pairs packed in f32x2 (0: one pixel per op)
#endif
constexpr int SUB = DBIE_FOLD_PIXELS;  // pixels summed in plain FP32 before a compensated fold
constexpr int SUB1 = 32;  // elements per fold where one accumulator takes every element (adjoints,
                          // the unpacked FP32 form): the per-accumulator length of the packed form
constexpr int GROUP_UNROLL = DBIE_GROUP_UNROLL;  // 4-pixel groups unrolled within a block
static_assert(TILE % SUB == 0 && SUB % 4 == 0, "fold blocks must tile the 256-pixel tile");
// The Hessian pass folds its 30 sums every 128 pixels (64 terms per lane): with ten sums per
// component the fold is ~8 % of its FP32 work at 64.  (The objective kernels keep SUB: the error
// bound of the certified decisions is derived for that block length.)
constexpr int SUB_HESS = 128;
static_assert(TILE % SUB_HESS == 0, "fold blocks must tile the 256-pixel tile");
__host__ __device__ constexpr int fold_pixels(int var) { return var == VAR_HESS ? SUB_HESS : SUB; }

// Ring of NSTAGE shared-memory tile buffers filled by TMA bulk copies.  Thread 0 issues; all
// warps consume.  `issued` / `consumed` count tiles over the CTA's lifetime, which fixes the
// mbarrier phase parity of every wait.
template <typename Elem, int NSTAGE, int NWARP>
struct TileRing {
  Elem* buf;
  uint64_t* full;
  uint64_t* empty;
  volatile int* abort_flag;
  unsigned* err;
  uint32_t tile_elems;
  uint32_t issued, consumed;
  bool skip_issue = false;   // fault injection: never issue, so the consumers' bounded waits expire

  __device__ void init_barriers() {  // thread 0, before the first __syncthreads
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), NWARP);
    }
    fence_mbar_init();
  }
  // Thread 0: copy tile `src` into the next stage (waits until that stage is released).
  __device__ bool issue(const Elem* src) {
    if (skip_issue) return false;
    const uint32_t st = issued % NSTAGE;
    if (issued >= NSTAGE &&
        !mbar_wait_bounded(smem_addr(&empty[st]), ((issued / NSTAGE) - 1) & 1, err,
                           ERR_TIMEOUT_EMPTY)) {
      *abort_flag = 1;
      return false;
    }
    const uint32_t bytes = tile_elems * (uint32_t)sizeof(Elem);
    mbar_arrive_expect_tx(smem_addr(&full[st]), bytes);
    tma_load_1d(smem_addr(buf + st * tile_elems), src, bytes, smem_addr(&full[st]));
    ++issued;
    return true;
  }
  // All threads: wait for the next tile; warp-uniform result (nullptr on timeout).
  __device__ const Elem* wait_next() {
    const uint32_t st = consumed % NSTAGE;
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(smem_addr(&full[st]),
                                                               (consumed / NSTAGE) & 1, err,
                                                               ERR_TIMEOUT_FULL));
    if (!ok) {
      *abort_flag = 1;
      return nullptr;
    }
    return buf + st * tile_elems;
  }
  // All threads: release the tile just consumed (one arrival per warp).
  __device__ void release(int lane) {
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_addr(&empty[consumed % NSTAGE]));
    ++consumed;
  }
  // Thread 0 at the end: wait for copies still in flight before shared memory goes away.
  __device__ void drain() {
    for (uint32_t u = consumed; u < issued; ++u)
      mbar_wait_bounded(smem_addr(&full[u % NSTAGE]), (u / NSTAGE) & 1, err, ERR_TIMEOUT_DRAIN);
  }
};

// Streams tiles [t0, t1) of `tiles` through the ring, calling body(tile_ptr) for each.  The
// producer keeps NSTAGE - 1 tiles ahead and refills the stage released one tile earlier, so the
// issuing thread rarely waits for a slow warp.
template <typename Elem, int NSTAGE, int NWARP, typename Body>
__device__ __forceinline__ void sweep_tiles(TileRing<Elem, NSTAGE, NWARP>& ring, const Elem* tiles,
                                            int t0, int t1, int tid, Body&& body) {
  const int ntl = t1 - t0;
  if (tid == 0)
    for (int s = 0; s < NSTAGE && s < ntl; ++s)
      if (!ring.issue(tiles + (int64_t)(t0 + s) * ring.tile_elems)) break;
  for (int t = 0; t < ntl; ++t) {
    const Elem* tp = ring.wait_next();
    if (tp == nullptr) break;
    body(tp);
    ring.release(tid & 31);
    if (tid == 0 && t >= 1 && (t - 1) + NSTAGE < ntl && !*ring.abort_flag)
      ring.issue(tiles + (int64_t)(t0 + t - 1 + NSTAGE) * ring.tile_elems);
    if (__any_sync(0xffffffffu, *ring.abort_flag != 0)) break;
  }
}

template <typename V, int VAR, bool TIED, int NS>
__device__ __forceinline__ void accumulatev(V* acc, const TermsV<V, VAR, TIED>& t, const V b[3]) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int lp = TIED ? 0 : p;
    // (the Hessian pass adds the rounded products phi b and cos(lambda r) b / r, which its
    // row-group form sums in pairs; the near-field correction subtracts the same values)
    if constexpr (is_nv(VAR)) acc[p * NS + 0] = vfma(t.ph[lp], t.t0[p], acc[p * NS + 0]);
    else if constexpr (has_hess(VAR)) acc[p * NS + 0] = vadd(acc[p * NS + 0], t.t0[p]);
    else acc[p * NS + 0] = vfma(t.u[lp], t.rb[p], acc[p * NS + 0]);
    if constexpr (has_grad(VAR)) {
      acc[p * NS + 1] = vadd(acc[p * NS + 1], t.t1[p]);
      acc[p * NS + 2] = vfma(t.t1[p], t.dx, acc[p * NS + 2]);
      acc[p * NS + 3] = vfma(t.t1[p], t.dy, acc[p * NS + 3]);
    }
    if constexpr (has_hess(VAR))
      acc[p * NS + idx_sl(VAR)] = vadd(acc[p * NS + idx_sl(VAR)], t.tl[p]);
    else if constexpr (has_dlam(VAR))
      acc[p * NS + idx_sl(VAR)] = vfma(t.cr[lp], b[p], acc[p * NS + idx_sl(VAR)]);
    if constexpr (has_newton(VAR)) {
      acc[p * NS + IDX_TX] = vfma(t.t0[p], t.dx, acc[p * NS + IDX_TX]);
      acc[p * NS + IDX_TY] = vfma(t.t0[p], t.dy, acc[p * NS + IDX_TY]);
    }
    if constexpr (has_hess(VAR)) {
      acc[p * NS + IDX_Q] = vfma(t.sn[lp], b[p], acc[p * NS + IDX_Q]);
      acc[p * NS + IDX_UX] = vfma(t.tl[p], t.dx, acc[p * NS + IDX_UX]);
      acc[p * NS + IDX_UY] = vfma(t.tl[p], t.dy, acc[p * NS + IDX_UY]);
    }
  }
}
// Hessian-pass sums of two pixel pairs of one boundary row (one 4-pixel group, packed): the
// pixels share dy, so each dy-weighted sum (Sy, Ty, Uy) takes one product of the two terms' sum
// instead of two products: Sy += (t1a + t1b) dy with S1 += t1a + t1b, and likewise Ty with
// S0 = sum phi b and Uy with Sl = sum cos(lambda r) b / r.  17 instead of 20 operations per
// component and group.
template <typename V, bool TIED, int NS>
__device__ __forceinline__ void accumulate_hess_row(V* acc, const TermsV<V, VAR_HESS, TIED>& ta,
                                                    const TermsV<V, VAR_HESS, TIED>& tb,
                                                    const V (&ba)[3], const V (&bb)[3], V dy) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int lp = TIED ? 0 : p;
    V* a = acc + p * NS;
    const V s0 = vadd(ta.t0[p], tb.t0[p]);
    a[0] = vadd(a[0], s0);
    a[IDX_TY] = vfma(s0, dy, a[IDX_TY]);
    a[IDX_TX] = vfma(tb.t0[p], tb.dx, vfma(ta.t0[p], ta.dx, a[IDX_TX]));
    const V s1 = vadd(ta.t1[p], tb.t1[p]);
    a[1] = vadd(a[1], s1);
    a[3] = vfma(s1, dy, a[3]);
    a[2] = vfma(tb.t1[p], tb.dx, vfma(ta.t1[p], ta.dx, a[2]));
    const V sl = vadd(ta.tl[p], tb.tl[p]);
    a[idx_sl(VAR_HESS)] = vadd(a[idx_sl(VAR_HESS)], sl);
    a[IDX_UY] = vfma(sl, dy, a[IDX_UY]);
    a[IDX_UX] = vfma(tb.tl[p], tb.dx, vfma(ta.tl[p], ta.dx, a[IDX_UX]));
    a[IDX_Q] = vfma(tb.sn[lp], bb[p], vfma(ta.sn[lp], ba[p], a[IDX_Q]));
  }
}
template <int VAR, bool TIED, int NS>
__device__ __forceinline__ void accumulate32(float* acc, const Terms32<VAR, TIED>& t,
                                             const float b[3]) {
  accumulatev<float, VAR, TIED, NS>(acc, t, b);
}

template <int VAR, bool TIED, int NS>
__device__ __forceinline__ void accumulate64(double* acc, const Terms64<VAR, TIED>& t) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    if constexpr (is_nv(VAR)) acc[p * NS + 0] += t.ph[p] * t.t0[p];
    else acc[p * NS + 0] += t.t0[p];
    if constexpr (has_grad(VAR)) {
      acc[p * NS + 1] += t.t1[p];
      acc[p * NS + 2] += t.t1[p] * t.dx;
      acc[p * NS + 3] += t.t1[p] * t.dy;
    }
    if constexpr (has_dlam(VAR)) acc[p * NS + idx_sl(VAR)] += t.tl[p];
    if constexpr (has_newton(VAR)) {
      acc[p * NS + IDX_TX] += t.t0[p] * t.dx;
      acc[p * NS + IDX_TY] += t.t0[p] * t.dy;
    }
    if constexpr (has_hess(VAR)) {
      acc[p * NS + IDX_Q] += t.tq[p];
      acc[p * NS + IDX_UX] += t.tl[p] * t.dx;
      acc[p * NS + IDX_UY] += t.tl[p] * t.dy;
    }
  }
}

// Fold a plain FP32 block sum `a` into the running sum `hi` with an error-free two-sum; the
// rounding error of the fold becomes the starting value of the next block's sum (so it is not
// lost), and hi + a is the compensated total at any time.
template <typename V>
__device__ __forceinline__ void fold2(V& hi, V& a) {
  const V s = vadd(hi, a);
  const V bp = vsub(s, hi);
  const V e = vadd(vsub(hi, vsub(s, bp)), vsub(a, bp));
  hi = s;
  a = e;
}

// Locate the problem owning work item `it` (item_off is a prefix array of length nprob + 1).
__device__ __forceinline__ int find_problem(const int32_t* item_off, int nprob, int it) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(item_off + mid) <= it) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------- g1 ----
// ROWS: every aligned group of 4 tile pixels lies on one boundary row (the host checks that the
// quadrature-point grid's row length is a multiple of 4), so dy and dy^2 + z^2 are per group.
template <typename Real, int VAR, bool TIED, int P, int NT, int NSTAGE, bool SPLIT = false,
          bool ROWS = false>
__device__ __forceinline__ void g1_body(const G1Args& a) {
  constexpr int NS = nsum_per_comp(VAR);
  constexpr int NSUM = 3 * NS;
  constexpr int Q = NT * P;
  constexpr int NWARP = NT / 32;
  constexpr bool F32 = sizeof(Real) == 4;
  static_assert(!SPLIT || F32, "split positions are an FP32-form feature");
  constexpr int NF = SPLIT ? NFIELD_SPLIT : NFIELD;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[NSTAGE];
  __shared__ __align__(8) uint64_t empty_bar[NSTAGE];
  __shared__ int s_item;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x;
  TileRing<Real, NSTAGE, NWARP> ring{reinterpret_cast<Real*>(smem_raw), full_bar, empty_bar,
                                     &s_abort, a.err, (uint32_t)(NF * TILE), 0u, 0u};
  if (tid == 0) {
    ring.init_barriers();
    s_abort = 0;
  }
  __syncthreads();
  const PlanHdr plan = *a.plan;

  for (;;) {
    // Thread 0 alone decides whether to stop, so the decision is uniform across the CTA.
    if (tid == 0) s_item = s_abort ? plan.nitems : atomicAdd(a.work, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();  // every thread has read s_item before it can be overwritten
    if (it >= plan.nitems) break;
#if DBIE_TRACE_ITEMS
    const unsigned long long t_item0 = global_ns();
#endif
    // fault injection: the CTA holding item 0 (its first item) never issues a tile copy
    ring.skip_issue = a.fault == 1 && it == 0;

    const int pidx = find_problem(a.item_off, a.nprob, it);
    const ProbDesc& pd = a.probs[pidx];
    const int local = it - __ldg(a.item_off + pidx);
    const int blk = local / plan.nsplit;
    const int sp = local - blk * plan.nsplit;
    const int qtotal = __ldg(a.q_cnt + pidx);
    const int t0 = (int)(((int64_t)sp * pd.ntiles) / plan.nsplit);
    const int t1 = (int)(((int64_t)(sp + 1) * pd.ntiles) / plan.nsplit);
    const Real* tiles = F32 ? reinterpret_cast<const Real*>(pd.tiles32)
                            : reinterpret_cast<const Real*>(pd.tiles64);

    Query<Real, TIED> q[P];
    bool valid[P];
    int64_t slot[P];
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const int j = blk * Q + tid + u * NT;
      valid[u] = j < qtotal;
      slot[u] = pd.q_off + j;
      float4 pos = make_float4(0.f, 0.f, 1.f, 0.f);
      Lam4 lam = make_lam4(0.0, 0.0, 0.0);
      if (valid[u]) {
        pos = a.qpos[slot[u]];
        lam = a.qlam[slot[u]];
      }
      q[u] = make_query<Real, TIED>(pos, lam);
    }

    Real acc[P][NSUM];
    float hi[F32 ? P : 1][F32 ? NSUM : 1];
    constexpr bool PK = F32 && DBIE_PACKED;
    // packed form: lane 0 sums the even pixels of each group of 4, lane 1 the odd ones
    f32x2 acc2[PK ? P : 1][PK ? NSUM : 1], hi2[PK ? P : 1][PK ? NSUM : 1];
#pragma unroll
    for (int u = 0; u < P; ++u)
#pragma unroll
      for (int s = 0; s < NSUM; ++s) {
        acc[u][s] = Real(0);
        if constexpr (F32) hi[u][s] = 0.f;
        if constexpr (PK) acc2[u][s] = hi2[u][s] = pack2(0.f, 0.f);
      }

    sweep_tiles(ring, tiles, t0, t1, tid, [&](const Real* sx) {
      if constexpr (PK) {
        Query<f32x2, TIED> q2[P];
#pragma unroll
        for (int u = 0; u < P; ++u) q2[u] = splat_query<TIED>(q[u]);
        constexpr int SUBV = fold_pixels(VAR);
#pragma unroll 1
        for (int k0 = 0; k0 < TILE; k0 += SUBV) {
#pragma unroll GROUP_UNROLL
          for (int k = k0; k < k0 + SUBV; k += 4) {
            const float4 X = *reinterpret_cast<const float4*>(sx + k);
            const float4 Y = *reinterpret_cast<const float4*>(sx + TILE + k);
            const float4 BX = *reinterpret_cast<const float4*>(sx + 2 * TILE + k);
            const float4 BY = *reinterpret_cast<const float4*>(sx + 3 * TILE + k);
            const float4 BZ = *reinterpret_cast<const float4*>(sx + 4 * TILE + k);
            float4 XL = make_float4(0.f, 0.f, 0.f, 0.f), YL = XL;
            if constexpr (SPLIT) {
              XL = *reinterpret_cast<const float4*>(sx + 5 * TILE + k);
              YL = *reinterpret_cast<const float4*>(sx + 6 * TILE + k);
            }
            // pixel pairs (0, 1) and (2, 3) of the group
            const f32x2 px2[2] = {pack2(X.x, X.y), pack2(X.z, X.w)};
            const f32x2 py2[2] = {pack2(Y.x, Y.y), pack2(Y.z, Y.w)};
            const f32x2 pxl2[2] = {pack2(XL.x, XL.y), pack2(XL.z, XL.w)};
            const f32x2 pyl2[2] = {pack2(YL.x, YL.y), pack2(YL.z, YL.w)};
            const f32x2 b2[2][3] = {{pack2(BX.x, BX.y), pack2(BY.x, BY.y), pack2(BZ.x, BZ.y)},
                                    {pack2(BX.z, BX.w), pack2(BY.z, BY.w), pack2(BZ.z, BZ.w)}};
            f32x2 dy2[P], dyz2[P];
            if constexpr (ROWS) {
#pragma unroll
              for (int u = 0; u < P; ++u) {
                const float dy = SPLIT ? __fsub_rn(__fsub_rn(q[u].y, Y.x), YL.x)
                                       : __fsub_rn(q[u].y, Y.x);
                const float dyz = __fmaf_rn(dy, dy, q[u].z2);
                dy2[u] = pack2(dy, dy);
                dyz2[u] = pack2(dyz, dyz);
              }
            }
            if constexpr (ROWS && has_hess(VAR)) {
#pragma unroll
              for (int u = 0; u < P; ++u) {
                TermsV<f32x2, VAR, TIED> tm[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  f32x2 dx = vsub(q2[u].x, px2[h]);
                  if constexpr (SPLIT) dx = vsub(dx, pxl2[h]);
                  pair_angularv<f32x2, VAR, TIED>(q2[u], pair_geomv_dz<f32x2>(dx, dy2[u], dyz2[u]),
                                                  b2[h], tm[h]);
                }
                accumulate_hess_row<f32x2, TIED, NS>(acc2[u], tm[0], tm[1], b2[0], b2[1], dy2[u]);
              }
            } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
              for (int u = 0; u < P; ++u) {
                f32x2 dx = vsub(q2[u].x, px2[h]);
                if constexpr (SPLIT) dx = vsub(dx, pxl2[h]);
                GeomV<f32x2> g;
                if constexpr (ROWS) {
                  g = pair_geomv_dz<f32x2>(dx, dy2[u], dyz2[u]);
                } else {
                  f32x2 dy = vsub(q2[u].y, py2[h]);
                  if constexpr (SPLIT) dy = vsub(dy, pyl2[h]);
                  g = pair_geomv_d<f32x2, TIED>(q2[u], dx, dy);
                }
                TermsV<f32x2, VAR, TIED> tm;
                pair_angularv<f32x2, VAR, TIED>(q2[u], g, b2[h], tm);
                accumulatev<f32x2, VAR, TIED, NS>(acc2[u], tm, b2[h]);
              }
            }
            }
          }
#pragma unroll
          for (int u = 0; u < P; ++u)
#pragma unroll
            for (int s = 0; s < NSUM; ++s) fold2(hi2[u][s], acc2[u][s]);
        }
      } else if constexpr (F32) {
#pragma unroll 1
        for (int k0 = 0; k0 < TILE; k0 += SUB1) {
#pragma unroll GROUP_UNROLL
          for (int k = k0; k < k0 + SUB1; k += 4) {
            const float4 X = *reinterpret_cast<const float4*>(sx + k);
            const float4 Y = *reinterpret_cast<const float4*>(sx + TILE + k);
            const float4 BX = *reinterpret_cast<const float4*>(sx + 2 * TILE + k);
            const float4 BY = *reinterpret_cast<const float4*>(sx + 3 * TILE + k);
            const float4 BZ = *reinterpret_cast<const float4*>(sx + 4 * TILE + k);
            float4 XL = make_float4(0.f, 0.f, 0.f, 0.f), YL = XL;
            if constexpr (SPLIT) {
              XL = *reinterpret_cast<const float4*>(sx + 5 * TILE + k);
              YL = *reinterpret_cast<const float4*>(sx + 6 * TILE + k);
            }
            const float pxl[4] = {XL.x, XL.y, XL.z, XL.w};
            const float pyl[4] = {YL.x, YL.y, YL.z, YL.w};
            const float px[4] = {X.x, X.y, X.z, X.w};
            const float py[4] = {Y.x, Y.y, Y.z, Y.w};
            const float bx[4] = {BX.x, BX.y, BX.z, BX.w};
            const float by[4] = {BY.x, BY.y, BY.z, BY.w};
            const float bz[4] = {BZ.x, BZ.y, BZ.z, BZ.w};
#if DBIE_STAGED
            // Geometry (one SFU rsqrt per pair) of the whole group first, then the angular part.
            Geom32 gm[4][P];
#pragma unroll
            for (int e = 0; e < 4; ++e)
#pragma unroll
              for (int u = 0; u < P; ++u)
                gm[e][u] = SPLIT ? pair_geom32_split<TIED>(q[u], px[e], py[e], pxl[e], pyl[e])
                                 : pair_geom32<TIED>(q[u], px[e], py[e]);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float b[3] = {bx[e], by[e], bz[e]};
#pragma unroll
              for (int u = 0; u < P; ++u) {
                Terms32<VAR, TIED> tm;
                pair_angular32<VAR, TIED>(q[u], gm[e][u], b, tm);
                accumulate32<VAR, TIED, NS>(acc[u], tm, b);
              }
            }
#else
            float dyg[P], dyzg[P];
            if constexpr (ROWS) {
#pragma unroll
              for (int u = 0; u < P; ++u) {
                dyg[u] = SPLIT ? __fsub_rn(__fsub_rn(q[u].y, py[0]), pyl[0]) : __fsub_rn(q[u].y, py[0]);
                dyzg[u] = __fmaf_rn(dyg[u], dyg[u], q[u].z2);
              }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float b[3] = {bx[e], by[e], bz[e]};
#pragma unroll
              for (int u = 0; u < P; ++u) {
                Terms32<VAR, TIED> tm;
                if constexpr (ROWS) {
                  const float dx = SPLIT ? __fsub_rn(__fsub_rn(q[u].x, px[e]), pxl[e])
                                         : __fsub_rn(q[u].x, px[e]);
                  pair_angular32<VAR, TIED>(q[u], pair_geom32_dz<TIED>(dx, dyg[u], dyzg[u]), b, tm);
                } else if constexpr (SPLIT) {
                  pair_terms32_split<VAR, TIED>(q[u], px[e], py[e], pxl[e], pyl[e], b, tm);
                } else {
                  pair_terms32<VAR, TIED>(q[u], px[e], py[e], b, tm);
                }
                accumulate32<VAR, TIED, NS>(acc[u], tm, b);
              }
            }
#endif
          }
#pragma unroll
          for (int u = 0; u < P; ++u)
#pragma unroll
            for (int s = 0; s < NSUM; ++s) fold2(hi[u][s], acc[u][s]);
        }
      } else {
#pragma unroll 2
        for (int k = 0; k < TILE; ++k) {
          const double b[3] = {sx[2 * TILE + k], sx[3 * TILE + k], sx[4 * TILE + k]};
          const double px = sx[k], py = sx[TILE + k];
#pragma unroll
          for (int u = 0; u < P; ++u) {
            Terms64<VAR, TIED> tm;
            pair_terms64<VAR, TIED>(q[u], px, py, b, tm);
            accumulate64<VAR, TIED, NS>(acc[u], tm);
          }
        }
      }
    });

#pragma unroll
    for (int u = 0; u < P; ++u) {
      if (!valid[u]) continue;
#pragma unroll
      for (int s = 0; s < NSUM; ++s) {
        double v;
        if constexpr (PK) {
          float h0, h1, a0, a1;
          unpack2(hi2[u][s], h0, h1);
          unpack2(acc2[u][s], a0, a1);
          v = ((double)h0 + (double)h1) + ((double)a0 + (double)a1);
        } else if constexpr (F32) {
          v = (double)hi[u][s] + (double)acc[u][s];
        } else {
          v = (double)acc[u][s];
        }
        a.out[((int64_t)it * NSUM + s) * Q + (tid + u * NT)] = v;
      }
    }
#if DBIE_TRACE_ITEMS
    // debugging aid (off by default): the item's start and end time and its SM
    if (tid == 0 && a.trace) {
      unsigned smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      a.trace[3 * (int64_t)it] = t_item0;
      a.trace[3 * (int64_t)it + 1] = global_ns();
      a.trace[3 * (int64_t)it + 2] = smid | ((unsigned long long)blockIdx.x << 16);
    }
#endif
  }
  if (tid == 0) ring.drain();
}

// --------------------------------------------------------------------------- vjp ----


template <typename Real, bool TIED, int P, int NT, int NSTAGE, bool SPLIT = false>
__device__ __forceinline__ void vjp_body(const VjpArgs& a) {
  constexpr int Q = NT * P;
  constexpr int NWARP = NT / 32;
  constexpr bool F32 = sizeof(Real) == 4;
  constexpr int NL = TIED ? 1 : 3;
  constexpr int NF = SPLIT ? NFIELD_SPLIT : NFIELD;   // fields of the boundary (pixel) tiles

  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[NSTAGE];
  __shared__ __align__(8) uint64_t empty_bar[NSTAGE];
  __shared__ int s_item;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x;
  TileRing<Real, NSTAGE, NWARP> ring{reinterpret_cast<Real*>(smem_raw), full_bar, empty_bar,
                                     &s_abort, a.err, (uint32_t)(VJP_NFIELD * TILE), 0u, 0u};
  if (tid == 0) {
    ring.init_barriers();
    s_abort = 0;
  }
  __syncthreads();
  const PlanHdr plan = *a.plan;
  const Real* ptiles = F32 ? reinterpret_cast<const Real*>(a.ptiles32)
                           : reinterpret_cast<const Real*>(a.ptiles64);
  const Real* btiles = F32 ? reinterpret_cast<const Real*>(a.btiles32)
                           : reinterpret_cast<const Real*>(a.btiles64);

  for (;;) {
    if (tid == 0) s_item = s_abort ? plan.nitems : atomicAdd(a.work, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= plan.nitems) break;
    const int blk = it / plan.nsplit;
    const int sp = it - blk * plan.nsplit;
    const int t0 = (int)(((int64_t)sp * a.nptiles) / plan.nsplit);
    const int t1 = (int)(((int64_t)(sp + 1) * a.nptiles) / plan.nsplit);

    Real px[P], py[P], pxl[P], pyl[P];
    bool valid[P];
    int kpix[P];
#pragma unroll
    for (int u = 0; u < P; ++u) {
      kpix[u] = blk * Q + tid + u * NT;
      valid[u] = kpix[u] < a.npix;
      const int k = valid[u] ? kpix[u] : 0;
      px[u] = *tile_field(btiles, k, 0, NF);
      py[u] = *tile_field(btiles, k, 1, NF);
      pxl[u] = SPLIT ? *tile_field(btiles, k, 5, NF) : Real(0);
      pyl[u] = SPLIT ? *tile_field(btiles, k, 6, NF) : Real(0);
    }
    Real acc[P][3];
    float hi[F32 ? P : 1][3];
#pragma unroll
    for (int u = 0; u < P; ++u)
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        acc[u][p] = Real(0);
        if constexpr (F32) hi[u][p] = 0.f;
      }

    sweep_tiles(ring, ptiles, t0, t1, tid, [&](const Real* sx) {
      const Real* X = sx;
      const Real* Y = sx + TILE;
      const Real* Z2 = sx + 2 * TILE;
      const Real* L = sx + 3 * TILE;
      const Real* W = sx + 6 * TILE;
      if constexpr (F32) {
#pragma unroll 1
        for (int k0 = 0; k0 < TILE; k0 += SUB1) {
#pragma unroll 4
          for (int k = k0; k < k0 + SUB1; ++k) {
            const float xi = X[k], yi = Y[k], z2 = Z2[k];
            float lam[NL];
#pragma unroll
            for (int l = 0; l < NL; ++l) lam[l] = L[l * TILE + k];
            const float w[3] = {W[k], W[TILE + k], W[2 * TILE + k]};
#pragma unroll
            for (int u = 0; u < P; ++u) {
              float dx = __fsub_rn(px[u], xi), dy = __fsub_rn(py[u], yi);
              if constexpr (SPLIT) {
                dx = __fadd_rn(dx, pxl[u]);
                dy = __fadd_rn(dy, pyl[u]);
              }
              const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, z2));
              const float ri = rsqrt_mufu(r2);
              const float r = __fmul_rn(r2, ri);
              const float ri3 = __fmul_rn(__fmul_rn(ri, ri), ri);
              if constexpr (TIED) {
                const float th = __fmul_rn(lam[0], r);
                const float phi = __fmul_rn(__fmaf_rn(th, sin_mufu(th), cos_mufu(th)), ri3);
#pragma unroll
                for (int p = 0; p < 3; ++p) acc[u][p] = __fmaf_rn(phi, w[p], acc[u][p]);
              } else {
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                  const float th = __fmul_rn(lam[p], r);
                  const float phi = __fmul_rn(__fmaf_rn(th, sin_mufu(th), cos_mufu(th)), ri3);
                  acc[u][p] = __fmaf_rn(phi, w[p], acc[u][p]);
                }
              }
            }
          }
#pragma unroll
          for (int u = 0; u < P; ++u)
#pragma unroll
            for (int p = 0; p < 3; ++p) fold2(hi[u][p], acc[u][p]);
        }
      } else {
#pragma unroll 2
        for (int k = 0; k < TILE; ++k) {
          const double xi = X[k], yi = Y[k], z2 = Z2[k];
#pragma unroll
          for (int u = 0; u < P; ++u) {
            const double dx = px[u] - xi, dy = py[u] - yi;
            const double r2 = dx * dx + dy * dy + z2;
            const double ri = rsqrt(r2);
            const double r = r2 * ri;
            const double ri3 = ri * ri * ri;
#pragma unroll
            for (int p = 0; p < 3; ++p) {
              double s, c;
              const double th = L[(TIED ? 0 : p) * TILE + k] * r;
              sincos(th, &s, &c);
              acc[u][p] += (th * s + c) * ri3 * W[p * TILE + k];
            }
          }
        }
      }
    });

#pragma unroll
    for (int u = 0; u < P; ++u) {
      if (!valid[u]) continue;
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        double v;
        if constexpr (F32) v = (double)hi[u][p] + (double)acc[u][p];
        else v = (double)acc[u][p];
        a.out[((int64_t)it * 3 + p) * Q + (tid + u * NT)] = v;
      }
    }
  }
  if (tid == 0) ring.drain();
}

// ------------------------------------------------------------------- general adjoint ----
// Transposed sum with seven kernel functions per component (the adjoint of the 12 objective sums
// and their lambda-derivatives, used by the gradient through the lambda search):
//   out_pk = sum_i [ phi (W0 + W5 dx + W6 dy) + psi (W1 + W2 dx + W3 dy) + W4 cos(lambda r) / r ],
// phi = u / r^3, psi = (lambda^2 cos(lambda r) - 3 u / r^2) / r^3, dx = x_i - x_k, dy = y_i - y_k,
// with the seven weights W_m of point i and component p in its record (VJP7_NFIELD fields:
// x, y, z^2, lambda_x, lambda_y, lambda_z, then W[p * 7 + m]).
template <typename Real, bool TIED, int P, int NT, int NSTAGE, bool SPLIT = false>
__device__ __forceinline__ void vjp7_body(const VjpArgs& a) {
  constexpr int Q = NT * P;
  constexpr int NWARP = NT / 32;
  constexpr bool F32 = sizeof(Real) == 4;
  constexpr int NL = TIED ? 1 : 3;
  constexpr int NF = SPLIT ? NFIELD_SPLIT : NFIELD;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[NSTAGE];
  __shared__ __align__(8) uint64_t empty_bar[NSTAGE];
  __shared__ int s_item;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x;
  TileRing<Real, NSTAGE, NWARP> ring{reinterpret_cast<Real*>(smem_raw), full_bar, empty_bar,
                                     &s_abort, a.err, (uint32_t)(VJP7_NFIELD * TILE), 0u, 0u};
  if (tid == 0) {
    ring.init_barriers();
    s_abort = 0;
  }
  __syncthreads();
  const PlanHdr plan = *a.plan;
  const Real* ptiles = F32 ? reinterpret_cast<const Real*>(a.ptiles32)
                           : reinterpret_cast<const Real*>(a.ptiles64);
  const Real* btiles = F32 ? reinterpret_cast<const Real*>(a.btiles32)
                           : reinterpret_cast<const Real*>(a.btiles64);

  for (;;) {
    if (tid == 0) s_item = s_abort ? plan.nitems : atomicAdd(a.work, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= plan.nitems) break;
    const int blk = it / plan.nsplit;
    const int sp = it - blk * plan.nsplit;
    const int t0 = (int)(((int64_t)sp * a.nptiles) / plan.nsplit);
    const int t1 = (int)(((int64_t)(sp + 1) * a.nptiles) / plan.nsplit);

    Real px[P], py[P], pxl[P], pyl[P];
    bool valid[P];
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const int kp = blk * Q + tid + u * NT;
      valid[u] = kp < a.npix;
      const int k = valid[u] ? kp : 0;
      px[u] = *tile_field(btiles, k, 0, NF);
      py[u] = *tile_field(btiles, k, 1, NF);
      pxl[u] = SPLIT ? *tile_field(btiles, k, 5, NF) : Real(0);
      pyl[u] = SPLIT ? *tile_field(btiles, k, 6, NF) : Real(0);
    }
    // FP64 form: one accumulator per pixel and component.  FP32 form: two points per f32x2
    // (adjacent in shared memory, so one 64-bit load fetches a field of both), the thread's
    // pixels in both lanes; each lane accumulates every second point and the lanes are added at
    // the end.
    Real acc[F32 ? 1 : P][3];
    f32x2 acc2[F32 ? P : 1][3], hi2[F32 ? P : 1][3];
    f32x2 px2[F32 ? P : 1], py2[F32 ? P : 1], pxl2[F32 ? P : 1], pyl2[F32 ? P : 1];
    if constexpr (F32) {
#pragma unroll
      for (int u = 0; u < P; ++u) {
        px2[u] = pack2(px[u], px[u]);
        py2[u] = pack2(py[u], py[u]);
        pxl2[u] = pack2(pxl[u], pxl[u]);
        pyl2[u] = pack2(pyl[u], pyl[u]);
#pragma unroll
        for (int p = 0; p < 3; ++p) acc2[u][p] = hi2[u][p] = vconst<f32x2>(0.f);
      }
    } else {
#pragma unroll
      for (int u = 0; u < P; ++u)
#pragma unroll
        for (int p = 0; p < 3; ++p) acc[u][p] = Real(0);
    }

    sweep_tiles(ring, ptiles, t0, t1, tid, [&](const Real* sx) {
      const Real* X = sx;
      const Real* Y = sx + TILE;
      const Real* Z2 = sx + 2 * TILE;
      const Real* L = sx + 3 * TILE;
      const Real* W = sx + 6 * TILE;
      if constexpr (F32) {
        auto ld2 = [](const Real* q) { return *reinterpret_cast<const f32x2*>(q); };
#pragma unroll 1
        for (int k0 = 0; k0 < TILE; k0 += SUB1) {
#pragma unroll 1
          for (int k = k0; k < k0 + SUB1; k += 2) {
            const f32x2 xi = ld2(X + k), yi = ld2(Y + k), z2 = ld2(Z2 + k);
            f32x2 lam[NL], lam2[NL];
#pragma unroll
            for (int l = 0; l < NL; ++l) {
              lam[l] = ld2(L + l * TILE + k);
              lam2[l] = vmul(lam[l], lam[l]);
            }
#pragma unroll
            for (int u = 0; u < P; ++u) {
              f32x2 dx = vsub(xi, px2[u]), dy = vsub(yi, py2[u]);
              if constexpr (SPLIT) {
                dx = vsub(dx, pxl2[u]);
                dy = vsub(dy, pyl2[u]);
              }
              // A = W0 + W5 dx + W6 dy and B = W1 + W2 dx + W3 dy of the point record
              auto wA = [&](const Real* w) {
                return vfma(ld2(w + 6 * TILE), dy, vfma(ld2(w + 5 * TILE), dx, ld2(w)));
              };
              auto wB = [&](const Real* w) {
                return vfma(ld2(w + 3 * TILE), dy, vfma(ld2(w + 2 * TILE), dx, ld2(w + TILE)));
              };
              const f32x2 r2 = vfma(dx, dx, vfma(dy, dy, z2));
              const f32x2 ri = vrsqrt(r2);
              const f32x2 r = vmul(r2, ri);
              const f32x2 ri2 = vmul(ri, ri);
              const f32x2 ri3 = vmul(ri2, ri);
              const f32x2 m3ri2 = vmul(vconst<f32x2>(-3.f), ri2);
              if constexpr (TIED) {
                // one lambda: phi, psi and cos(lambda r) / r are shared by the three components
                const f32x2 th = vmul(lam[0], r);
                const f32x2 sn = vsin(th), c = vcos(th);
                const f32x2 uu = vfma(th, sn, c);
                const f32x2 ph = vmul(uu, ri3);
                const f32x2 ps = vmul(vfma(uu, m3ri2, vmul(lam2[0], c)), ri3);
                const f32x2 cr = vmul(c, ri);
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                  const Real* w = W + p * VJP7_NW * TILE + k;
                  acc2[u][p] =
                      vfma(ph, wA(w), vfma(ps, wB(w), vfma(ld2(w + 4 * TILE), cr, acc2[u][p])));
                }
              } else {
                // per component: phi A + psi B + w4 cos / r with A = w0 + w5 dx + w6 dy and
                // B = w1 + w2 dx + w3 dy, regrouped by the two factors u / r^3 and cos:
                //   (u / r^3) (A - 3 B / r^2) + cos (lambda^2 B / r^3 + w4 / r),
                // 13 operations per component instead of 14.
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                  const f32x2 th = vmul(lam[p], r);
                  const f32x2 sn = vsin(th), c = vcos(th);
                  const f32x2 uu = vfma(th, sn, c);
                  const Real* w = W + p * VJP7_NW * TILE + k;
                  const f32x2 A = wA(w), B = wB(w);
                  const f32x2 T = vfma(m3ri2, B, A);
                  const f32x2 G = vfma(vmul(lam2[p], ri3), B, vmul(ld2(w + 4 * TILE), ri));
                  acc2[u][p] = vfma(vmul(uu, ri3), T, vfma(c, G, acc2[u][p]));
                }
              }
            }
          }
#pragma unroll
          for (int u = 0; u < P; ++u)
#pragma unroll
            for (int p = 0; p < 3; ++p) fold2(hi2[u][p], acc2[u][p]);
        }
      } else {
#pragma unroll 1
        for (int k = 0; k < TILE; ++k) {
          const double xi = X[k], yi = Y[k], z2 = Z2[k];
#pragma unroll
          for (int u = 0; u < P; ++u) {
            const double dx = xi - px[u], dy = yi - py[u];
            const double r2 = dx * dx + dy * dy + z2;
            const double ri = rsqrt(r2);
            const double r = r2 * ri;
            const double ri2 = ri * ri;
            const double ri3 = ri2 * ri;
            double ph[NL], ps[NL], cr[NL];
#pragma unroll
            for (int l = 0; l < NL; ++l) {
              const double lm = L[l * TILE + k];
              double sn, c;
              const double th = lm * r;
              sincos(th, &sn, &c);
              const double uu = th * sn + c;
              ph[l] = uu * ri3;
              ps[l] = (lm * lm * c - 3.0 * uu * ri2) * ri3;
              cr[l] = c * ri;
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) {
              const int l = TIED ? 0 : p;
              const double* w = W + p * VJP7_NW * TILE + k;
              acc[u][p] += ph[l] * (w[0] + w[5 * TILE] * dx + w[6 * TILE] * dy) +
                           ps[l] * (w[TILE] + w[2 * TILE] * dx + w[3 * TILE] * dy) +
                           w[4 * TILE] * cr[l];
            }
          }
        }
      }
    });

#pragma unroll
    for (int u = 0; u < P; ++u) {
      if (!valid[u]) continue;
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        double v;
        if constexpr (F32) {
          float h0, h1, a0, a1;
          unpack2(hi2[u][p], h0, h1);
          unpack2(acc2[u][p], a0, a1);
          v = (((double)h0 + (double)a0) + (double)h1) + (double)a1;
        } else {
          v = (double)acc[u][p];
        }
        a.out[((int64_t)it * 3 + p) * Q + (tid + u * NT)] = v;
      }
    }
  }
  if (tid == 0) ring.drain();
}

// Kernel entry points.  MINB > 1 caps registers so that MINB CTAs fit on an SM; MINB = 1 leaves
// the register allocation to the compiler (a plain __launch_bounds__(NT)).
template <typename Real, int VAR, bool TIED, int P, int NT, int NSTAGE, bool SPLIT = false,
          bool ROWS = false>
__global__ void __launch_bounds__(NT) g1_kernel(const G1Args a) {
  g1_body<Real, VAR, TIED, P, NT, NSTAGE, SPLIT, ROWS>(a);
}
template <typename Real, int VAR, bool TIED, int P, int NT, int NSTAGE, int MINB,
          bool ROWS = false>
__global__ void __launch_bounds__(NT, MINB) g1_kernel_mb(const G1Args a) {
  g1_body<Real, VAR, TIED, P, NT, NSTAGE, false, ROWS>(a);
}
template <typename Real, bool TIED, int P, int NT, int NSTAGE, bool SPLIT = false>
__global__ void __launch_bounds__(NT) vjp_kernel(const VjpArgs a) {
  vjp_body<Real, TIED, P, NT, NSTAGE, SPLIT>(a);
}
template <typename Real, bool TIED, int P, int NT, int NSTAGE, int MINB>
__global__ void __launch_bounds__(NT, MINB) vjp_kernel_mb(const VjpArgs a) {
  vjp_body<Real, TIED, P, NT, NSTAGE>(a);
}
template <typename Real, bool TIED, int P, int NT, int NSTAGE, bool SPLIT = false>
__global__ void __launch_bounds__(NT) vjp7_kernel(const VjpArgs a) {
  vjp7_body<Real, TIED, P, NT, NSTAGE, SPLIT>(a);
}

}  // namespace dbie
