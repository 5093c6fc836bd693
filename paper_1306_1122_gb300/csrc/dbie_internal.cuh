// dbie_internal.cuh -- device-side building blocks of the DBIE library (sm_103a).
//
// Layout of the boundary on the device ("tile-blocked SoA"): pixels are grouped in tiles of
// TILE consecutive row-major pixels; a tile stores TILE x, then TILE y, then TILE values of
// b_p = B_p0 * dA / (2 pi) for p = x, y, z.  One tile is one contiguous block that a single
// cp.async.bulk copy moves into shared memory.  The last tile is padded with b = 0 pixels,
// which add exactly zero to every sum.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dbie {

constexpr int TILE = 256;            // pixels (or points, for the adjoint) per tile
constexpr int NFIELD = 5;            // x, y, bx, by, bz
// FP32 tiles of element Gauss points (Eq. 15) carry their positions as float pairs (hi + lo):
// x, y, bx, by, bz, x_lo, y_lo.  The pair sums form x_i - x_k as (x_i - x_hi) - x_lo, so the
// FP32 rounding of an irrational Gauss abscissa does not enter the kernel.
constexpr int NFIELD_SPLIT = 7;
constexpr int VJP_NFIELD = 9;        // x, y, z^2, lx, ly, lz, wx, wy, wz
constexpr int VJP7_NW = 7;           // weights per component of the general adjoint (see VjpArgs)
constexpr int VJP7_NFIELD = 6 + 3 * VJP7_NW;   // x, y, z^2, lx, ly, lz, 21 weights
constexpr int NEAR_W = 3;            // near-field window half width (pixels): 7 x 7 window
constexpr double TWO_PI = 6.283185307179586476925286766559;

// Error word bits (set with atomicOr, read by the host after synchronising).
constexpr unsigned ERR_TIMEOUT_FULL = 1u;
constexpr unsigned ERR_TIMEOUT_EMPTY = 2u;
constexpr unsigned ERR_TIMEOUT_DRAIN = 4u;
constexpr unsigned ERR_BAD_PLAN = 8u;
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;   // 2 s per wait

// Pair-sum variants: which per-component sums are accumulated (Sect. 2.1 / Eq. 13):
//   S0 = sum phi b, S1 = sum psi b, Sx = sum psi (x_i - x_k) b, Sy = sum psi (y_i - y_k) b,
//   Sl = sum cos(lambda r) b / r, with phi = u / r^3, u = lambda r sin(lambda r) + cos(lambda r),
//   psi = phi'(r) / r = (lambda^2 cos(lambda r) - 3 u / r^2) / r^3.
// Then B_p = z S0, dB_p/dx = z Sx, dB_p/dy = z Sy, dB_p/dz = S0 + z^2 S1, dB_p/dlambda = z lambda Sl.
// VAR_OBJN adds Tx = sum phi (x_i - x_k) b and Ty = sum phi (y_i - y_k) b, which with S_lambda
// give the exact lambda-derivatives of the objective sums: dS0/dlambda = lambda Sl,
// dS1/dlambda = -lambda S0, dSx/dlambda = -lambda Tx, dSy/dlambda = -lambda Ty.
// VAR_HESS adds Q = sum sin(lambda r) b, Ux = sum cos(lambda r) (x_i - x_k) b / r and Uy, the
// second derivatives: dSl/dlambda = -Q, dTx/dlambda = lambda Ux, dTy/dlambda = lambda Uy.
// VAR_NV (noise variance) sums phi^2 s over a boundary whose "b" fields hold
// s = sigma^2 (dA / 2 pi)^2, so that Var B_p = z^2 S0 (B is linear in B0, Eq. 16).
enum Variant {
  VAR_V = 0, VAR_VL = 1, VAR_OBJ = 2, VAR_OBJL = 3, VAR_OBJN = 4, VAR_HESS = 5, VAR_NV = 6
};
constexpr int NVAR = 7;
__host__ __device__ constexpr int nsum_per_comp(int var) {
  return var == VAR_V ? 1 : var == VAR_VL ? 2 : var == VAR_OBJ ? 4 : var == VAR_OBJL ? 5
       : var == VAR_OBJN ? 7 : var == VAR_HESS ? 10 : 1;
}
__host__ __device__ constexpr bool has_grad(int var) {
  return var == VAR_OBJ || var == VAR_OBJL || var == VAR_OBJN || var == VAR_HESS;
}
__host__ __device__ constexpr bool has_dlam(int var) {
  return var == VAR_VL || var == VAR_OBJL || var == VAR_OBJN || var == VAR_HESS;
}
__host__ __device__ constexpr bool has_newton(int var) {
  return var == VAR_OBJN || var == VAR_HESS;
}
__host__ __device__ constexpr bool has_hess(int var) { return var == VAR_HESS; }
__host__ __device__ constexpr bool is_nv(int var) { return var == VAR_NV; }
// indices of Tx, Ty (VAR_OBJN, VAR_HESS) and of Q, Ux, Uy (VAR_HESS) within a component's block
constexpr int IDX_TX = 5, IDX_TY = 6, IDX_Q = 7, IDX_UX = 8, IDX_UY = 9;
// index of the Sl sum within a component's block
__host__ __device__ constexpr int idx_sl(int var) { return var == VAR_VL ? 1 : 4; }

// Lambda triple of a query (FP64; the mixed form rounds it to FP32 when loading).
struct __align__(32) Lam4 {
  double x, y, z, w;
};
__host__ __device__ inline Lam4 make_lam4(double x, double y, double z) { return Lam4{x, y, z, 0.0}; }

// ------------------------------------------------------------------ problem and plan ----
constexpr int MAX_GAUSS = 8;          // Gauss points per element side (Eq. 15 elements)

struct ProbDesc {
  const float* tiles32;     // tile-blocked float boundary (quadrature points)
  const double* tiles64;    // tile-blocked double boundary
  const float* tilesff;     // tile-blocked float-float boundary (hi, lo pairs of tiles64)
  int32_t ntiles;
  int32_t nx, ny;           // quadrature-point grid: pixels, or (elements x quad_g) per side
  int32_t quad_g;           // 0: pixel centres (Eq. 16); g: nine-node elements, g x g Gauss (Eq. 15)
  int32_t near_w;           // near-field window half width in quadrature-point indices
  int32_t nf32;             // fields per FP32 tile: NFIELD, or NFIELD_SPLIT (Gauss points)
  double gx[MAX_GAUSS];     // Gauss abscissae on [-1, 1] (quad_g > 0)
  double x0, y0, hx, hy;     // node (pixel-centre) origin and spacing
  double step;              // initial simplex edge of this problem's lambda search
  double g_scale;           // Delta V / Delta sigma of Eq. 9 for this problem
  double near_z;            // FP64 near field for z <= near_z (0: off)
  double pxe_z;             // pixel-exact near field for z <= pxe_z (0: off)
  double area;              // pixel area of the midpoint weights (dA; usually hx hy)
  int64_t q_off;            // first query slot of this problem
  int64_t qff_off;          // first float-float re-evaluation slot (2 per point)
  int64_t pt_off;           // first global point index
  int64_t npts;
};

// Launch plan of one pair-sum pass, written on the device (solve rounds) or by a one-thread
// kernel (single evaluations), so that kernels can be captured in CUDA graphs.
struct PlanHdr {
  int32_t nitems;           // work items = sum over problems of blocks * nsplit
  int32_t nsplit;           // tile-range splits (same for all problems of the pass)
  int32_t qper;             // queries per item (CTA size * points per thread)
  int32_t pad0;
};

struct G1Args {
  const ProbDesc* probs;
  int32_t nprob;
  int32_t fault;            // fault injection (tests): 1 = the CTA of item 0 issues no tile copy
  const PlanHdr* plan;
  const int32_t* item_off;  // [nprob + 1] prefix of items per problem
  const int32_t* q_cnt;     // [nprob] queries per problem in this pass
  int32_t* work;            // dynamic item counter (zero before the launch)
  const float4* qpos;       // [slot] x, y, z, problem index (int bits)
  const Lam4* qlam;         // [slot] lambda_x, lambda_y, lambda_z
  double* out;              // per work item a chunk of nsum * qper partial sums (see out_index)
  unsigned* err;
  unsigned long long* trace; // DBIE_TRACE_ITEMS builds: per item start, end (ns) and SM (or null)
  const Lam4* qlam0;        // [slot] difference sums only: the reference lambda of each query
};

// Position of partial sum s of the query with local index j (within its problem) for split
// `sp`: work item = item_off[problem] + (j / qper) * nsplit + sp owns a dense chunk of
// nsum * qper values, so the buffer size is bounded by the number of items, not by nsplit.
__host__ __device__ inline int64_t out_index(const PlanHdr& h, const int32_t* item_off, int pidx,
                                             int64_t j, int sp, int s, int nsum) {
  const int64_t blk = j / h.qper;
  const int64_t r = j - blk * h.qper;
  const int64_t item = (int64_t)item_off[pidx] + blk * h.nsplit + sp;
  return (item * nsum + s) * h.qper + r;
}

// Point tiles for the adjoint: per tile TILE x, y, z^2, lambda_x, lambda_y, lambda_z and the
// weights w_p = gB_p * z (padding points carry w = 0).
struct VjpArgs {
  const float* ptiles32;    // tile-blocked point records (mixed form)
  const double* ptiles64;   // (FP64 form)
  int32_t nptiles;
  int32_t npix;             // real pixels
  const float* btiles32;    // boundary tiles (pixel coordinates)
  const double* btiles64;
  const PlanHdr* plan;      // nitems = pixel blocks * nsplit
  int32_t* work;
  double* out;              // per item (pixel block, split): 3 * qper partial sums
  unsigned* err;
};

// ------------------------------------------------------------------ PTX helpers ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on an mbarrier phase: gives up after WAIT_LIMIT_NS and sets `code` in *err.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned* err,
                                                  unsigned code) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > WAIT_LIMIT_NS) {
      atomicOr(err, code);
      return false;
    }
  }
}
// TMA bulk copy global -> shared (non-tensor, non-multicast), completion counted on `bar`.
__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void* src, uint32_t bytes,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// MUFU approximations (PTX sin/cos/rsqrt .approx); argument in radians.
__device__ __forceinline__ float sin_mufu(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_mufu(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_mufu(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ------------------------------------------------------------------ per-pair terms ----
// A query (evaluation point and its lambda) held in registers.
template <typename Real, bool TIED>
struct Query {
  Real x, y, z2;
  Real l[TIED ? 1 : 3];
  Real l2[TIED ? 1 : 3];
};

template <typename Real, bool TIED>
__device__ __forceinline__ Query<Real, TIED> make_query(float4 pos, Lam4 lam) {
  Query<Real, TIED> q;
  if constexpr (sizeof(Real) == 4) {
    q.x = pos.x;
    q.y = pos.y;
    q.z2 = __fmul_rn(pos.z, pos.z);
    const float l0 = (float)lam.x, l1 = (float)lam.y, l2 = (float)lam.z;
    q.l[0] = l0;
    q.l2[0] = __fmul_rn(l0, l0);
    if constexpr (!TIED) {
      q.l[1] = l1; q.l2[1] = __fmul_rn(l1, l1);
      q.l[2] = l2; q.l2[2] = __fmul_rn(l2, l2);
    }
  } else {
    q.x = (double)pos.x;
    q.y = (double)pos.y;
    q.z2 = (double)pos.z * (double)pos.z;
    q.l[0] = lam.x;
    q.l2[0] = lam.x * lam.x;
    if constexpr (!TIED) {
      q.l[1] = lam.y; q.l2[1] = lam.y * lam.y;
      q.l[2] = lam.z; q.l2[2] = lam.z * lam.z;
    }
  }
  return q;
}

// ---------------------------------------------------------------- FP32 lanes ----
// The FP32 pair terms are written once for a "lane" type V: float (one pixel), or f32x2 (two
// pixels packed in a 64-bit register pair, PTX add/sub/mul/fma.rn.f32x2).  Each packed
// instruction rounds each lane like its scalar counterpart, and the SFU operations (rsqrt, sin,
// cos) act lane by lane.  The packed form issues one instruction for two pixels' FP32
// arithmetic.  Sequences of packed instructions are not guaranteed to keep that rounding: with
// the assembler's optimisation on (any level above 0), composed error-free transformations on
// f32x2 (a square-root refinement, a float-float sine) came out different from the scalar ones,
// as if products were fused into the following additions.  The packed terms are therefore FP32
// terms of the same accuracy, not bit copies of the scalar terms, and float-float arithmetic
// runs on scalar floats only.
struct f32x2 {
  unsigned long long v;
};
__device__ __forceinline__ f32x2 pack2(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(f32x2 x, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ f32x2 vadd(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f32x2 vsub(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f32x2 vmul(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f32x2 vfma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ float vsin(float x) { return sin_mufu(x); }
__device__ __forceinline__ float vcos(float x) { return cos_mufu(x); }
__device__ __forceinline__ float vrsqrt(float x) { return rsqrt_mufu(x); }
__device__ __forceinline__ f32x2 vsin(f32x2 x) {
  float a, b;
  unpack2(x, a, b);
  return pack2(sin_mufu(a), sin_mufu(b));
}
__device__ __forceinline__ f32x2 vcos(f32x2 x) {
  float a, b;
  unpack2(x, a, b);
  return pack2(cos_mufu(a), cos_mufu(b));
}
__device__ __forceinline__ f32x2 vrsqrt(f32x2 x) {
  float a, b;
  unpack2(x, a, b);
  return pack2(rsqrt_mufu(a), rsqrt_mufu(b));
}
template <typename V>
__device__ __forceinline__ V vconst(float a) {
  if constexpr (sizeof(V) == 4) return a;
  else return pack2(a, a);
}

// A query with every member in both lanes.
template <bool TIED>
__device__ __forceinline__ Query<f32x2, TIED> splat_query(const Query<float, TIED>& q) {
  Query<f32x2, TIED> r;
  r.x = pack2(q.x, q.x);
  r.y = pack2(q.y, q.y);
  r.z2 = pack2(q.z2, q.z2);
#pragma unroll
  for (int p = 0; p < (TIED ? 1 : 3); ++p) {
    r.l[p] = pack2(q.l[p], q.l[p]);
    r.l2[p] = pack2(q.l2[p], q.l2[p]);
  }
  return r;
}

// Per-pair factors of the FP32 form.  The running sums take them as
//   S0 += u * rb (fused), S1 += t1, Sx += t1 * dx (fused), Sy += t1 * dy (fused),
//   Sl += cr * b (fused),  with rb = b / r^3, t1 = psi b = (lambda^2 c - 3 u / r^2) rb, cr = c / r,
// so the exact contribution of a pixel is a product of two rounded FP32 factors.  Every factor
// is computed with an explicit rounding so that the near-field kernel, which replaces these
// contributions by FP64 ones, reproduces the scalar form's contributions exactly (a product of
// two FP32 values is exact in FP64); the packed form's may differ from them by a rounding of a
// factor, which the subtraction then leaves in the sum (of the order of the FP32 terms' own
// error).
template <typename V, int VAR, bool TIED>
struct TermsV {
  V dx, dy;
  V u[TIED ? 1 : 3];
  V rb[3];
  V t1[has_grad(VAR) ? 3 : 1];
  V cr[has_dlam(VAR) ? (TIED ? 1 : 3) : 1];
  V t0[has_newton(VAR) || is_nv(VAR) ? 3 : 1];  // phi b = u rb (rounded): Tx, Ty; phi s (NV)
  V sn[has_hess(VAR) ? (TIED ? 1 : 3) : 1];      // sin(lambda r), the factor of Q
  V tl[has_hess(VAR) ? 3 : 1];                   // cos(lambda r) b / r (rounded): Ux, Uy
  V ph[is_nv(VAR) ? (TIED ? 1 : 3) : 1];         // phi = u / r^3 (rounded)
};
template <int VAR, bool TIED>
using Terms32 = TermsV<float, VAR, TIED>;

// Geometry of one pair: dx, dy, r, -3/r^2 and 1/r^3 (SFU rsqrt).
template <typename V>
struct GeomV {
  V dx, dy, r, ri, m3ri2, ri3;
};
using Geom32 = GeomV<float>;

// From dx, dy and dyz = dy^2 + z^2 (rounded as fma(dy, dy, z^2)): pixels of one boundary row
// share dy and dyz, so a group of them computes these once (same bits as per pixel).
template <typename V>
__device__ __forceinline__ GeomV<V> pair_geomv_dz(V dx, V dy, V dyz) {
  GeomV<V> g;
  g.dx = dx;
  g.dy = dy;
  const V r2 = vfma(g.dx, g.dx, dyz);
  g.ri = vrsqrt(r2);
  g.r = vmul(r2, g.ri);
  const V ri2 = vmul(g.ri, g.ri);
  g.ri3 = vmul(ri2, g.ri);
  g.m3ri2 = vmul(vconst<V>(-3.f), ri2);
  return g;
}
template <typename V, bool TIED>
__device__ __forceinline__ GeomV<V> pair_geomv_d(const Query<V, TIED>& q, V dx, V dy) {
  return pair_geomv_dz<V>(dx, dy, vfma(dy, dy, q.z2));
}
template <bool TIED>
__device__ __forceinline__ Geom32 pair_geom32_dz(float dx, float dy, float dyz) {
  return pair_geomv_dz<float>(dx, dy, dyz);
}
template <bool TIED>
__device__ __forceinline__ Geom32 pair_geom32_d(const Query<float, TIED>& q, float dx, float dy) {
  return pair_geomv_d<float, TIED>(q, dx, dy);
}
template <bool TIED>
__device__ __forceinline__ Geom32 pair_geom32(const Query<float, TIED>& q, float px, float py) {
  return pair_geom32_d<TIED>(q, __fsub_rn(q.x, px), __fsub_rn(q.y, py));
}
// Same, for a pixel position given as a float pair (hi + lo).
template <bool TIED>
__device__ __forceinline__ Geom32 pair_geom32_split(const Query<float, TIED>& q, float px, float py,
                                                    float pxl, float pyl) {
  return pair_geom32_d<TIED>(q, __fsub_rn(__fsub_rn(q.x, px), pxl),
                             __fsub_rn(__fsub_rn(q.y, py), pyl));
}

// Angular part: sin, cos of lambda r (SFU) and the factors of the sums.
template <typename V, int VAR, bool TIED>
__device__ __forceinline__ void pair_angularv(const Query<V, TIED>& q, const GeomV<V>& g,
                                              const V b[3], TermsV<V, VAR, TIED>& t) {
  t.dx = g.dx;
  t.dy = g.dy;
#pragma unroll
  for (int p = 0; p < 3; ++p) t.rb[p] = vmul(g.ri3, b[p]);
#pragma unroll
  for (int p = 0; p < (TIED ? 1 : 3); ++p) {
    const V th = vmul(q.l[p], g.r);
    const V s = vsin(th), c = vcos(th);
    t.u[p] = vfma(th, s, c);
    if constexpr (is_nv(VAR)) t.ph[p] = vmul(t.u[p], g.ri3);
    if constexpr (has_hess(VAR)) t.sn[p] = s;
    if constexpr (has_newton(VAR) || is_nv(VAR)) {
      if constexpr (TIED) {
#pragma unroll
        for (int pp = 0; pp < 3; ++pp) t.t0[pp] = vmul(t.u[0], t.rb[pp]);
      } else {
        t.t0[p] = vmul(t.u[p], t.rb[p]);
      }
    }
    if constexpr (has_grad(VAR)) {
      // w = lambda^2 c - 3 u / r^2, as fma(u, -3 / r^2, lambda^2 c)
      const V w = vfma(t.u[p], g.m3ri2, vmul(q.l2[p], c));
      if constexpr (TIED) {
#pragma unroll
        for (int pp = 0; pp < 3; ++pp) t.t1[pp] = vmul(w, t.rb[pp]);
      } else {
        t.t1[p] = vmul(w, t.rb[p]);
      }
    }
    if constexpr (has_dlam(VAR)) t.cr[p] = vmul(c, g.ri);
    if constexpr (has_hess(VAR)) {
      if constexpr (TIED) {
#pragma unroll
        for (int pp = 0; pp < 3; ++pp) t.tl[pp] = vmul(t.cr[0], b[pp]);
      } else {
        t.tl[p] = vmul(t.cr[p], b[p]);
      }
    }
  }
}
template <int VAR, bool TIED>
__device__ __forceinline__ void pair_angular32(const Query<float, TIED>& q, const Geom32& g,
                                               const float b[3], Terms32<VAR, TIED>& t) {
  pair_angularv<float, VAR, TIED>(q, g, b, t);
}

template <int VAR, bool TIED>
__device__ __forceinline__ void pair_terms32(const Query<float, TIED>& q, float px, float py,
                                             const float b[3], Terms32<VAR, TIED>& t) {
  pair_angular32<VAR, TIED>(q, pair_geom32<TIED>(q, px, py), b, t);
}
template <int VAR, bool TIED>
__device__ __forceinline__ void pair_terms32_split(const Query<float, TIED>& q, float px, float py,
                                                   float pxl, float pyl, const float b[3],
                                                   Terms32<VAR, TIED>& t) {
  pair_angular32<VAR, TIED>(q, pair_geom32_split<TIED>(q, px, py, pxl, pyl), b, t);
}

// FP64 terms (used by the FP64 form and by the near-field correction).
template <int VAR, bool TIED>
struct Terms64 {
  double dx, dy;
  double t0[3];
  double t1[has_grad(VAR) ? 3 : 1];
  double tl[has_dlam(VAR) ? 3 : 1];
  double tq[has_hess(VAR) ? 3 : 1];   // sin(lambda r) b
  double ph[is_nv(VAR) ? 3 : 1];      // phi
};
// (Tx and Ty of the FP64 form are t0 * dx and t0 * dy.)

// FP64 pair terms; `sc(theta, s, c)` supplies sin and cos of lambda r (FP64 sincos by default).
template <int VAR, bool TIED, typename SinCos>
__device__ __forceinline__ void pair_terms64_sc(const Query<double, TIED>& q, double px, double py,
                                                const double b[3], Terms64<VAR, TIED>& t,
                                                SinCos&& sc) {
  constexpr int NL = TIED ? 1 : 3;
  t.dx = q.x - px;
  t.dy = q.y - py;
  const double r2 = t.dx * t.dx + t.dy * t.dy + q.z2;
  const double ri = rsqrt(r2);
  const double r = r2 * ri;
  const double ri2 = ri * ri;
  const double ri3 = ri2 * ri;
  double th[NL], s[NL], c[NL];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    th[l] = q.l[l] * r;
    sc(th[l], s[l], c[l]);
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int lp = TIED ? 0 : p;
    const double u = th[lp] * s[lp] + c[lp];
    const double rb = ri3 * b[p];
    t.t0[p] = u * rb;
    if constexpr (has_grad(VAR)) t.t1[p] = (q.l2[lp] * c[lp] - 3.0 * u * ri2) * rb;
    if constexpr (has_dlam(VAR)) t.tl[p] = c[lp] * ri * b[p];
    if constexpr (has_hess(VAR)) t.tq[p] = s[lp] * b[p];
    if constexpr (is_nv(VAR)) t.ph[p] = u * ri3;
  }
}
template <int VAR, bool TIED>
__device__ __forceinline__ void pair_terms64(const Query<double, TIED>& q, double px, double py,
                                             const double b[3], Terms64<VAR, TIED>& t) {
  pair_terms64_sc<VAR, TIED>(q, px, py, b, t,
                             [](double th, double& s, double& c) { sincos(th, &s, &c); });
}

// Address of field f of pixel (quadrature point) k in a tile-blocked boundary of nf fields.
template <typename Real>
__device__ __forceinline__ const Real* tile_field(const Real* tiles, int64_t k, int f,
                                                  int nf = NFIELD) {
  return tiles + (k / TILE) * (int64_t)(nf * TILE) + f * TILE + (k % TILE);
}

}  // namespace dbie
