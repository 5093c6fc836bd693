// ff_math.cuh -- float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48
// significant bits.  On GB300 the FP64 pipe issues 1/64 as many operations as the FP32 pipe, so
// a pair term in float-float (several hundred FP32 operations) costs about a ninth of the same
// term in native FP64.  The building blocks are the error-free transformations of Knuth (two-sum)
// and Dekker (fast two-sum), and the exact product by a fused multiply-add.  The operations are
// written over the lane type V of dbie_internal.cuh's vadd/vsub/vmul/vfma (float here), whose
// explicitly rounded intrinsics the compiler can neither contract nor reorder.  (A version with
// two pixels per f32x2 operation measured only 9 % faster on GB300 and was dropped.)
#pragma once
#include "dbie_internal.cuh"

namespace dbie {
namespace ff {

template <typename V>
struct dsv {
  V hi, lo;
};
using ds = dsv<float>;

template <typename V>
__device__ __forceinline__ dsv<V> neg(dsv<V> x) {
  return dsv<V>{vsub(vconst<V>(0.f), x.hi), vsub(vconst<V>(0.f), x.lo)};
}
// s + e = a + b exactly (Knuth).
template <typename V>
__device__ __forceinline__ dsv<V> two_sum(V a, V b) {
  const V s = vadd(a, b);
  const V bb = vsub(s, a);
  const V e = vadd(vsub(a, vsub(s, bb)), vsub(b, bb));
  return dsv<V>{s, e};
}
// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker).
template <typename V>
__device__ __forceinline__ dsv<V> fast_two_sum(V a, V b) {
  const V s = vadd(a, b);
  return dsv<V>{s, vsub(b, vsub(s, a))};
}
// p + e = a * b exactly.
template <typename V>
__device__ __forceinline__ dsv<V> two_prod(V a, V b) {
  const V p = vmul(a, b);
  return dsv<V>{p, vfma(a, b, vsub(vconst<V>(0.f), p))};
}
// x + y; relative error about 2^-44 of |x| + |y|.
template <typename V>
__device__ __forceinline__ dsv<V> add(dsv<V> x, dsv<V> y) {
  const dsv<V> s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, vadd(s.lo, vadd(x.lo, y.lo)));
}
template <typename V>
__device__ __forceinline__ dsv<V> sub(dsv<V> x, dsv<V> y) {
  return add(x, neg(y));
}
// x * y; relative error about 2^-44.
template <typename V>
__device__ __forceinline__ dsv<V> mul(dsv<V> x, dsv<V> y) {
  const dsv<V> p = two_prod(x.hi, y.hi);
  V e = vfma(x.hi, y.lo, p.lo);
  e = vfma(x.lo, y.hi, e);
  return fast_two_sum(p.hi, e);
}
// x * f for a float f (the same in every lane).
template <typename V>
__device__ __forceinline__ dsv<V> mul_f(dsv<V> x, float f) {
  const V fv = vconst<V>(f);
  const dsv<V> p = two_prod(x.hi, fv);
  return fast_two_sum(p.hi, vfma(x.lo, fv, p.lo));
}
// x * y without the final renormalisation: hi is the rounded product, lo the exact rounding
// error plus the cross terms (|lo| a few ulp of hi).  For operands of further float-float
// operations, which take such pairs as they are; saves the fast two-sum of mul.
template <typename V>
__device__ __forceinline__ dsv<V> mul_nr(dsv<V> x, dsv<V> y) {
  const dsv<V> p = two_prod(x.hi, y.hi);
  return dsv<V>{p.hi, vfma(x.lo, y.hi, vfma(x.hi, y.lo, p.lo))};
}
template <typename V>
__device__ __forceinline__ dsv<V> mul_f_nr(dsv<V> x, float f) {
  const V fv = vconst<V>(f);
  const dsv<V> p = two_prod(x.hi, fv);
  return dsv<V>{p.hi, vfma(x.lo, fv, p.lo)};
}
// Running sum: acc.hi takes the terms by an exact two-sum, acc.lo collects the rounding errors
// and the low parts (renormalised only when the sum is read).
template <typename V>
__device__ __forceinline__ void acc_add(dsv<V>& acc, dsv<V> t) {
  const dsv<V> s = two_sum(acc.hi, t.hi);
  acc.hi = s.hi;
  acc.lo = vadd(acc.lo, vadd(s.lo, t.lo));
}
__device__ __forceinline__ double to_double(ds x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ ds from_double(double v) {
  const float hi = (float)v;
  return ds{hi, (float)(v - (double)hi)};
}

// Round to the nearest integer (ties to even) by adding and removing 1.5 * 2^23: exact for
// |x| < 2^22, with a plain FP32 add and subtract.
template <typename V>
__device__ __forceinline__ V rint_magic(V x) {
  const V m = vconst<V>(12582912.0f);
  return vsub(vadd(x, m), m);
}

// r = sqrt(x) and ri = 1 / sqrt(x) for x > 0: the SFU reciprocal square root of x.hi (relative
// error ~2^-23) followed by one Newton correction of each, computed from the exact residuals
// x - s^2 and 1 - r y, which leaves a relative error of order 2^-46.
template <typename V>
__device__ __forceinline__ void sqrt_rsqrt(dsv<V> x, dsv<V>& r, dsv<V>& ri) {
  const V y = vrsqrt(x.hi);
  const V s = vmul(x.hi, y);
  const dsv<V> p = two_prod(s, s);
  const V res = vadd(vsub(vsub(x.hi, p.hi), p.lo), x.lo);
  r = fast_two_sum(s, vmul(vmul(res, y), vconst<V>(0.5f)));
  const dsv<V> t = mul(r, dsv<V>{y, vconst<V>(0.f)});
  const V res2 = vsub(vsub(vconst<V>(1.0f), t.hi), t.lo);
  ri = fast_two_sum(y, vmul(res2, y));
}

// Cody-Waite reduction constant 2 pi = Q1 + Q2 + Q3: Q1 and Q2 carry 12 significant bits each,
// so k Q1 and k Q2 are exact in FP32 for |k| < 2^11 (|theta| up to about 12,800 rad).
constexpr float TWO_PI_1 = 0x1.92p+2f;
constexpr float TWO_PI_2 = 0x1.fb4p-10f;
constexpr float TWO_PI_3 = 0x1.4442d2p-22f;
constexpr float INV_TWO_PI = 0.159154943091895336f;
constexpr int SC_TABLE = 52;   // sin and cos of j / 16 for j = 0..51 (|t| <= pi after reduction)

// Table in shared memory, one float4 per entry: hi and lo of sin(j/16), hi and lo of cos(j/16),
// filled by the first SC_TABLE threads of the CTA from FP64 sine and cosine.
__device__ __forceinline__ void fill_sincos_table(float4* tab, int tid) {
  if (tid < SC_TABLE) {
    double s, c;
    sincos((double)tid / 16.0, &s, &c);
    const ds S = from_double(s), C = from_double(c);
    tab[tid] = make_float4(S.hi, S.lo, C.hi, C.lo);
  }
}

// Table entry for a (possibly negative) index j in float: sin is odd, cos even.  The index is
// clamped to the table, so no input (an angle beyond the reduction's range, NaN) reads outside it.
__device__ __forceinline__ void table_lookup(const float4* tab, float jf, ds& S, ds& C) {
  const float aj = fabsf(jf);
  const float4 t = tab[aj < (float)SC_TABLE ? (int)aj : SC_TABLE - 1];   // (NaN: the last entry)
  const float sg = jf < 0.0f ? -1.0f : 1.0f;
  S = ds{t.x * sg, t.y * sg};
  C = ds{t.z, t.w};
}

// sin and cos of a float-float angle (|theta| < 12,800; sincos_ds_any below takes any angle).
// theta = k 2 pi + t by a three-part
// Cody-Waite reduction (|t| <= pi), t = j/16 + tau (|tau| <= 1/32) against the table, then
//   sin(tau) = tau - tau^3/6 + tau^5/120,   cos(tau) - 1 = -tau^2/2 + tau^4/24 - tau^6/720
// (truncation below 6e-15 at |tau| = 1/32), combined by the angle-sum formulas.  Absolute error
// about 1e-13 + 5e-15 |theta|.
template <typename V>
__device__ __forceinline__ void sincos_ds(dsv<V> th, const float4* tab, dsv<V>& s_out,
                                          dsv<V>& c_out) {
  const V kf = rint_magic(vmul(th.hi, vconst<V>(INV_TWO_PI)));
  const V nk = vsub(vconst<V>(0.f), kf);
  const V a1 = vfma(nk, vconst<V>(TWO_PI_1), th.hi);                 // exact
  dsv<V> t = two_sum(a1, vmul(nk, vconst<V>(TWO_PI_2)));             // k Q2 exact
  t.lo = vadd(t.lo, vfma(nk, vconst<V>(TWO_PI_3), th.lo));
  t = two_sum(t.hi, t.lo);
  const V jf = rint_magic(vmul(t.hi, vconst<V>(16.0f)));
  const dsv<V> tau = two_sum(vsub(t.hi, vmul(jf, vconst<V>(0.0625f))), t.lo);  // exact difference
  const V t2 = vmul(tau.hi, tau.hi);
  // sin(tau): tau + tau^3 (-1/6 + tau^2/120)
  const V c3 = vmul(vmul(t2, tau.hi), vfma(t2, vconst<V>(1.0f / 120.0f), vconst<V>(-1.0f / 6.0f)));
  const dsv<V> sn = two_sum(tau.hi, vadd(tau.lo, c3));
  // cos(tau) - 1 with tau^2 = q + 2 tau.hi tau.lo, q = tau.hi^2 exact
  const dsv<V> q = two_prod(tau.hi, tau.hi);
  V cl = vfma(vsub(vconst<V>(0.f), tau.hi), tau.lo, vmul(vconst<V>(-0.5f), q.lo));
  cl = vfma(vmul(t2, t2), vfma(t2, vconst<V>(-1.0f / 720.0f), vconst<V>(1.0f / 24.0f)), cl);
  const dsv<V> cm1 = fast_two_sum(vmul(vconst<V>(-0.5f), q.hi), cl);
  dsv<V> S, C;
  table_lookup(tab, jf, S, C);
  // sin(j/16 + tau) = S + (S (cos tau - 1) + C sin tau); cos = C + (C (cos tau - 1) - S sin tau).
  // The correction terms are small (|cos tau - 1| < 4.9e-4, |sin tau| < 0.032), so their products
  // stay unnormalised pairs and are summed once.
  s_out = add(S, add(mul_nr(S, cm1), mul_nr(C, sn)));
  c_out = add(C, sub(mul_nr(C, cm1), mul_nr(S, sn)));
}

// sincos_ds for any angle: |theta| < SC_MAX_ARG by the reduction above, larger (rare: a search's
// trial lambda far out) or non-finite angles by FP64 sincos.
constexpr float SC_MAX_ARG = 12000.0f;
__device__ __forceinline__ void sincos_ds_any(ds th, const float4* tab, ds& s_out, ds& c_out) {
  if (fabsf(th.hi) < SC_MAX_ARG) {
    sincos_ds<float>(th, tab, s_out, c_out);
  } else {
    double s, c;
    sincos(to_double(th), &s, &c);
    s_out = from_double(s);
    c_out = from_double(c);
  }
}

}  // namespace ff
}  // namespace dbie
