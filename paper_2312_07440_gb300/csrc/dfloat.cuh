// Double-float ("df") arithmetic for the FP32 modes: a value is the unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// FP32 mode keeps the kinematic invariants that feed the propagators
// ((K - p)^2 - m^2 formed by cancellation) and the mass-shell reshuffle at far
// better than single precision.  GB300 issues FP64 at 1/64 of the FP32 rate,
// so doing that work in FP64 (and converting the FP64 momenta to float with
// F2F, itself an FP64-pipe instruction) made the FP64 pipe the bottleneck of
// the FP32 kernels.  Here the same quantities are formed from error-free
// transformations on the FP32 pipe and the FP64 -> df split uses integer
// operations only.
//
// Building blocks (all with explicit _rn intrinsics, so the compiler neither
// contracts nor reassociates them):
//   TwoSum (Knuth): s + e == a + b exactly;
//   Fast2Sum (Dekker): the same for |a| >= |b|;
//   TwoProd via FMA: p + e == a * b exactly.
// df + df is the accurate pairwise sum (both parts added by TwoSum, two
// renormalisations); df * df the FMA-based product; the relative error of
// both is a small multiple of u^2 = 2^-48 (Joldes, Muller and Popescu,
// ACM TOMS 44 (2017), "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic").  The square root is one Newton
// correction of the float root, also accurate to a few u^2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rw {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ df df_add(df x, df y) {
  df s = df_two_sum(x.hi, y.hi);
  const df t = df_two_sum(x.lo, y.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_add_f(df x, float y) {
  df s = df_two_sum(x.hi, y);
  s.lo = __fadd_rn(s.lo, x.lo);
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_mul(df x, df y) {
  const df c = df_two_prod(x.hi, y.hi);
  const float t = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
  return df_fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}

__device__ __forceinline__ df df_mul_f(df x, float y) {
  const df c = df_two_prod(x.hi, y);
  return df_fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}

// multiplication by a power of two is exact
__device__ __forceinline__ df df_scale(df x, float pow2) { return {__fmul_rn(x.hi, pow2), __fmul_rn(x.lo, pow2)}; }

// x >= 0; one Newton correction of the correctly rounded float root:
// r = s + (x - s^2) / (2 s), with x - s^2 formed exactly by FMA.
__device__ __forceinline__ df df_sqrt(df x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  const float s = __fsqrt_rn(x.hi);
  const float e = __fadd_rn(__fmaf_rn(-s, s, x.hi), x.lo);
  return df_fast_two_sum(s, __fmul_rn(e, __fdiv_rn(0.5f, s)));
}

// Minkowski product sum_mu g_mu a^mu b^mu: products exact (TwoProd), their
// high parts summed by TwoSum, every low-order term accumulated in float; the
// error is a few u^2 times sum |a^mu b^mu|, so a cancelling product keeps ~48
// bits relative to its terms.
__device__ __forceinline__ df df_dot4(const df (&a)[4], const df (&b)[4]) {
  df s = df_two_prod(a[0].hi, b[0].hi);
  float lo = __fadd_rn(s.lo, __fmaf_rn(a[0].hi, b[0].lo, __fmul_rn(a[0].lo, b[0].hi)));
  s.lo = 0.0f;
#pragma unroll
  for (int m = 1; m < 4; ++m) {
    const df p = df_two_prod(a[m].hi, b[m].hi);
    const float t = __fadd_rn(p.lo, __fmaf_rn(a[m].hi, b[m].lo, __fmul_rn(a[m].lo, b[m].hi)));
    const df u = df_two_sum(s.hi, -p.hi);
    s.hi = u.hi;
    lo = __fadd_rn(lo, __fsub_rn(u.lo, t));
  }
  return df_fast_two_sum(s.hi, lo);
}

// |p|^2 of the spatial part, same scheme as df_dot4 (no cancellation)
__device__ __forceinline__ df df_norm3(const df (&a)[4]) {
  df s = df_two_prod(a[1].hi, a[1].hi);
  float lo = __fadd_rn(s.lo, __fmul_rn(2.0f, __fmul_rn(a[1].hi, a[1].lo)));
#pragma unroll
  for (int m = 2; m < 4; ++m) {
    const df p = df_two_prod(a[m].hi, a[m].hi);
    const float t = __fadd_rn(p.lo, __fmul_rn(2.0f, __fmul_rn(a[m].hi, a[m].lo)));
    const df u = df_two_sum(s.hi, p.hi);
    s.hi = u.hi;
    lo = __fadd_rn(lo, __fadd_rn(u.lo, t));
  }
  return df_fast_two_sum(s.hi, lo);
}

// Split a double into hi = the float nearest to x (ties to even, the result
// of the IEEE binary64 -> binary32 conversion) and lo = x - hi rounded to
// float, with integer operations on the IEEE 754 fields only:
//   x = (-1)^s 1.m 2^(e-1023), m = 52 bits;  hi keeps the top 23 bits of m,
//   rounded up when the 29 dropped bits are above half (or exactly half and
//   the kept part is odd; the carry may run into the exponent, which is the
//   correct rounding); lo = (-1)^s n 2^(e-1075), n = the dropped bits minus
//   2^29 if hi was rounded up (|n| <= 2^28), converted to float with a
//   single rounding.
// Zero and values below the float normal range (|x| < 2^-126) give hi = lo =
// +-0, values beyond it +-inf, NaN stays NaN; lo is 0 for |x| < 2^-74.
__device__ __forceinline__ df df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = unsigned(b >> 32), lw = unsigned(b);
  const unsigned sgn = hw & 0x80000000u;
  const int e = int((hw >> 20) & 0x7FFu);
  const unsigned m23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const unsigned rem = lw & 0x1FFFFFFFu;
  const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
  const int ef = e - 896;
  if (ef <= 0 || ef >= 255) {
    float h;
    if (e == 0x7FF)
      h = __uint_as_float(sgn | 0x7F800000u | (((hw & 0xFFFFFu) | lw) ? 0x400000u : 0u));
    else
      h = __uint_as_float(ef <= 0 ? sgn : (sgn | 0x7F800000u));
    return {h, 0.0f};
  }
  const float hi = __uint_as_float((sgn | (unsigned(ef) << 23) | m23) + up);
  float lo = 0.0f;
  if (e >= 949) {
    const int n = int(rem) - int(up << 29);
    const int nh = n >> 14;          // |nh| <= 2^14
    const int nl = n & 0x3FFF;       // 0 <= nl < 2^14
    const float fh = __fsub_rn(__int_as_float(0x4B400000 + nh), 12582912.0f);  // exact
    const float fl = __fsub_rn(__int_as_float(0x4B000000 | nl), 8388608.0f);    // exact
    const float v = __fmaf_rn(fh, 16384.0f, fl);                                 // RN(n)
    lo = __fmul_rn(v, __int_as_float((e - 948) << 23));                          // exact
    if (sgn) lo = -lo;
  }
  return {hi, lo};
}

}  // namespace rw
