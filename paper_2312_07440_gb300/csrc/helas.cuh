// Device building blocks of the helicity amplitudes (HELAS-style, written for
// sm_103a): complex arithmetic, external wavefunctions, colour-ordered
// vertices and propagators.  Templated on the working precision R (double in
// FP64 mode, float in FP32 mode).
//
// Conventions: metric (+,-,-,-); Dirac matrices in the chiral basis
// gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]], spinors stored as
// (L0, L1, R0, R1); all gluon momenta in the vertices are incoming.
// The amplitudes are the colour-ordered partial amplitudes A(sigma) of the
// decomposition M_ij = sum_sigma (t^{a_sigma1} ... t^{a_sigman})_ij A(sigma)
// (t^a = lambda^a / 2) with the strong coupling stripped (g = 1).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace rw {

template <class R>
struct cx {
  R r, i;
};
template <class R>
struct cv {  // complex Lorentz vector, upper index
  cx<R> c[4];
};
template <class R>
struct sp {  // Dirac spinor (or a row spinor ubar)
  cx<R> c[4];
};

template <class R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.r + b.r, a.i + b.i}; }
template <class R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.r - b.r, a.i - b.i}; }
template <class R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.r, -a.i}; }
template <class R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <class R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.r, s * a.i}; }
template <class R>
__device__ __forceinline__ cx<R> conjg(cx<R> a) { return {a.r, -a.i}; }
template <class R>
__device__ __forceinline__ cx<R> times_i(cx<R> a) { return {-a.i, a.r}; }

// ---------------------------------------------------------------------------
// Fused arithmetic.  Every product-sum below is written as a chain of fused
// multiply-adds into its accumulator (a*b + c with one rounding), so a
// complex product costs 2 MUL + 2 FMA and each further product accumulated
// into a sum 4 FMA, with no separate additions.  On GB300's FP64 pipe every
// instruction counts; the flop counts quoted are those of the formulas
// (an FMA is 2 flops), unchanged by the fusion.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R fmadd(R a, R b, R c);
template <>
__device__ __forceinline__ double fmadd<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <>
__device__ __forceinline__ float fmadd<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// a*b
template <class R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return {fmadd(a.r, b.r, -(a.i * b.i)), fmadd(a.r, b.i, a.i * b.r)};
}
// acc + a*b
template <class R>
__device__ __forceinline__ cx<R> cmac(cx<R> a, cx<R> b, cx<R> acc) {
  return {fmadd(a.r, b.r, fmadd(-a.i, b.i, acc.r)), fmadd(a.r, b.i, fmadd(a.i, b.r, acc.i))};
}
// acc - a*b
template <class R>
__device__ __forceinline__ cx<R> cmsc(cx<R> a, cx<R> b, cx<R> acc) {
  return {fmadd(-a.r, b.r, fmadd(a.i, b.i, acc.r)), fmadd(-a.r, b.i, fmadd(-a.i, b.r, acc.i))};
}
// acc + s*a, s real
template <class R>
__device__ __forceinline__ cx<R> rmac(R s, cx<R> a, cx<R> acc) {
  return {fmadd(s, a.r, acc.r), fmadd(s, a.i, acc.i)};
}

// a.b (Minkowski, no conjugation): 30 flops
template <class R>
__device__ __forceinline__ cx<R> dot(const cv<R>& a, const cv<R>& b) {
  cx<R> s = cmul(a.c[0], b.c[0]);
  s = cmsc(a.c[1], b.c[1], s);
  s = cmsc(a.c[2], b.c[2], s);
  return cmsc(a.c[3], b.c[3], s);
}
// p.a with a real vector p: 14 flops
template <class R>
__device__ __forceinline__ cx<R> dotr(const R (&p)[4], const cv<R>& a) {
  cx<R> s = {p[0] * a.c[0].r, p[0] * a.c[0].i};
  s = rmac(-p[1], a.c[1], s);
  s = rmac(-p[2], a.c[2], s);
  return rmac(-p[3], a.c[3], s);
}
template <class R>
__device__ __forceinline__ cv<R> neg(const cv<R>& a) {
  return {{-a.c[0], -a.c[1], -a.c[2], -a.c[3]}};
}
template <class R>
__device__ __forceinline__ void addto(cv<R>& a, const cv<R>& b) {
#pragma unroll
  for (int m = 0; m < 4; ++m) a.c[m] = a.c[m] + b.c[m];
}
template <class R>
__device__ __forceinline__ void spadd(sp<R>& a, const sp<R>& b) {
#pragma unroll
  for (int m = 0; m < 4; ++m) a.c[m] = a.c[m] + b.c[m];
}
template <class R>
__device__ __forceinline__ sp<R> spneg(const sp<R>& a) {
  sp<R> o;
#pragma unroll
  for (int m = 0; m < 4; ++m) o.c[m] = -a.c[m];
  return o;
}
template <class R>
__device__ __forceinline__ void spsub(sp<R>& a, const sp<R>& b) {
#pragma unroll
  for (int m = 0; m < 4; ++m) a.c[m] = a.c[m] - b.c[m];
}

// four reals passed by value (out-of-line calls)
template <class R>
struct v4 {
  R m[4];
};

// Colour-ordered 3-gluon vertex and the off-shell gluon propagator,
// c = -1/K^2 (Feynman gauge, g stripped), K = P1 + P2:
//   out = c [ -J1 (2P1+P2).J2 + (J1.J2)(P1-P2) + J2 (2P2+P1).J1 ]     (156 flops)
// vvv returns it, vvv_acc adds it to o (+8 flops).
template <class R, bool ACC>
__device__ __forceinline__ void vvv_body(cv<R>& o, const cv<R>& J1, const R (&P1)[4], const cv<R>& J2,
                                         const R (&P2)[4], R c) {
  R a[4], b[4], d[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    a[m] = fmadd(R(2), P1[m], P2[m]);
    b[m] = fmadd(R(2), P2[m], P1[m]);
    d[m] = P1[m] - P2[m];
  }
  const cx<R> s1 = c * dotr(a, J2);
  const cx<R> s2 = c * dotr(b, J1);
  const cx<R> s12 = c * dot(J1, J2);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    cx<R> t = ACC ? rmac(d[m], s12, o.c[m]) : cx<R>{d[m] * s12.r, d[m] * s12.i};
    t = cmac(J2.c[m], s2, t);
    o.c[m] = cmsc(J1.c[m], s1, t);
  }
}
#ifdef RW_FP32_OUTLINED_CURRENTS
constexpr bool kOutlinedCur32 = true;
#else
constexpr bool kOutlinedCur32 = false;
#endif
#ifdef RW_FP64_OUTLINED_CURRENTS
constexpr bool kOutlinedCur64 = true;
#else
constexpr bool kOutlinedCur64 = false;
#endif
#if defined(RW_FP32_OUTLINED_CURRENTS) || defined(RW_FP64_OUTLINED_CURRENTS)
template <class R, bool ACC>
__device__ __noinline__ cv<R> vvv_call(cv<R> o, cv<R> J1, v4<R> P1, cv<R> J2, v4<R> P2, R c) {
  vvv_body<R, ACC>(o, J1, P1.m, J2, P2.m, c);
  return o;
}
#endif
template <class R, bool ACC>
__device__ __forceinline__ void vvv_impl(cv<R>& o, const cv<R>& J1, const R (&P1)[4], const cv<R>& J2,
                                         const R (&P2)[4], R c) {
#if defined(RW_FP32_OUTLINED_CURRENTS) || defined(RW_FP64_OUTLINED_CURRENTS)
  if constexpr (sizeof(R) == 4 ? kOutlinedCur32 : kOutlinedCur64) {
    o = vvv_call<R, ACC>(o, J1, v4<R>{{P1[0], P1[1], P1[2], P1[3]}}, J2, v4<R>{{P2[0], P2[1], P2[2], P2[3]}}, c);
    return;
  }
#endif
  vvv_body<R, ACC>(o, J1, P1, J2, P2, c);
}
template <class R>
__device__ __forceinline__ cv<R> vvv(const cv<R>& J1, const R (&P1)[4], const cv<R>& J2, const R (&P2)[4], R c) {
  cv<R> o;
  vvv_impl<R, false>(o, J1, P1, J2, P2, c);
  return o;
}
template <class R>
__device__ __forceinline__ void vvv_acc(cv<R>& o, const cv<R>& J1, const R (&P1)[4], const cv<R>& J2,
                                        const R (&P2)[4], R c) {
  vvv_impl<R, true>(o, J1, P1, J2, P2, c);
}

// Colour-ordered 4-gluon vertex with the propagator c = +1/K^2:
//   out += c [ 2 J2 (J1.J3) - J1 (J2.J3) - J3 (J1.J2) ]                 (193 flops)
template <class R>
__device__ __forceinline__ void vvvv_body(cv<R>& o, const cv<R>& J1, const cv<R>& J2, const cv<R>& J3, R c) {
  const cx<R> t13 = (R(2) * c) * dot(J1, J3);
  const cx<R> t23 = c * dot(J2, J3);
  const cx<R> t12 = c * dot(J1, J2);
#pragma unroll
  for (int m = 0; m < 4; ++m) o.c[m] = cmsc(J3.c[m], t12, cmsc(J1.c[m], t23, cmac(J2.c[m], t13, o.c[m])));
}
#if defined(RW_FP32_OUTLINED_CURRENTS) || defined(RW_FP64_OUTLINED_CURRENTS)
template <class R>
__device__ __noinline__ cv<R> vvvv_call(cv<R> o, cv<R> J1, cv<R> J2, cv<R> J3, R c) {
  vvvv_body<R>(o, J1, J2, J3, c);
  return o;
}
#endif
template <class R>
__device__ __forceinline__ void vvvv_acc(cv<R>& o, const cv<R>& J1, const cv<R>& J2, const cv<R>& J3, R c) {
#if defined(RW_FP32_OUTLINED_CURRENTS) || defined(RW_FP64_OUTLINED_CURRENTS)
  if constexpr (sizeof(R) == 4 ? kOutlinedCur32 : kOutlinedCur64) {
    o = vvvv_call<R>(o, J1, J2, J3, c);
    return;
  }
#endif
  vvvv_body<R>(o, J1, J2, J3, c);
}

// A complex vector in Weyl-block form: a0 - a3, a0 + a3, a1 + i a2, a1 - i a2
// (the entries of the 2x2 blocks of a-slash in the chiral basis)   (8 flops)
template <class R>
struct ws {
  cx<R> am, ap, bp, bm;
};
template <class R>
__device__ __forceinline__ ws<R> weyl_form(const cv<R>& a) {
  return {a.c[0] - a.c[3], a.c[0] + a.c[3], {a.c[1].r - a.c[2].i, a.c[1].i + a.c[2].r},
          {a.c[1].r + a.c[2].i, a.c[1].i - a.c[2].r}};
}

// Jslash psi = gamma^mu J_mu psi: 56 flops from the Weyl-block form, 64 from
// the vector.  slash returns it, slash_acc adds it to o (+8 flops).
template <class R, bool ACC>
__device__ __forceinline__ void slash_body(sp<R>& o, const ws<R>& a, const sp<R>& s) {
  o.c[0] = cmsc(a.bm, s.c[3], ACC ? cmac(a.am, s.c[2], o.c[0]) : cmul(a.am, s.c[2]));
  o.c[1] = cmsc(a.bp, s.c[2], ACC ? cmac(a.ap, s.c[3], o.c[1]) : cmul(a.ap, s.c[3]));
  o.c[2] = cmac(a.bm, s.c[1], ACC ? cmac(a.ap, s.c[0], o.c[2]) : cmul(a.ap, s.c[0]));
  o.c[3] = cmac(a.am, s.c[1], ACC ? cmac(a.bp, s.c[0], o.c[3]) : cmul(a.bp, s.c[0]));
}
// Out-of-line copies of the slash and the gluon vertices, for amplitude code
// whose unrolled chains would not fit the instruction cache: a translation
// unit defines RW_FP32_OUTLINED_SLASH / RW_FP32_OUTLINED_CURRENTS (FP32) or
// RW_FP64_OUTLINED_SLASH / RW_FP64_OUTLINED_CURRENTS (FP64) before including.
#if defined(RW_FP32_OUTLINED_SLASH) || defined(RW_FP64_OUTLINED_SLASH)
template <class R, bool ACC>
__device__ __noinline__ sp<R> slash_call(sp<R> o, ws<R> a, sp<R> s) {
  slash_body<R, ACC>(o, a, s);
  return o;
}
#endif
#ifdef RW_FP32_OUTLINED_SLASH
constexpr bool kOutlinedSlash32 = true;
#else
constexpr bool kOutlinedSlash32 = false;
#endif
#ifdef RW_FP64_OUTLINED_SLASH
constexpr bool kOutlinedSlash64 = true;
#else
constexpr bool kOutlinedSlash64 = false;
#endif
template <class R, bool ACC>
__device__ __forceinline__ void slash_impl(sp<R>& o, const ws<R>& a, const sp<R>& s) {
#if defined(RW_FP32_OUTLINED_SLASH) || defined(RW_FP64_OUTLINED_SLASH)
  if constexpr (sizeof(R) == 4 ? kOutlinedSlash32 : kOutlinedSlash64) {
    o = slash_call<R, ACC>(o, a, s);
    return;
  }
#endif
  slash_body<R, ACC>(o, a, s);
}
template <class R>
__device__ __forceinline__ sp<R> slash(const ws<R>& a, const sp<R>& s) {
  sp<R> o;
  slash_impl<R, false>(o, a, s);
  return o;
}
template <class R>
__device__ __forceinline__ sp<R> slash(const cv<R>& a, const sp<R>& s) {
  return slash(weyl_form(a), s);
}
template <class R>
__device__ __forceinline__ void slash_acc(sp<R>& o, const ws<R>& a, const sp<R>& s) {
  slash_impl<R, true>(o, a, s);
}
template <class R>
__device__ __forceinline__ void slash_acc(sp<R>& o, const cv<R>& a, const sp<R>& s) {
  slash_impl<R, true>(o, weyl_form(a), s);
}

// Top propagator applied to a spinor, with the factor folded in:
//   (qc slash + mc) chi,  qc = c q, mc = c m,  c = -1/(q^2 - m^2)         (58 flops)
// Each real component is one chain: am s2 - (q1 - i q2) s3 + mc s0, etc.
template <class R>
__device__ __forceinline__ sp<R> fprop(const R (&q)[4], R mc, const sp<R>& s) {
  const R ap = q[0] + q[3], am = q[0] - q[3], q1 = q[1], q2 = q[2];
  sp<R> o;
  o.c[0] = {fmadd(mc, s.c[0].r, fmadd(-q2, s.c[3].i, fmadd(-q1, s.c[3].r, am * s.c[2].r))),
            fmadd(mc, s.c[0].i, fmadd(q2, s.c[3].r, fmadd(-q1, s.c[3].i, am * s.c[2].i)))};
  o.c[1] = {fmadd(mc, s.c[1].r, fmadd(q2, s.c[2].i, fmadd(-q1, s.c[2].r, ap * s.c[3].r))),
            fmadd(mc, s.c[1].i, fmadd(-q2, s.c[2].r, fmadd(-q1, s.c[2].i, ap * s.c[3].i)))};
  o.c[2] = {fmadd(mc, s.c[2].r, fmadd(q2, s.c[1].i, fmadd(q1, s.c[1].r, ap * s.c[0].r))),
            fmadd(mc, s.c[2].i, fmadd(-q2, s.c[1].r, fmadd(q1, s.c[1].i, ap * s.c[0].i)))};
  o.c[3] = {fmadd(mc, s.c[3].r, fmadd(-q2, s.c[0].i, fmadd(q1, s.c[0].r, am * s.c[1].r))),
            fmadd(mc, s.c[3].i, fmadd(q2, s.c[0].r, fmadd(q1, s.c[0].i, am * s.c[1].i)))};
  return o;
}

// Fermion current ubar gamma^mu psi (upper index), ubar a row spinor       (72 flops)
template <class R>
__device__ __forceinline__ cv<R> fcur(const sp<R>& u, const sp<R>& s) {
  // ubar_L sigma^mu psi_R + ubar_R sigmabar^mu psi_L
  const cx<R> a = u.c[0] * s.c[2], b = u.c[1] * s.c[3], c = u.c[0] * s.c[3], d = u.c[1] * s.c[2];
  const cx<R> a2 = u.c[2] * s.c[0], b2 = u.c[3] * s.c[1], c2 = u.c[2] * s.c[1], d2 = u.c[3] * s.c[0];
  cv<R> o;
  o.c[0] = (a + b) + (a2 + b2);
  o.c[1] = (c + d) - (c2 + d2);
  o.c[2] = times_i((d - c) - (d2 - c2));
  o.c[3] = (a - b) - (a2 - b2);
  return o;
}

// ubar . X: a row spinor times a column spinor                           (30 flops)
template <class R>
__device__ __forceinline__ cx<R> rowcol(const sp<R>& u, const sp<R>& x) {
  return cmac(u.c[3], x.c[3], cmac(u.c[2], x.c[2], cmac(u.c[1], x.c[1], cmul(u.c[0], x.c[0]))));
}

// ---------------------------------------------------------------------------
// External wavefunctions, computed in the working precision T from momenta
// already converted to T, with formulas free of cancellation: |p| + p_z is
// formed as p_T^2/(|p| - p_z) when p_z < 0, and sqrt(E - |p|) as m/sqrt(E + |p|).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }

// Helicity eigen-2-spinors chi_{+-}(p) along pvec (phi = 0 when p_T = 0)
// and |p|.
template <class T>
__device__ __forceinline__ T chi_pm(const T (&p)[4], cx<T> (&cp)[2], cx<T> (&cm)[2]) {
  const T pt2 = p[1] * p[1] + p[2] * p[2];
  const T pp = sqrt(pt2 + p[3] * p[3]);
  const T ppz = p[3] >= T(0) ? pp + p[3] : pt2 / (pp - p[3]);  // |p| + p_z
  if (ppz > T(0) && pp > T(0)) {
    const T s = rsqrt_t<T>(T(2) * pp * ppz);  // 1/sqrt(2|p|(|p|+p_z))
    const T c = ppz * s;                      // cos(theta/2)
    cp[0] = {c, T(0)};
    cp[1] = {p[1] * s, p[2] * s};
    cm[0] = {-p[1] * s, p[2] * s};
    cm[1] = {c, T(0)};
  } else {  // along -z (or p = 0)
    cp[0] = {T(0), T(0)};
    cp[1] = {T(1), T(0)};
    cm[0] = {T(-1), T(0)};
    cm[1] = {T(0), T(0)};
  }
  return pp;
}

// w+ = sqrt(E + |p|), w- = sqrt(E - |p|) = m / w+
template <class T>
__device__ __forceinline__ void omegas(T E, T pp, T m, T& wp, T& wm) {
  const T a = E + pp;
  const T r = rsqrt_t<T>(a);
  wp = a * r;
  wm = m * r;
}

// ubar(p, lambda) for an outgoing fermion (row spinor), index 0: lambda=+1/2, 1: -1/2.
// u(p,+) = (w- chi+, w+ chi+), u(p,-) = (w+ chi-, w- chi-); ubar = (u_R^*, u_L^*).
template <class T>
__device__ __forceinline__ void ubar_out(const T (&p)[4], T m, sp<T> (&ub)[2]) {
  cx<T> cp[2], cm[2];
  const T pp = chi_pm(p, cp, cm);
  T wp, wm;
  omegas(p[0], pp, m, wp, wm);
  ub[0].c[0] = conjg(wp * cp[0]);
  ub[0].c[1] = conjg(wp * cp[1]);
  ub[0].c[2] = conjg(wm * cp[0]);
  ub[0].c[3] = conjg(wm * cp[1]);
  ub[1].c[0] = conjg(wm * cm[0]);
  ub[1].c[1] = conjg(wm * cm[1]);
  ub[1].c[2] = conjg(wp * cm[0]);
  ub[1].c[3] = conjg(wp * cm[1]);
}

// v(p, lambda) for an outgoing antifermion: v(p,+) = (w+ chi-, -w- chi-),
// v(p,-) = (w- chi+, -w+ chi+).
template <class T>
__device__ __forceinline__ void v_out(const T (&p)[4], T m, sp<T> (&v)[2]) {
  cx<T> cp[2], cm[2];
  const T pp = chi_pm(p, cp, cm);
  T wp, wm;
  omegas(p[0], pp, m, wp, wm);
  v[0].c[0] = wp * cm[0];
  v[0].c[1] = wp * cm[1];
  v[0].c[2] = (-wm) * cm[0];
  v[0].c[3] = (-wm) * cm[1];
  v[1].c[0] = wm * cp[0];
  v[1].c[1] = wm * cp[1];
  v[1].c[2] = (-wp) * cp[0];
  v[1].c[3] = (-wp) * cp[1];
}

// u(p, lambda) for an incoming fermion
template <class T>
__device__ __forceinline__ void u_in(const T (&p)[4], T m, sp<T> (&u)[2]) {
  cx<T> cp[2], cm[2];
  const T pp = chi_pm(p, cp, cm);
  T wp, wm;
  omegas(p[0], pp, m, wp, wm);
  u[0].c[0] = wm * cp[0];
  u[0].c[1] = wm * cp[1];
  u[0].c[2] = wp * cp[0];
  u[0].c[3] = wp * cp[1];
  u[1].c[0] = wp * cm[0];
  u[1].c[1] = wp * cm[1];
  u[1].c[2] = wm * cm[0];
  u[1].c[3] = wm * cm[1];
}

// vbar(p, lambda) = v^dagger gamma^0 for an incoming antifermion (row spinor)
template <class T>
__device__ __forceinline__ void vbar_in(const T (&p)[4], T m, sp<T> (&vb)[2]) {
  sp<T> v[2];
  v_out<T>(p, m, v);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    vb[h].c[0] = conjg(v[h].c[2]);
    vb[h].c[1] = conjg(v[h].c[3]);
    vb[h].c[2] = conjg(v[h].c[0]);
    vb[h].c[3] = conjg(v[h].c[1]);
  }
}

// Transverse polarisation eps(k, lambda) = (-lambda e1 - i e2)/sqrt(2),
// e1 = (0, cos t cos f, cos t sin f, -sin t), e2 = (0, -sin f, cos f, 0);
// index 0: lambda = +1, 1: lambda = -1; conjugated for an outgoing gluon.
template <class T>
__device__ __forceinline__ void polvec(const T (&k)[4], bool outgoing, cv<T> (&e)[2]) {
  const T pt2 = k[1] * k[1] + k[2] * k[2];
  const T ikk = rsqrt_t<T>(pt2 + k[3] * k[3]);
  T cf = T(1), sf = T(0), st = T(0);
  if (pt2 > T(0)) {
    const T ipt = rsqrt_t<T>(pt2);
    cf = k[1] * ipt;
    sf = k[2] * ipt;
    st = pt2 * ipt * ikk;
  }
  const T ct = k[3] * ikk;
  const T r2 = T(0.70710678118654752440);
  const T e1[4] = {T(0), ct * cf, ct * sf, -st};
  const T e2[4] = {T(0), -sf, cf, T(0)};
  const T sgn = outgoing ? T(-1) : T(1);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    e[0].c[m] = {-r2 * e1[m], -sgn * r2 * e2[m]};
    e[1].c[m] = {r2 * e1[m], -sgn * r2 * e2[m]};
  }
}

}  // namespace rw
