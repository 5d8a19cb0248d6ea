// Per-event set-up for g g -> t tbar + n g: external wavefunctions of both
// helicities (in the working precision R, cancellation-free formulas) and the
// propagator invariants, whose dot products are formed at ~double precision
// -- FP64 in FP64 mode, double-float (dfloat.cuh) in the FP32 modes -- so
// that FP32 mode never forms p^2 - m^2 by cancellation in single precision,
// before the reciprocals are taken in R.
#pragma once
#include "dfloat.cuh"
#include "helas.cuh"

namespace rw {

template <class R, int NG>
struct QcdExt {
  cv<R> eps[NG][2];  // gluon polarisations (conjugated for outgoing gluons)
  sp<R> ub[2];       // top: ubar(p3, lambda)
  sp<R> v[2];        // antitop: v(p4, lambda)
};

template <class R, int NG>
struct QcdKin {
  R P[1 << NG][4];   // summed incoming momentum of each gluon subset
  R cg[1 << NG];     // -1/K^2  (3-gluon vertex + gluon propagator)
  R c4[1 << NG];     // +1/K^2  (4-gluon vertex + gluon propagator)
  R qc[1 << NG][4];  // c (K - p4), c = -1/((K - p4)^2 - m^2)  (top propagator)
  R mc[1 << NG];     // c m
};

// Store for the gluon currents of three or more gluons (generated code puts
// each once and gets it at every use).  Registers: a plain array indexed by
// constants.  Shared memory (FP32): this thread's slice of the dynamic shared
// memory, [slot][half][thread] float4 so a warp's accesses are conflict-free;
// the accesses are volatile, so the compiler neither keeps a stored current
// in registers nor moves a read above the write of its slot.  The kernel
// places its own shared data after NS * 32 * blockDim.x bytes.
template <class R, int NS, bool SMEM>
struct JStore {
  cv<R> v[NS > 0 ? NS : 1];
  __device__ __forceinline__ void put(int s, const cv<R>& x) { v[s] = x; }
  __device__ __forceinline__ cv<R> get(int s) const { return v[s]; }
};

template <int NS>
struct JStore<float, NS, true> {
  unsigned base, stride;
  __device__ __forceinline__ JStore() {
    extern __shared__ float4 rw_dyn_smem[];
    base = (unsigned)__cvta_generic_to_shared(rw_dyn_smem + threadIdx.x);
    stride = 16u * blockDim.x;
  }
  __device__ __forceinline__ void put(int s, const cv<float>& x) const {
    const unsigned a = base + 2u * (unsigned)s * stride;
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x.c[0].r), "f"(x.c[0].i), "f"(x.c[1].r),
                 "f"(x.c[1].i));
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a + stride), "f"(x.c[2].r), "f"(x.c[2].i),
                 "f"(x.c[3].r), "f"(x.c[3].i));
  }
  __device__ __forceinline__ cv<float> get(int s) const {
    const unsigned a = base + 2u * (unsigned)s * stride;
    cv<float> x;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(x.c[0].r), "=f"(x.c[0].i), "=f"(x.c[1].r), "=f"(x.c[1].i)
                 : "r"(a));
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(x.c[2].r), "=f"(x.c[2].i), "=f"(x.c[3].r), "=f"(x.c[3].i)
                 : "r"(a + stride));
    return x;
  }
};

// particle index of gluon g on the top line: 0, 1 incoming, then 4, 5, ...
__host__ __device__ constexpr int gluon_particle(int g) { return g < 2 ? g : g + 2; }

__device__ __forceinline__ double dot4(const double (&a)[4], const double (&b)[4]) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

// Double-double arithmetic for the FP64 set-up's invariants of several
// gluons: Knuth's TwoSum, the FMA form of TwoProduct, one rounding at the end.
// A gluon propagator 1/K^2 of an incoming and an outgoing gluon near the beam
// axis has K^2 ~ 1e2-1e3 GeV^2 while k_i.k_j-style products are ~1e6 GeV^2,
// so K^2 formed in plain FP64 carries relative errors of ~1e-13, which the
// largest-|M|^2 events (near-collinear emission) pass on to |M|^2.
struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(double a, double b) {
  const double s = a + b;
  const double bp = s - a;
  return {s, (a - (s - bp)) + (b - bp)};
}

__device__ __forceinline__ dd dd_add(dd x, double y) {
  const dd s = dd_two_sum(x.hi, y);
  const double lo = s.lo + x.lo;
  const double h = s.hi + lo;
  return {h, lo - (h - s.hi)};
}

__device__ __forceinline__ dd dd_add(dd x, dd y) {
  const dd s = dd_two_sum(x.hi, y.hi);
  const double lo = s.lo + (x.lo + y.lo);
  const double h = s.hi + lo;
  return {h, lo - (h - s.hi)};
}

// Minkowski product a.b carried to double-double: every product exact as
// p + e (FMA), the p added by TwoSum
__device__ __forceinline__ dd dd_dot4(const double (&a)[4], const double (&b)[4]) {
  dd acc = {0.0, 0.0};
  double small = 0.0;
#pragma unroll
  for (int m4 = 0; m4 < 4; ++m4) {
    const double x = m4 ? -a[m4] : a[m4];
    const double q = x * b[m4];
    small += fma(x, b[m4], -q);
    acc = dd_add(acc, q);
  }
  acc.lo += small;
  return acc;
}

// K^2 and (K - p4)^2 - m^2 of every gluon subset K = sum_{i in S} k_i from the
// momenta themselves (no mass-shell assumption), each rounded once from
// double-double: K^2 = sum_i k_i.k_i + 2 sum_{i<j} k_i.k_j and
// (K - p4)^2 - m^2 = K^2 - 2 sum_i k_i.p4 + (p4.p4 - m^2), with the pairwise
// products formed once.  Out of line: its temporaries stay out of the
// amplitude code's register allocation.
template <int NG>
__device__ __noinline__ void subset_invariants_dd(const double (&k)[NG][4], const double (&p4)[4], double m,
                                                  double (&K2)[1 << NG], double (&den)[1 << NG]) {
  dd kk[NG], kp[NG], d[NG][NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) {
    kk[i] = dd_dot4(k[i], k[i]);
    kp[i] = dd_dot4(k[i], p4);
#pragma unroll
    for (int j = i + 1; j < NG; ++j) d[i][j] = dd_dot4(k[i], k[j]);
  }
  dd pm = dd_dot4(p4, p4);
  const double m2 = m * m;
  pm = dd_add(pm, dd{-m2, -fma(m, m, -m2)});
  constexpr int FULL = (1 << NG) - 1;
#pragma unroll
  for (int msk = 1; msk <= FULL; ++msk) {
    dd s = {0.0, 0.0};
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      if (!((msk >> i) & 1)) continue;
      s = dd_add(s, kk[i]);
#pragma unroll
      for (int j = i + 1; j < NG; ++j)
        if ((msk >> j) & 1) s = dd_add(s, dd{2.0 * d[i][j].hi, 2.0 * d[i][j].lo});
    }
    K2[msk] = s.hi + s.lo;
    if (msk != FULL) {
#pragma unroll
      for (int i = 0; i < NG; ++i)
        if ((msk >> i) & 1) s = dd_add(s, dd{-2.0 * kp[i].hi, -2.0 * kp[i].lo});
      s = dd_add(s, pm);
      den[msk] = s.hi + s.lo;
    } else {
      den[msk] = 0.0;
    }
  }
}

template <class R, int NG, int NEXT>
__device__ __forceinline__ void qcd_setup(const double (&p)[NEXT][4], double m, QcdExt<R, NG>& X,
                                          QcdKin<R, NG>& Kn) {
  static_assert(NEXT == NG + 2, "t tbar + NG gluons");
  double k[NG][4];
  R kw[NG][4];  // incoming gluon momenta in the working precision
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const int ip = gluon_particle(g);
    const double s = ip < 2 ? 1.0 : -1.0;
    R kr[4];
#pragma unroll
    for (int m4 = 0; m4 < 4; ++m4) {
      k[g][m4] = s * p[ip][m4];
      kr[m4] = R(p[ip][m4]);
      kw[g][m4] = ip < 2 ? kr[m4] : -kr[m4];
    }
    polvec<R>(kr, ip >= 2, X.eps[g]);
  }
  {
    R p3[4], p4[4];
#pragma unroll
    for (int m4 = 0; m4 < 4; ++m4) {
      p3[m4] = R(p[2][m4]);
      p4[m4] = R(p[3][m4]);
    }
    ubar_out<R>(p3, R(m), X.ub);
    v_out<R>(p4, R(m), X.v);
  }
  // Invariants: the dot products, where cancellation happens, in FP64 (two
  // or three gluons: double-double, see subset_invariants_dd); the
  // reciprocals in the working precision.
  [[maybe_unused]] double K2dd[1 << NG], dendd[1 << NG];
  if constexpr (NG >= 3) subset_invariants_dd<NG>(k, p[3], m, K2dd, dendd);
  double d[NG][NG];
#pragma unroll
  for (int i = 0; i < NG; ++i)
#pragma unroll
    for (int j = i + 1; j < NG; ++j) d[i][j] = dot4(k[i], k[j]);  // gluons are massless: k_i^2 = 0
  constexpr int FULL = (1 << NG) - 1;
#pragma unroll
  for (int msk = 1; msk <= FULL; ++msk) {
    double P[4] = {0.0, 0.0, 0.0, 0.0};
    double K2 = 0.0;
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      if (!((msk >> i) & 1)) continue;
      ++cnt;
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) P[m4] += k[i][m4];
#pragma unroll
      for (int j = i + 1; j < NG; ++j)
        if ((msk >> j) & 1) K2 += 2.0 * d[i][j];
    }
    // vertex momenta: subset sums in the working precision
#pragma unroll
    for (int m4 = 0; m4 < 4; ++m4) {
      R v = R(0);
#pragma unroll
      for (int i = 0; i < NG; ++i)
        if ((msk >> i) & 1) v += kw[i][m4];
      Kn.P[msk][m4] = v;
    }
    if constexpr (NG >= 3) K2 = K2dd[msk];
    if (cnt >= 2) {
      const R inv = R(1) / R(K2);
      Kn.cg[msk] = -inv;
      Kn.c4[msk] = inv;
    } else {
      Kn.cg[msk] = R(0);
      Kn.c4[msk] = R(0);
    }
    if (msk != FULL) {
      // (K - p4)^2 - m^2 = K^2 - 2 K.p4  (p4^2 = m^2); several gluons: as above
      double den;
      if constexpr (NG >= 3)
        den = dendd[msk];
      else
        den = K2 - 2.0 * dot4(P, p[3]);
      const R c = R(-1) / R(den);
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) Kn.qc[msk][m4] = c * R(P[m4] - p[3][m4]);
      Kn.mc[msk] = c * R(m);
    } else {
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) Kn.qc[msk][m4] = R(0);
      Kn.mc[msk] = R(0);
    }
  }
}

// Move the outgoing particles (2..NEXT-1) onto the mass shells m_t (tops),
// 0 (gluons) at fixed partonic energy: p_i -> xi p_i (3-momenta) with
// sum_i sqrt(m_i^2 + xi^2 |p_i|^2) = sum_i E_i.  Newton's method from xi = 1
// in FP32 to ~1e-7, then NREF Newton steps in FP64 (quadratic convergence:
// one step leaves ~1e-14, two reach double precision).
// Returns false when the new masses do not fit (sum m_i >= E).
template <int NEXT, int NREF>
__device__ __forceinline__ bool reshuffle_tops(const double (&p)[NEXT][4], double mt, double (&q)[NEXT][4]) {
  double etot = 0.0, p2[NEXT];
#pragma unroll
  for (int i = 2; i < NEXT; ++i) {
    etot += p[i][0];
    p2[i] = p[i][1] * p[i][1] + p[i][2] * p[i][2] + p[i][3] * p[i][3];
  }
#pragma unroll
  for (int i = 0; i < NEXT; ++i)
#pragma unroll
    for (int m4 = 0; m4 < 4; ++m4) q[i][m4] = p[i][m4];
  if (!(2.0 * mt < etot)) return false;
  const double mt2 = mt * mt;
  const float etf = float(etot), mt2f = float(mt2);
  float xf = 1.0f;
  for (int it = 0; it < 40; ++it) {
    float f = -etf, df = 0.0f;
#pragma unroll
    for (int i = 2; i < NEXT; ++i) {
      const float pf = float(p2[i]);
      const float e = sqrtf((i < 4 ? mt2f : 0.0f) + xf * xf * pf);
      f += e;
      df += xf * pf / e;
    }
    float step = f / df;
    if (xf - step <= 0.0f) step = 0.5f * xf;
    xf -= step;
    if (fabsf(step) <= 2e-7f * xf) break;
  }
  double xi = xf, e[NEXT];
#pragma unroll
  for (int it = 0; it < NREF; ++it) {
    double f = -etot, df = 0.0;
#pragma unroll
    for (int i = 2; i < NEXT; ++i) {
      e[i] = sqrt((i < 4 ? mt2 : 0.0) + xi * xi * p2[i]);
      f += e[i];
      df += xi * p2[i] / e[i];
    }
    const double xn = xi - f / df;
    // energies at the new xi to first order: e' = e + (xn^2 - xi^2) |p|^2 / (2 e),
    // exact to O((xn - xi)^2) (the last step is ~1e-7 relative in FP32 refinement,
    // ~1e-14 after two FP64 steps)
    if (it == NREF - 1) {
#pragma unroll
      for (int i = 2; i < NEXT; ++i) e[i] += (xn - xi) * (xn + xi) * p2[i] / (2.0 * e[i]);
    }
    xi = xn;
  }
#pragma unroll
  for (int i = 2; i < NEXT; ++i) {
#pragma unroll
    for (int m4 = 1; m4 < 4; ++m4) q[i][m4] = xi * p[i][m4];
    q[i][0] = e[i];
  }
  return true;
}

// FP32 modes: the same set-up from double-float momenta (the split of the
// FP64 inputs); invariants in double-float, everything else in float.
template <class R, int NG, int NEXT>
__device__ __forceinline__ void qcd_setup(const df (&p)[NEXT][4], double m, QcdExt<R, NG>& X, QcdKin<R, NG>& Kn) {
  static_assert(NEXT == NG + 2, "t tbar + NG gluons");
  static_assert(sizeof(R) == 4, "double-float set-up feeds FP32 amplitudes");
  df k[NG][4];
  R kw[NG][4];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const int ip = gluon_particle(g);
    R kr[4];
#pragma unroll
    for (int m4 = 0; m4 < 4; ++m4) {
      k[g][m4] = ip < 2 ? p[ip][m4] : df_neg(p[ip][m4]);
      kr[m4] = p[ip][m4].hi;
      kw[g][m4] = ip < 2 ? kr[m4] : -kr[m4];
    }
    polvec<R>(kr, ip >= 2, X.eps[g]);
  }
  {
    R p3[4], p4[4];
#pragma unroll
    for (int m4 = 0; m4 < 4; ++m4) {
      p3[m4] = p[2][m4].hi;
      p4[m4] = p[3][m4].hi;
    }
    ubar_out<R>(p3, R(m), X.ub);
    v_out<R>(p4, R(m), X.v);
  }
  df d[NG][NG];
#pragma unroll
  for (int i = 0; i < NG; ++i)
#pragma unroll
    for (int j = i + 1; j < NG; ++j) d[i][j] = df_scale(df_dot4(k[i], k[j]), 2.0f);  // 2 k_i.k_j
  constexpr int FULL = (1 << NG) - 1;
#pragma unroll
  for (int msk = 1; msk <= FULL; ++msk) {
    df P[4];
    df K2 = {0.0f, 0.0f};
    bool first = true;
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      if (!((msk >> i) & 1)) continue;
      ++cnt;
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) P[m4] = first ? k[i][m4] : df_add(P[m4], k[i][m4]);
      first = false;
#pragma unroll
      for (int j = i + 1; j < NG; ++j)
        if ((msk >> j) & 1) K2 = df_add(K2, d[i][j]);
    }
#pragma unroll
    for (int m4 = 0; m4 < 4; ++m4) {
      R v = R(0);
#pragma unroll
      for (int i = 0; i < NG; ++i)
        if ((msk >> i) & 1) v += kw[i][m4];
      Kn.P[msk][m4] = v;
    }
    if (cnt >= 2) {
      const R inv = R(1) / K2.hi;
      Kn.cg[msk] = -inv;
      Kn.c4[msk] = inv;
    } else {
      Kn.cg[msk] = R(0);
      Kn.c4[msk] = R(0);
    }
    if (msk != FULL) {
      // (K - p4)^2 - m^2 = K^2 - 2 K.p4  (p4^2 = m^2)
      const df den = df_sub(K2, df_scale(df_dot4(P, p[3]), 2.0f));
      const R c = R(-1) / den.hi;
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) Kn.qc[msk][m4] = c * df_sub(P[m4], p[3][m4]).hi;
      Kn.mc[msk] = c * R(m);
    } else {
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) Kn.qc[msk][m4] = R(0);
      Kn.mc[msk] = R(0);
    }
  }
}

// FP32 modes: the reshuffle on double-float momenta.  The FP32 Newton
// iteration as above, then one Newton step in double-float (from ~1e-7 to
// the double-float precision), energies updated to first order as above, so
// that the moved momenta are on their mass shells to ~1e-14 relative.
template <int NEXT>
__device__ __forceinline__ bool reshuffle_tops(const df (&p)[NEXT][4], double mt, df (&q)[NEXT][4]) {
  df etot = {0.0f, 0.0f}, p2[NEXT];
#pragma unroll
  for (int i = 2; i < NEXT; ++i) {
    etot = i == 2 ? p[i][0] : df_add(etot, p[i][0]);
    p2[i] = df_norm3(p[i]);
  }
#pragma unroll
  for (int i = 0; i < NEXT; ++i)
#pragma unroll
    for (int m4 = 0; m4 < 4; ++m4) q[i][m4] = p[i][m4];
  const df mtd = df_from_double(mt);
  if (!(df_sub(etot, df_scale(mtd, 2.0f)).hi > 0.0f)) return false;
  const df mt2 = df_mul(mtd, mtd);
  const float etf = etot.hi, mt2f = mt2.hi;
  float xf = 1.0f;
  for (int it = 0; it < 40; ++it) {
    float f = -etf, dfx = 0.0f;
#pragma unroll
    for (int i = 2; i < NEXT; ++i) {
      const float pf = p2[i].hi;
      const float e = sqrtf((i < 4 ? mt2f : 0.0f) + xf * xf * pf);
      f += e;
      dfx += xf * pf / e;
    }
    float step = f / dfx;
    if (xf - step <= 0.0f) step = 0.5f * xf;
    xf -= step;
    if (fabsf(step) <= 2e-7f * xf) break;
  }
  const df xi2 = df_two_prod(xf, xf);
  df e[NEXT];
  df f = df_neg(etot);
  float dfx = 0.0f;
#pragma unroll
  for (int i = 2; i < NEXT; ++i) {
    const df a = df_mul(xi2, p2[i]);
    e[i] = df_sqrt(i < 4 ? df_add(mt2, a) : a);
    f = df_add(f, e[i]);
    dfx += xf * p2[i].hi / e[i].hi;
  }
  const float corr = -f.hi / dfx;
  const df xn = df_fast_two_sum(xf, corr);
#pragma unroll
  for (int i = 2; i < NEXT; ++i) {
    // e' = e + (xn^2 - xi^2) |p|^2 / (2 e), exact to O(corr^2)
    e[i] = df_add_f(e[i], corr * (2.0f * xf + corr) * p2[i].hi / (2.0f * e[i].hi));
#pragma unroll
    for (int m4 = 1; m4 < 4; ++m4) q[i][m4] = df_mul(xn, p[i][m4]);
    q[i][0] = e[i];
  }
  return true;
}

}  // namespace rw
