// Per-event set-up for g g -> t tbar + n g: external wavefunctions of both
// helicities (in the working precision R, cancellation-free formulas) and the
// propagator invariants, whose dot products are formed in FP64 from the FP64
// momenta (so FP32 mode never forms p^2 - m^2 by cancellation in single
// precision) before the reciprocals are taken in R.
#pragma once
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

// particle index of gluon g on the top line: 0, 1 incoming, then 4, 5, ...
__host__ __device__ constexpr int gluon_particle(int g) { return g < 2 ? g : g + 2; }

__device__ __forceinline__ double dot4(const double (&a)[4], const double (&b)[4]) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
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
  // Invariants: the dot products, where cancellation happens, in FP64;
  // the reciprocals in the working precision.
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
    if (cnt >= 2) {
      const R inv = R(1) / R(K2);
      Kn.cg[msk] = -inv;
      Kn.c4[msk] = inv;
    } else {
      Kn.cg[msk] = R(0);
      Kn.c4[msk] = R(0);
    }
    if (msk != FULL) {
      // (K - p4)^2 - m^2 = K^2 - 2 K.p4  (p4^2 = m^2)
      const double den = K2 - 2.0 * dot4(P, p[3]);
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

}  // namespace rw
