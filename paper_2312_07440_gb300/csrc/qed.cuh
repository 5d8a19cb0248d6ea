// Building blocks and per-event set-up of e- e+ -> n photons (massless QED).
//
// With massless electrons each spinor on the line has one chirality: the
// chain starts from the right-handed part of u(p0, +), every gamma matrix
// (photon vertex, propagator) swaps the chiral blocks, and it closes on the
// left-handed slot of vbar(p1, -).  The chains therefore run on
// two-component Weyl spinors with the 2x2 blocks of the chiral-basis
// (gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]]) Dirac matrices:
//   a-slash on (0, s_R) -> (A s_R, 0),  A  = [[a0 - a3, -(a1 - i a2)], [-(a1 + i a2), a0 + a3]],
//   a-slash on (s_L, 0) -> (0, B s_L),  B  = [[a0 + a3, a1 - i a2], [a1 + i a2, a0 - a3]].
// The other electron helicity gives the complex-conjugate amplitudes (all
// helicities flipped), so the helicity sum is doubled instead of evaluated.
#pragma once
#include "dfloat.cuh"
#include "helas.cuh"

namespace rw {

template <class R>
struct w2 {  // two-component Weyl spinor
  cx<R> c[2];
};

// eps-slash on a right-handed spinor -> left-handed                        (28 flops)
template <class R>
__device__ __forceinline__ w2<R> sl_RL(const ws<R>& a, const w2<R>& s) {
  return {{cmsc(a.bm, s.c[1], cmul(a.am, s.c[0])), cmsc(a.bp, s.c[0], cmul(a.ap, s.c[1]))}};
}
// o += eps-slash s, fused                                                  (+4 flops)
template <class R>
__device__ __forceinline__ void sl_RL_acc(w2<R>& o, const ws<R>& a, const w2<R>& s) {
  o.c[0] = cmsc(a.bm, s.c[1], cmac(a.am, s.c[0], o.c[0]));
  o.c[1] = cmsc(a.bp, s.c[0], cmac(a.ap, s.c[1], o.c[1]));
}

// massless propagator qslash/q^2 on a left-handed spinor -> right-handed;
// q = (q0 + q3, q0 - q3, q1, q2) / q^2                                     (20 flops)
template <class R>
__device__ __forceinline__ w2<R> pr_LR(const R (&q)[4], const w2<R>& s) {
  const cx<R> s0 = s.c[0], s1 = s.c[1];
  return {{{fmadd(q[3], s1.i, fmadd(q[2], s1.r, q[0] * s0.r)), fmadd(-q[3], s1.r, fmadd(q[2], s1.i, q[0] * s0.i))},
           {fmadd(q[1], s1.r, fmadd(-q[3], s0.i, q[2] * s0.r)), fmadd(q[1], s1.i, fmadd(q[3], s0.r, q[2] * s0.i))}}};
}

// vbar (left-handed slot, a row) . psi                                     (14 flops)
template <class R>
__device__ __forceinline__ cx<R> close_L(const w2<R>& vb, const w2<R>& s) {
  return cmac(vb.c[1], s.c[1], cmul(vb.c[0], s.c[0]));
}

template <class R, int NA>
struct QedExt {
  w2<R> u;            // right-handed part of u(p0, +1/2)
  w2<R> vb;           // left-handed slot of vbar(p1, -1/2)
  ws<R> eps[NA][2];   // eps*(k_i, +), eps*(k_i, -) in Weyl-block form
};

template <class R, int NA>
struct QedKin {
  R q[1 << NA][4];  // per photon subset T: (q0 + q3, q0 - q3, q1, q2) / q^2, q = p0 - k_T
};

template <class R, int NA, int NEXT>
__device__ __forceinline__ void qed_wavefunctions(const R (&pr)[NEXT][4], QedExt<R, NA>& X) {
  sp<R> u4[2], vb4[2];
  u_in<R>(pr[0], R(0), u4);
  vbar_in<R>(pr[1], R(0), vb4);
  X.u = {{u4[0].c[2], u4[0].c[3]}};
  X.vb = {{vb4[1].c[0], vb4[1].c[1]}};
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    cv<R> e[2];
    polvec<R>(pr[2 + i], true, e);
    X.eps[i][0] = weyl_form(e[0]);
    X.eps[i][1] = weyl_form(e[1]);
  }
}

// FP64 momenta: q^2 = -2 sum_{i in T} p0.k_i + 2 sum_{i<j in T} k_i.k_j from
// FP64 dot products, q in FP64, then scaled and rounded to R.
template <class R, int NA, int NEXT>
__device__ __forceinline__ void qed_setup(const double (&p)[NEXT][4], QedExt<R, NA>& X, QedKin<R, NA>& Kn) {
  static_assert(NEXT == NA + 2, "e- e+ + NA photons");
  R pr[NEXT][4];
#pragma unroll
  for (int i = 0; i < NEXT; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) pr[i][m] = R(p[i][m]);
  qed_wavefunctions<R, NA, NEXT>(pr, X);
  auto dot = [](const double (&a)[4], const double (&b)[4]) {
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  };
  double d0[NA], dk[NA][NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    d0[i] = dot(p[0], p[2 + i]);
#pragma unroll
    for (int j = i + 1; j < NA; ++j) dk[i][j] = dot(p[2 + i], p[2 + j]);
  }
  constexpr int FULL = (1 << NA) - 1;
#pragma unroll
  for (int msk = 1; msk < FULL; ++msk) {
    double q[4] = {p[0][0], p[0][1], p[0][2], p[0][3]}, q2 = 0.0;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      if (!((msk >> i) & 1)) continue;
#pragma unroll
      for (int m = 0; m < 4; ++m) q[m] -= p[2 + i][m];
      q2 -= 2.0 * d0[i];
#pragma unroll
      for (int j = i + 1; j < NA; ++j)
        if ((msk >> j) & 1) q2 += 2.0 * dk[i][j];
    }
    const R c = R(1) / R(q2);
    Kn.q[msk][0] = c * R(q[0] + q[3]);
    Kn.q[msk][1] = c * R(q[0] - q[3]);
    Kn.q[msk][2] = c * R(q[1]);
    Kn.q[msk][3] = c * R(q[2]);
  }
}

// FP32 modes: the same from double-float momenta, the invariants q^2 in
// double-float (dfloat.cuh), everything else -- the numerator vector q
// included, which is never formed by cancellation against itself -- in float.
template <class R, int NA, int NEXT>
__device__ __forceinline__ void qed_setup(const df (&p)[NEXT][4], QedExt<R, NA>& X, QedKin<R, NA>& Kn) {
  static_assert(NEXT == NA + 2, "e- e+ + NA photons");
  static_assert(sizeof(R) == 4, "double-float set-up feeds FP32 amplitudes");
  R pr[NEXT][4];
#pragma unroll
  for (int i = 0; i < NEXT; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) pr[i][m] = p[i][m].hi;
  qed_wavefunctions<R, NA, NEXT>(pr, X);
  df d0[NA], dk[NA][NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    d0[i] = df_scale(df_dot4(p[0], p[2 + i]), -2.0f);
#pragma unroll
    for (int j = i + 1; j < NA; ++j) dk[i][j] = df_scale(df_dot4(p[2 + i], p[2 + j]), 2.0f);
  }
  constexpr int FULL = (1 << NA) - 1;
#pragma unroll
  for (int msk = 1; msk < FULL; ++msk) {
    R q[4] = {pr[0][0], pr[0][1], pr[0][2], pr[0][3]};
    df q2 = {0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      if (!((msk >> i) & 1)) continue;
#pragma unroll
      for (int m = 0; m < 4; ++m) q[m] -= pr[2 + i][m];
      q2 = df_add(q2, d0[i]);
#pragma unroll
      for (int j = i + 1; j < NA; ++j)
        if ((msk >> j) & 1) q2 = df_add(q2, dk[i][j]);
    }
    const R c = R(1) / q2.hi;
    Kn.q[msk][0] = c * (q[0] + q[3]);
    Kn.q[msk][1] = c * (q[0] - q[3]);
    Kn.q[msk][2] = c * q[1];
    Kn.q[msk][3] = c * q[2];
  }
}

}  // namespace rw
