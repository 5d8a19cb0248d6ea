// ---- generated by gen/qed_gen.py: ee_5a (e- e+ -> 5 photons), do not edit ----
// 120 Feynman diagrams, 128 helicities; 30 off-shell electron spinors per helicity configuration.
#pragma once
#include "qed.cuh"

namespace rw { namespace ee_5a {
constexpr int NA = 5;
constexpr int NEXT = 7;
constexpr int NHEL = 128;
constexpr int NDIAG = 120;
constexpr int MAX_LB = 5;  // helicity levels that can be spread over lanes
constexpr int IDENT = 5;  // identical photons (1/IDENT!)

// Sum over this lane's photon helicities of |A|^2 (e = 1), electron helicity
// fixed and doubled.  Levels 0..LB-1 (photons 0..LB-1) take their helicity from
// the lane index, the others loop.
template <class R, int LB>
__device__ __forceinline__ R hel_sum(const QedExt<R, NA>& X, const QedKin<R, NA>& Kn, int lane) {
  R acc = R(0);
  const w2<R> S0 = X.u;
  #pragma unroll 1
  for (int i0 = 0; i0 < (LB > 0 ? 1 : 2); ++i0) {
    const int h0 = LB > 0 ? ((lane >> (LB - 1 - 0)) & 1) : i0;
    const ws<R>& E0 = X.eps[0][h0];
    w2<R> t1 = sl_RL(E0, S0);
    const w2<R> S1 = pr_LR(Kn.q[1], t1);
    #pragma unroll 1
    for (int i1 = 0; i1 < (LB > 1 ? 1 : 2); ++i1) {
      const int h1 = LB > 1 ? ((lane >> (LB - 1 - 1)) & 1) : i1;
      const ws<R>& E1 = X.eps[1][h1];
      w2<R> t2 = sl_RL(E1, S0);
      const w2<R> S2 = pr_LR(Kn.q[2], t2);
      w2<R> t3 = sl_RL(E0, S2);
      sl_RL_acc(t3, E1, S1);
      const w2<R> S3 = pr_LR(Kn.q[3], t3);
      #pragma unroll 1
      for (int i2 = 0; i2 < (LB > 2 ? 1 : 2); ++i2) {
        const int h2 = LB > 2 ? ((lane >> (LB - 1 - 2)) & 1) : i2;
        const ws<R>& E2 = X.eps[2][h2];
        w2<R> t4 = sl_RL(E2, S0);
        const w2<R> S4 = pr_LR(Kn.q[4], t4);
        w2<R> t5 = sl_RL(E0, S4);
        sl_RL_acc(t5, E2, S1);
        const w2<R> S5 = pr_LR(Kn.q[5], t5);
        w2<R> t6 = sl_RL(E1, S4);
        sl_RL_acc(t6, E2, S2);
        const w2<R> S6 = pr_LR(Kn.q[6], t6);
        w2<R> t7 = sl_RL(E0, S6);
        sl_RL_acc(t7, E1, S5);
        sl_RL_acc(t7, E2, S3);
        const w2<R> S7 = pr_LR(Kn.q[7], t7);
        #pragma unroll 1
        for (int i3 = 0; i3 < (LB > 3 ? 1 : 2); ++i3) {
          const int h3 = LB > 3 ? ((lane >> (LB - 1 - 3)) & 1) : i3;
          const ws<R>& E3 = X.eps[3][h3];
          w2<R> t8 = sl_RL(E3, S0);
          const w2<R> S8 = pr_LR(Kn.q[8], t8);
          w2<R> t9 = sl_RL(E0, S8);
          sl_RL_acc(t9, E3, S1);
          const w2<R> S9 = pr_LR(Kn.q[9], t9);
          w2<R> t10 = sl_RL(E1, S8);
          sl_RL_acc(t10, E3, S2);
          const w2<R> S10 = pr_LR(Kn.q[10], t10);
          w2<R> t12 = sl_RL(E2, S8);
          sl_RL_acc(t12, E3, S4);
          const w2<R> S12 = pr_LR(Kn.q[12], t12);
          w2<R> t11 = sl_RL(E0, S10);
          sl_RL_acc(t11, E1, S9);
          sl_RL_acc(t11, E3, S3);
          const w2<R> S11 = pr_LR(Kn.q[11], t11);
          w2<R> t13 = sl_RL(E0, S12);
          sl_RL_acc(t13, E2, S9);
          sl_RL_acc(t13, E3, S5);
          const w2<R> S13 = pr_LR(Kn.q[13], t13);
          w2<R> t14 = sl_RL(E1, S12);
          sl_RL_acc(t14, E2, S10);
          sl_RL_acc(t14, E3, S6);
          const w2<R> S14 = pr_LR(Kn.q[14], t14);
          w2<R> t15 = sl_RL(E0, S14);
          sl_RL_acc(t15, E1, S13);
          sl_RL_acc(t15, E2, S11);
          sl_RL_acc(t15, E3, S7);
          const w2<R> S15 = pr_LR(Kn.q[15], t15);
          #pragma unroll 1
          for (int i4 = 0; i4 < (LB > 4 ? 1 : 2); ++i4) {
            const int h4 = LB > 4 ? ((lane >> (LB - 1 - 4)) & 1) : i4;
            const ws<R>& E4 = X.eps[4][h4];
            w2<R> t16 = sl_RL(E4, S0);
            const w2<R> S16 = pr_LR(Kn.q[16], t16);
            w2<R> t17 = sl_RL(E0, S16);
            sl_RL_acc(t17, E4, S1);
            const w2<R> S17 = pr_LR(Kn.q[17], t17);
            w2<R> t18 = sl_RL(E1, S16);
            sl_RL_acc(t18, E4, S2);
            const w2<R> S18 = pr_LR(Kn.q[18], t18);
            w2<R> t20 = sl_RL(E2, S16);
            sl_RL_acc(t20, E4, S4);
            const w2<R> S20 = pr_LR(Kn.q[20], t20);
            w2<R> t24 = sl_RL(E3, S16);
            sl_RL_acc(t24, E4, S8);
            const w2<R> S24 = pr_LR(Kn.q[24], t24);
            w2<R> t19 = sl_RL(E0, S18);
            sl_RL_acc(t19, E1, S17);
            sl_RL_acc(t19, E4, S3);
            const w2<R> S19 = pr_LR(Kn.q[19], t19);
            w2<R> t21 = sl_RL(E0, S20);
            sl_RL_acc(t21, E2, S17);
            sl_RL_acc(t21, E4, S5);
            const w2<R> S21 = pr_LR(Kn.q[21], t21);
            w2<R> t22 = sl_RL(E1, S20);
            sl_RL_acc(t22, E2, S18);
            sl_RL_acc(t22, E4, S6);
            const w2<R> S22 = pr_LR(Kn.q[22], t22);
            w2<R> t25 = sl_RL(E0, S24);
            sl_RL_acc(t25, E3, S17);
            sl_RL_acc(t25, E4, S9);
            const w2<R> S25 = pr_LR(Kn.q[25], t25);
            w2<R> t26 = sl_RL(E1, S24);
            sl_RL_acc(t26, E3, S18);
            sl_RL_acc(t26, E4, S10);
            const w2<R> S26 = pr_LR(Kn.q[26], t26);
            w2<R> t28 = sl_RL(E2, S24);
            sl_RL_acc(t28, E3, S20);
            sl_RL_acc(t28, E4, S12);
            const w2<R> S28 = pr_LR(Kn.q[28], t28);
            w2<R> t23 = sl_RL(E0, S22);
            sl_RL_acc(t23, E1, S21);
            sl_RL_acc(t23, E2, S19);
            sl_RL_acc(t23, E4, S7);
            const w2<R> S23 = pr_LR(Kn.q[23], t23);
            w2<R> t27 = sl_RL(E0, S26);
            sl_RL_acc(t27, E1, S25);
            sl_RL_acc(t27, E3, S19);
            sl_RL_acc(t27, E4, S11);
            const w2<R> S27 = pr_LR(Kn.q[27], t27);
            w2<R> t29 = sl_RL(E0, S28);
            sl_RL_acc(t29, E2, S25);
            sl_RL_acc(t29, E3, S21);
            sl_RL_acc(t29, E4, S13);
            const w2<R> S29 = pr_LR(Kn.q[29], t29);
            w2<R> t30 = sl_RL(E1, S28);
            sl_RL_acc(t30, E2, S26);
            sl_RL_acc(t30, E3, S22);
            sl_RL_acc(t30, E4, S14);
            const w2<R> S30 = pr_LR(Kn.q[30], t30);
            w2<R> T = sl_RL(E0, S30);
            sl_RL_acc(T, E1, S29);
            sl_RL_acc(T, E2, S27);
            sl_RL_acc(T, E3, S23);
            sl_RL_acc(T, E4, S15);
            const cx<R> A = close_L(X.vb, T);
            acc += A.r * A.r + A.i * A.i;
          }
        }
      }
    }
  }
  return R(2) * acc;  // x2: the other electron helicity (all helicities flipped)
}

// floating-point operations of one full helicity sum (all levels, all loop trips)
constexpr long FLOPS_HEL_SUM = 72736;
}}  // namespace
