// ---- generated by gen/qcd_gen.py: gg_ttg (g g -> t tbar + 1 g), do not edit ----
// 16 Feynman diagrams, 6 colour orderings, 32 helicities.
// colour matrix C = Cint / 9
#pragma once
#include "colour_mma.cuh"
#include "qcd.cuh"

namespace rw { namespace gg_ttg {
constexpr int NG = 3;
constexpr int NEXT = 5;
constexpr int K = 6;
constexpr int NHEL = 32;
constexpr int NDIAG = 16;
constexpr int MAX_LB = 3;  // helicity levels that can be spread over lanes
constexpr int NJS = 3;  // currents of 3+ gluons, one JStore slot each
constexpr int CDEN = 9;
constexpr int IDENT = 1;  // identical outgoing gluons (1/IDENT!)
constexpr unsigned OUTGOING_GLUONS = 4u;  // bit g: gluon g outgoing
__host__ __device__ constexpr int cint(int i, int j) { constexpr int c[K * K] = {64, -8, -8, 1, 1, 10, -8, 64, 1, 10, -8, 1, -8, 1, 64, -8, 10, 1, 1, 10, -8, 64, 1, -8, 1, -8, 10, 1, 64, -8, 10, 1, 1, -8, -8, 64}; return c[i * K + j]; }
constexpr int ORDER[K][NG] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
static __device__ const short CI[K * K] = {64, -8, -8, 1, 1, 10, -8, 64, 1, 10, -8, 1, -8, 1, 64, -8, 10, 1, 1, 10, -8, 64, 1, -8, 1, -8, 10, 1, 64, -8, 10, 1, 1, -8, -8, 64};  // row-major C_int for the tensor-core sum

// Sum over this lane's helicities of sum_{s,t} Cint_st Re(A_s^* A_t), g = 1;
// helicities with gluon 0 at +1 only, doubled (J^dagger C J(h) = J^dagger C J(-h)).
// CM: colour sum by FMA (CM_FMA, any R) or on the tensor cores (CM_FP16/CM_BF16, R = float).
template <class R, int LB, int CM = CM_FMA, bool JS = false>
__device__ __forceinline__ R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& Kn, int lane) {
  static_assert(CM == CM_FMA || sizeof(R) == 4, "tensor-core colour sum takes FP32 amplitudes");
  const ColourMma<K, CM == CM_FMA ? CM_FP16 : CM> cmma(CM == CM_FMA ? nullptr : CI);
  JStore<R, NJS, JS> js;
  R acc = R(0);
  {
    const int h0 = 0;
    const cv<R> E0 = h0 ? X.eps[0][1] : X.eps[0][0];
    #pragma unroll 1
    for (int i1 = 0; i1 < (LB >= 1 ? 1 : 2); ++i1) {
      const int h1 = LB >= 1 ? ((lane >> (LB - 1)) & 1) : i1;
      const cv<R> E1 = h1 ? X.eps[1][1] : X.eps[1][0];
      cv<R> J0_1 = vvv(E0, Kn.P[1], E1, Kn.P[2], Kn.cg[3]);
      const cv<R> J1_0 = neg(J0_1);
      #pragma unroll 1
      for (int i2 = 0; i2 < (LB >= 2 ? 1 : 2); ++i2) {
        const int h2 = LB >= 2 ? ((lane >> (LB - 2)) & 1) : i2;
        const cv<R> E2 = h2 ? X.eps[2][1] : X.eps[2][0];
        cv<R> J0_2 = vvv(E0, Kn.P[1], E2, Kn.P[4], Kn.cg[5]);
        cv<R> J1_2 = vvv(E1, Kn.P[2], E2, Kn.P[4], Kn.cg[6]);
        const cv<R> J2_0 = neg(J0_2);
        const cv<R> J2_1 = neg(J1_2);
        cv<R> J0_1_2 = vvv(E0, Kn.P[1], J1_2, Kn.P[6], Kn.cg[7]);
        vvv_acc(J0_1_2, J0_1, Kn.P[3], E2, Kn.P[4], Kn.cg[7]);
        vvvv_acc(J0_1_2, E0, E1, E2, Kn.c4[7]);
        js.put(0, J0_1_2);
        cv<R> J0_2_1 = vvv(E0, Kn.P[1], J2_1, Kn.P[6], Kn.cg[7]);
        vvv_acc(J0_2_1, J0_2, Kn.P[5], E1, Kn.P[2], Kn.cg[7]);
        vvvv_acc(J0_2_1, E0, E2, E1, Kn.c4[7]);
        js.put(1, J0_2_1);
        cv<R> J1_0_2 = vvv(E1, Kn.P[2], J0_2, Kn.P[5], Kn.cg[7]);
        vvv_acc(J1_0_2, J1_0, Kn.P[3], E2, Kn.P[4], Kn.cg[7]);
        vvvv_acc(J1_0_2, E1, E0, E2, Kn.c4[7]);
        js.put(2, J1_0_2);
        #pragma unroll 1
        for (int i3 = 0; i3 < (LB >= 3 ? 1 : 2); ++i3) {
          const int h3 = LB >= 3 ? ((lane >> (LB - 3)) & 1) : i3;
          const sp<R> S_E = h3 ? X.v[1] : X.v[0];
          sp<R> tS_0 = slash(E0, S_E);
          const sp<R> S_0 = fprop(Kn.qc[1], Kn.mc[1], tS_0);
          sp<R> tS_1_0 = slash(E1, S_0);
          slash_acc(tS_1_0, J1_0, S_E);
          const sp<R> S_1_0 = fprop(Kn.qc[3], Kn.mc[3], tS_1_0);
          sp<R> X5 = slash(E2, S_1_0);
          slash_acc(X5, J2_1, S_0);
          slash_acc(X5, js.get(0), S_E);
          const cx<R> A5_0 = rowcol(X.ub[0], X5), A5_1 = rowcol(X.ub[1], X5);
          sp<R> tS_2_0 = slash(E2, S_0);
          slash_acc(tS_2_0, J2_0, S_E);
          const sp<R> S_2_0 = fprop(Kn.qc[5], Kn.mc[5], tS_2_0);
          sp<R> X3 = slash(E1, S_2_0);
          slash_acc(X3, J1_2, S_0);
          slash_acc(X3, js.get(1), S_E);
          const cx<R> A3_0 = rowcol(X.ub[0], X3), A3_1 = rowcol(X.ub[1], X3);
          sp<R> tS_1 = slash(E1, S_E);
          const sp<R> S_1 = fprop(Kn.qc[2], Kn.mc[2], tS_1);
          sp<R> tS_0_1 = slash(E0, S_1);
          slash_acc(tS_0_1, J0_1, S_E);
          const sp<R> S_0_1 = fprop(Kn.qc[3], Kn.mc[3], tS_0_1);
          sp<R> X4 = slash(E2, S_0_1);
          slash_acc(X4, J2_0, S_1);
          slash_acc(X4, js.get(2), S_E);
          const cx<R> A4_0 = rowcol(X.ub[0], X4), A4_1 = rowcol(X.ub[1], X4);
          sp<R> tS_2_1 = slash(E2, S_1);
          slash_acc(tS_2_1, J2_1, S_E);
          const sp<R> S_2_1 = fprop(Kn.qc[6], Kn.mc[6], tS_2_1);
          sp<R> X1 = slash(E0, S_2_1);
          slash_acc(X1, J0_2, S_1);
          slash_acc(X1, js.get(1), S_E);
          const cx<R> A1_0 = rowcol(X.ub[0], X1), A1_1 = rowcol(X.ub[1], X1);
          sp<R> tS_2 = slash(E2, S_E);
          const sp<R> S_2 = fprop(Kn.qc[4], Kn.mc[4], tS_2);
          sp<R> tS_0_2 = slash(E0, S_2);
          slash_acc(tS_0_2, J0_2, S_E);
          const sp<R> S_0_2 = fprop(Kn.qc[5], Kn.mc[5], tS_0_2);
          sp<R> X2 = slash(E1, S_0_2);
          slash_acc(X2, J1_0, S_2);
          slash_acc(X2, js.get(2), S_E);
          const cx<R> A2_0 = rowcol(X.ub[0], X2), A2_1 = rowcol(X.ub[1], X2);
          sp<R> tS_1_2 = slash(E1, S_2);
          slash_acc(tS_1_2, J1_2, S_E);
          const sp<R> S_1_2 = fprop(Kn.qc[6], Kn.mc[6], tS_1_2);
          sp<R> X0 = slash(E0, S_1_2);
          slash_acc(X0, J0_1, S_2);
          slash_acc(X0, js.get(0), S_E);
          const cx<R> A0_0 = rowcol(X.ub[0], X0), A0_1 = rowcol(X.ub[1], X0);
          if constexpr (CM != CM_FMA) {
            const cx<float> Aa0[K] = {A0_0, A1_0, A2_0, A3_0, A4_0, A5_0};
            const cx<float> Aa1[K] = {A0_1, A1_1, A2_1, A3_1, A4_1, A5_1};
            acc += R(2) * (cmma.sum(Aa0) + cmma.sum(Aa1));  // x2 helicity flip
          } else {
            R cs = R(0);
            { const R zr = R(64) * R(0.5) * A0_0.r + R(-8) * A1_0.r + R(-8) * A2_0.r + R(1) * A3_0.r + R(1) * A4_0.r + R(10) * A5_0.r; const R zi = R(64) * R(0.5) * A0_0.i + R(-8) * A1_0.i + R(-8) * A2_0.i + R(1) * A3_0.i + R(1) * A4_0.i + R(10) * A5_0.i;
              cs += A0_0.r * zr + A0_0.i * zi; }
            { const R zr = R(64) * R(0.5) * A1_0.r + R(1) * A2_0.r + R(10) * A3_0.r + R(-8) * A4_0.r + R(1) * A5_0.r; const R zi = R(64) * R(0.5) * A1_0.i + R(1) * A2_0.i + R(10) * A3_0.i + R(-8) * A4_0.i + R(1) * A5_0.i;
              cs += A1_0.r * zr + A1_0.i * zi; }
            { const R zr = R(64) * R(0.5) * A2_0.r + R(-8) * A3_0.r + R(10) * A4_0.r + R(1) * A5_0.r; const R zi = R(64) * R(0.5) * A2_0.i + R(-8) * A3_0.i + R(10) * A4_0.i + R(1) * A5_0.i;
              cs += A2_0.r * zr + A2_0.i * zi; }
            { const R zr = R(64) * R(0.5) * A3_0.r + R(1) * A4_0.r + R(-8) * A5_0.r; const R zi = R(64) * R(0.5) * A3_0.i + R(1) * A4_0.i + R(-8) * A5_0.i;
              cs += A3_0.r * zr + A3_0.i * zi; }
            { const R zr = R(64) * R(0.5) * A4_0.r + R(-8) * A5_0.r; const R zi = R(64) * R(0.5) * A4_0.i + R(-8) * A5_0.i;
              cs += A4_0.r * zr + A4_0.i * zi; }
            { const R zr = R(64) * R(0.5) * A5_0.r; const R zi = R(64) * R(0.5) * A5_0.i;
              cs += A5_0.r * zr + A5_0.i * zi; }
            { const R zr = R(64) * R(0.5) * A0_1.r + R(-8) * A1_1.r + R(-8) * A2_1.r + R(1) * A3_1.r + R(1) * A4_1.r + R(10) * A5_1.r; const R zi = R(64) * R(0.5) * A0_1.i + R(-8) * A1_1.i + R(-8) * A2_1.i + R(1) * A3_1.i + R(1) * A4_1.i + R(10) * A5_1.i;
              cs += A0_1.r * zr + A0_1.i * zi; }
            { const R zr = R(64) * R(0.5) * A1_1.r + R(1) * A2_1.r + R(10) * A3_1.r + R(-8) * A4_1.r + R(1) * A5_1.r; const R zi = R(64) * R(0.5) * A1_1.i + R(1) * A2_1.i + R(10) * A3_1.i + R(-8) * A4_1.i + R(1) * A5_1.i;
              cs += A1_1.r * zr + A1_1.i * zi; }
            { const R zr = R(64) * R(0.5) * A2_1.r + R(-8) * A3_1.r + R(10) * A4_1.r + R(1) * A5_1.r; const R zi = R(64) * R(0.5) * A2_1.i + R(-8) * A3_1.i + R(10) * A4_1.i + R(1) * A5_1.i;
              cs += A2_1.r * zr + A2_1.i * zi; }
            { const R zr = R(64) * R(0.5) * A3_1.r + R(1) * A4_1.r + R(-8) * A5_1.r; const R zi = R(64) * R(0.5) * A3_1.i + R(1) * A4_1.i + R(-8) * A5_1.i;
              cs += A3_1.r * zr + A3_1.i * zi; }
            { const R zr = R(64) * R(0.5) * A4_1.r + R(-8) * A5_1.r; const R zi = R(64) * R(0.5) * A4_1.i + R(-8) * A5_1.i;
              cs += A4_1.r * zr + A4_1.i * zi; }
            { const R zr = R(64) * R(0.5) * A5_1.r; const R zi = R(64) * R(0.5) * A5_1.i;
              cs += A5_1.r * zr + A5_1.i * zi; }
            acc += R(4) * cs;  // x2 symmetric colour sum, x2 helicity flip
          }
        }
      }
    }
  }
  return acc;
}

// floating-point operations of one full helicity sum (all levels, all loop trips)
constexpr long FLOPS_HEL_SUM = 34644;
}}  // namespace
