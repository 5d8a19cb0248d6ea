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
// CM: colour sum by FMA (CM_FMA, any R) or on the tensor cores (CM_FP16/CM_BF16, R = float);
// CM_STORE_FP16/CM_STORE_BF16: no colour sum here, each J vector goes to sink->put()
// for a later tensor-core pass (the return value is then 0).
template <class R, int LB, int CM = CM_FMA, bool JS = false, class Sink = NoSink>
__device__ __forceinline__ R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& Kn, int lane,
                                     [[maybe_unused]] Sink* sink = nullptr) {
  static_assert(CM == CM_FMA || sizeof(R) == 4, "tensor-core colour sum takes FP32 amplitudes");
  constexpr bool MMA = CM == CM_FP16 || CM == CM_BF16;
  const ColourMma<K, MMA ? CM : CM_FP16> cmma(MMA ? CI : nullptr, JS ? NJS * 32 : 0);
  JStore<R, NJS, JS> js;
  R acc = R(0);
  [[maybe_unused]] R cc0_0 = R(0), cc1_0 = R(0), cc2_0 = R(0), cc3_0 = R(0), cc0_1 = R(0), cc1_1 = R(0), cc2_1 = R(0), cc3_1 = R(0);  // per distinct c_ij and top helicity
  {
    const int h0 = 0;
    const cv<R> E0 = h0 ? X.eps[0][1] : X.eps[0][0];
    const ws<R> W0 = weyl_form(E0);
    [[maybe_unused]] sp<R> S_0v0, S_0v1;
    if constexpr (LB < 3) {
      S_0v0 = fprop(Kn.qc[1], Kn.mc[1], slash(W0, X.v[0]));
      S_0v1 = fprop(Kn.qc[1], Kn.mc[1], slash(W0, X.v[1]));
    }
    #pragma unroll 1
    for (int i1 = 0; i1 < (LB >= 1 ? 1 : 2); ++i1) {
      const int h1 = LB >= 1 ? ((lane >> (LB - 1)) & 1) : i1;
      const cv<R> E1 = h1 ? X.eps[1][1] : X.eps[1][0];
      const ws<R> W1 = weyl_form(E1);
      cv<R> J0_1 = vvv(E0, Kn.P[1], E1, Kn.P[2], Kn.cg[3]);
      const cv<R> J1_0 = neg(J0_1);
      #pragma unroll 1
      for (int i2 = 0; i2 < (LB >= 2 ? 1 : 2); ++i2) {
        const int h2 = LB >= 2 ? ((lane >> (LB - 2)) & 1) : i2;
        const cv<R> E2 = h2 ? X.eps[2][1] : X.eps[2][0];
        const ws<R> W2 = weyl_form(E2);
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
          constexpr bool SH = sizeof(R) == 8;  // share every repeated slash (FP64)
          sp<R> S_0;
          if constexpr (LB < 3) S_0 = h3 ? S_0v1 : S_0v0;
          else S_0 = fprop(Kn.qc[1], Kn.mc[1], slash(W0, S_E));
          sp<R> tS_1_0;
          [[maybe_unused]] sp<R> Y0_1__E;  // Jslash(0,1) psi(E)
          if constexpr (true) Y0_1__E = slash(J0_1, S_E);
          if constexpr (true) tS_1_0 = spneg(Y0_1__E); else tS_1_0 = slash(J1_0, S_E);
          slash_acc(tS_1_0, W1, S_0);  // single-gluon term, fused
          const sp<R> S_1_0 = fprop(Kn.qc[3], Kn.mc[3], tS_1_0);
          sp<R> X5;
          [[maybe_unused]] sp<R> Y1_2__0;  // Jslash(1,2) psi(0)
          [[maybe_unused]] sp<R> Y0_1_2__E;  // Jslash(0,1,2) psi(E)
          if constexpr (true) Y1_2__0 = slash(J1_2, S_0);
          if constexpr (true) X5 = spneg(Y1_2__0); else X5 = slash(J2_1, S_0);
          if constexpr (SH) Y0_1_2__E = slash(js.get(0), S_E);
          if constexpr (SH) spadd(X5, Y0_1_2__E); else slash_acc(X5, js.get(0), S_E);
          slash_acc(X5, W2, S_1_0);  // single-gluon term, fused
          const cx<R> A5_0 = rowcol(X.ub[0], X5), A5_1 = rowcol(X.ub[1], X5);
          sp<R> tS_2_0;
          [[maybe_unused]] sp<R> Y0_2__E;  // Jslash(0,2) psi(E)
          if constexpr (true) Y0_2__E = slash(J0_2, S_E);
          if constexpr (true) tS_2_0 = spneg(Y0_2__E); else tS_2_0 = slash(J2_0, S_E);
          slash_acc(tS_2_0, W2, S_0);  // single-gluon term, fused
          const sp<R> S_2_0 = fprop(Kn.qc[5], Kn.mc[5], tS_2_0);
          sp<R> X3;
          [[maybe_unused]] sp<R> Y0_2_1__E;  // Jslash(0,2,1) psi(E)
          if constexpr (true) X3 = Y1_2__0; else X3 = slash(J1_2, S_0);
          if constexpr (true) Y0_2_1__E = slash(js.get(1), S_E);
          if constexpr (true) spadd(X3, Y0_2_1__E); else slash_acc(X3, js.get(1), S_E);
          slash_acc(X3, W1, S_2_0);  // single-gluon term, fused
          const cx<R> A3_0 = rowcol(X.ub[0], X3), A3_1 = rowcol(X.ub[1], X3);
          sp<R> tS_1 = slash(W1, S_E);
          const sp<R> S_1 = fprop(Kn.qc[2], Kn.mc[2], tS_1);
          sp<R> tS_0_1;
          if constexpr (true) tS_0_1 = Y0_1__E; else tS_0_1 = slash(J0_1, S_E);
          slash_acc(tS_0_1, W0, S_1);  // single-gluon term, fused
          const sp<R> S_0_1 = fprop(Kn.qc[3], Kn.mc[3], tS_0_1);
          sp<R> X4;
          [[maybe_unused]] sp<R> Y0_2__1;  // Jslash(0,2) psi(1)
          [[maybe_unused]] sp<R> Y1_0_2__E;  // Jslash(1,0,2) psi(E)
          if constexpr (true) Y0_2__1 = slash(J0_2, S_1);
          if constexpr (true) X4 = spneg(Y0_2__1); else X4 = slash(J2_0, S_1);
          if constexpr (true) Y1_0_2__E = slash(js.get(2), S_E);
          if constexpr (true) spadd(X4, Y1_0_2__E); else slash_acc(X4, js.get(2), S_E);
          slash_acc(X4, W2, S_0_1);  // single-gluon term, fused
          const cx<R> A4_0 = rowcol(X.ub[0], X4), A4_1 = rowcol(X.ub[1], X4);
          sp<R> tS_2_1;
          [[maybe_unused]] sp<R> Y1_2__E;  // Jslash(1,2) psi(E)
          if constexpr (true) Y1_2__E = slash(J1_2, S_E);
          if constexpr (true) tS_2_1 = spneg(Y1_2__E); else tS_2_1 = slash(J2_1, S_E);
          slash_acc(tS_2_1, W2, S_1);  // single-gluon term, fused
          const sp<R> S_2_1 = fprop(Kn.qc[6], Kn.mc[6], tS_2_1);
          sp<R> X1;
          if constexpr (true) X1 = Y0_2__1; else X1 = slash(J0_2, S_1);
          if constexpr (true) spadd(X1, Y0_2_1__E); else slash_acc(X1, js.get(1), S_E);
          slash_acc(X1, W0, S_2_1);  // single-gluon term, fused
          const cx<R> A1_0 = rowcol(X.ub[0], X1), A1_1 = rowcol(X.ub[1], X1);
          sp<R> tS_2 = slash(W2, S_E);
          const sp<R> S_2 = fprop(Kn.qc[4], Kn.mc[4], tS_2);
          sp<R> tS_0_2;
          if constexpr (true) tS_0_2 = Y0_2__E; else tS_0_2 = slash(J0_2, S_E);
          slash_acc(tS_0_2, W0, S_2);  // single-gluon term, fused
          const sp<R> S_0_2 = fprop(Kn.qc[5], Kn.mc[5], tS_0_2);
          sp<R> X2;
          [[maybe_unused]] sp<R> Y0_1__2;  // Jslash(0,1) psi(2)
          if constexpr (true) Y0_1__2 = slash(J0_1, S_2);
          if constexpr (true) X2 = spneg(Y0_1__2); else X2 = slash(J1_0, S_2);
          if constexpr (true) spadd(X2, Y1_0_2__E); else slash_acc(X2, js.get(2), S_E);
          slash_acc(X2, W1, S_0_2);  // single-gluon term, fused
          const cx<R> A2_0 = rowcol(X.ub[0], X2), A2_1 = rowcol(X.ub[1], X2);
          sp<R> tS_1_2;
          if constexpr (true) tS_1_2 = Y1_2__E; else tS_1_2 = slash(J1_2, S_E);
          slash_acc(tS_1_2, W1, S_2);  // single-gluon term, fused
          const sp<R> S_1_2 = fprop(Kn.qc[6], Kn.mc[6], tS_1_2);
          sp<R> X0;
          if constexpr (true) X0 = Y0_1__2; else X0 = slash(J0_1, S_2);
          if constexpr (SH) spadd(X0, Y0_1_2__E); else slash_acc(X0, js.get(0), S_E);
          slash_acc(X0, W0, S_1_2);  // single-gluon term, fused
          const cx<R> A0_0 = rowcol(X.ub[0], X0), A0_1 = rowcol(X.ub[1], X0);
          if constexpr (CM != CM_FMA) {
            const cx<float> Aa0[K] = {A0_0, A1_0, A2_0, A3_0, A4_0, A5_0};
            const cx<float> Aa1[K] = {A0_1, A1_1, A2_1, A3_1, A4_1, A5_1};
            if constexpr (MMA) {
              acc += R(2) * (cmma.sum(Aa0) + cmma.sum(Aa1));  // x2 helicity flip
            } else {
              sink->put(Aa0);
              sink->put(Aa1);
            }
          } else {
            cc0_0 = fmadd(A0_0.r, A0_0.r, fmadd(A0_0.i, A0_0.i, cc0_0));
            cc1_0 = fmadd(A0_0.r, A1_0.r, fmadd(A0_0.i, A1_0.i, cc1_0));
            cc1_0 = fmadd(A0_0.r, A2_0.r, fmadd(A0_0.i, A2_0.i, cc1_0));
            cc2_0 = fmadd(A0_0.r, A3_0.r, fmadd(A0_0.i, A3_0.i, cc2_0));
            cc2_0 = fmadd(A0_0.r, A4_0.r, fmadd(A0_0.i, A4_0.i, cc2_0));
            cc3_0 = fmadd(A0_0.r, A5_0.r, fmadd(A0_0.i, A5_0.i, cc3_0));
            cc0_0 = fmadd(A1_0.r, A1_0.r, fmadd(A1_0.i, A1_0.i, cc0_0));
            cc2_0 = fmadd(A1_0.r, A2_0.r, fmadd(A1_0.i, A2_0.i, cc2_0));
            cc3_0 = fmadd(A1_0.r, A3_0.r, fmadd(A1_0.i, A3_0.i, cc3_0));
            cc1_0 = fmadd(A1_0.r, A4_0.r, fmadd(A1_0.i, A4_0.i, cc1_0));
            cc2_0 = fmadd(A1_0.r, A5_0.r, fmadd(A1_0.i, A5_0.i, cc2_0));
            cc0_0 = fmadd(A2_0.r, A2_0.r, fmadd(A2_0.i, A2_0.i, cc0_0));
            cc1_0 = fmadd(A2_0.r, A3_0.r, fmadd(A2_0.i, A3_0.i, cc1_0));
            cc3_0 = fmadd(A2_0.r, A4_0.r, fmadd(A2_0.i, A4_0.i, cc3_0));
            cc2_0 = fmadd(A2_0.r, A5_0.r, fmadd(A2_0.i, A5_0.i, cc2_0));
            cc0_0 = fmadd(A3_0.r, A3_0.r, fmadd(A3_0.i, A3_0.i, cc0_0));
            cc2_0 = fmadd(A3_0.r, A4_0.r, fmadd(A3_0.i, A4_0.i, cc2_0));
            cc1_0 = fmadd(A3_0.r, A5_0.r, fmadd(A3_0.i, A5_0.i, cc1_0));
            cc0_0 = fmadd(A4_0.r, A4_0.r, fmadd(A4_0.i, A4_0.i, cc0_0));
            cc1_0 = fmadd(A4_0.r, A5_0.r, fmadd(A4_0.i, A5_0.i, cc1_0));
            cc0_0 = fmadd(A5_0.r, A5_0.r, fmadd(A5_0.i, A5_0.i, cc0_0));
            cc0_1 = fmadd(A0_1.r, A0_1.r, fmadd(A0_1.i, A0_1.i, cc0_1));
            cc1_1 = fmadd(A0_1.r, A1_1.r, fmadd(A0_1.i, A1_1.i, cc1_1));
            cc1_1 = fmadd(A0_1.r, A2_1.r, fmadd(A0_1.i, A2_1.i, cc1_1));
            cc2_1 = fmadd(A0_1.r, A3_1.r, fmadd(A0_1.i, A3_1.i, cc2_1));
            cc2_1 = fmadd(A0_1.r, A4_1.r, fmadd(A0_1.i, A4_1.i, cc2_1));
            cc3_1 = fmadd(A0_1.r, A5_1.r, fmadd(A0_1.i, A5_1.i, cc3_1));
            cc0_1 = fmadd(A1_1.r, A1_1.r, fmadd(A1_1.i, A1_1.i, cc0_1));
            cc2_1 = fmadd(A1_1.r, A2_1.r, fmadd(A1_1.i, A2_1.i, cc2_1));
            cc3_1 = fmadd(A1_1.r, A3_1.r, fmadd(A1_1.i, A3_1.i, cc3_1));
            cc1_1 = fmadd(A1_1.r, A4_1.r, fmadd(A1_1.i, A4_1.i, cc1_1));
            cc2_1 = fmadd(A1_1.r, A5_1.r, fmadd(A1_1.i, A5_1.i, cc2_1));
            cc0_1 = fmadd(A2_1.r, A2_1.r, fmadd(A2_1.i, A2_1.i, cc0_1));
            cc1_1 = fmadd(A2_1.r, A3_1.r, fmadd(A2_1.i, A3_1.i, cc1_1));
            cc3_1 = fmadd(A2_1.r, A4_1.r, fmadd(A2_1.i, A4_1.i, cc3_1));
            cc2_1 = fmadd(A2_1.r, A5_1.r, fmadd(A2_1.i, A5_1.i, cc2_1));
            cc0_1 = fmadd(A3_1.r, A3_1.r, fmadd(A3_1.i, A3_1.i, cc0_1));
            cc2_1 = fmadd(A3_1.r, A4_1.r, fmadd(A3_1.i, A4_1.i, cc2_1));
            cc1_1 = fmadd(A3_1.r, A5_1.r, fmadd(A3_1.i, A5_1.i, cc1_1));
            cc0_1 = fmadd(A4_1.r, A4_1.r, fmadd(A4_1.i, A4_1.i, cc0_1));
            cc1_1 = fmadd(A4_1.r, A5_1.r, fmadd(A4_1.i, A5_1.i, cc1_1));
            cc0_1 = fmadd(A5_1.r, A5_1.r, fmadd(A5_1.i, A5_1.i, cc0_1));
          }
        }
      }
    }
  }
  if constexpr (CM == CM_FMA) acc = R(2) * (R(64) * (cc0_0 + cc0_1) + R(-16) * (cc1_0 + cc1_1) + R(2) * (cc2_0 + cc2_1) + R(20) * (cc3_0 + cc3_1));  // x2 helicity flip
  return acc;
}

// floating-point operations of one full helicity sum (all levels, all loop trips)
constexpr long FLOPS_HEL_SUM = 28077;
}}  // namespace
