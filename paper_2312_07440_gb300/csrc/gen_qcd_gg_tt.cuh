// ---- generated by gen/qcd_gen.py: gg_tt (g g -> t tbar + 0 g), do not edit ----
// 3 Feynman diagrams, 2 colour orderings, 16 helicities.
// colour matrix C = Cint / 3
#pragma once
#include "colour_mma.cuh"
#include "qcd.cuh"

namespace rw { namespace gg_tt {
constexpr int NG = 2;
constexpr int NEXT = 4;
constexpr int K = 2;
constexpr int NHEL = 16;
constexpr int NDIAG = 3;
constexpr int MAX_LB = 2;  // helicity levels that can be spread over lanes
constexpr int NJS = 0;  // currents of 3+ gluons, one JStore slot each
constexpr int CDEN = 3;
constexpr int IDENT = 1;  // identical outgoing gluons (1/IDENT!)
constexpr unsigned OUTGOING_GLUONS = 0u;  // bit g: gluon g outgoing
__host__ __device__ constexpr int cint(int i, int j) { constexpr int c[K * K] = {16, -2, -2, 16}; return c[i * K + j]; }
constexpr int ORDER[K][NG] = {{0, 1}, {1, 0}};
static __device__ const short CI[K * K] = {16, -2, -2, 16};  // row-major C_int for the tensor-core sum

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
  [[maybe_unused]] R cc0_0 = R(0), cc1_0 = R(0), cc0_1 = R(0), cc1_1 = R(0);  // per distinct c_ij and top helicity
  {
    const int h0 = 0;
    const cv<R> E0 = h0 ? X.eps[0][1] : X.eps[0][0];
    const ws<R> W0 = weyl_form(E0);
    [[maybe_unused]] sp<R> S_0v0, S_0v1;
    if constexpr (LB < 2) {
      S_0v0 = fprop(Kn.qc[1], Kn.mc[1], slash(W0, X.v[0]));
      S_0v1 = fprop(Kn.qc[1], Kn.mc[1], slash(W0, X.v[1]));
    }
    #pragma unroll 1
    for (int i1 = 0; i1 < (LB >= 1 ? 1 : 2); ++i1) {
      const int h1 = LB >= 1 ? ((lane >> (LB - 1)) & 1) : i1;
      const cv<R> E1 = h1 ? X.eps[1][1] : X.eps[1][0];
      const ws<R> W1 = weyl_form(E1);
      cv<R> J0_1 = vvv(E0, Kn.P[1], E1, Kn.P[2], Kn.cg[3]);
      const ws<R> WJ0_1 = weyl_form(J0_1);
      const cv<R> J1_0 = neg(J0_1);
      #pragma unroll 1
      for (int i2 = 0; i2 < (LB >= 2 ? 1 : 2); ++i2) {
        const int h2 = LB >= 2 ? ((lane >> (LB - 2)) & 1) : i2;
        const sp<R> S_E = h2 ? X.v[1] : X.v[0];
        constexpr bool SH = sizeof(R) == 8;  // share every repeated slash (FP64)
        sp<R> S_0;
        if constexpr (LB < 2) S_0 = h2 ? S_0v1 : S_0v0;
        else S_0 = fprop(Kn.qc[1], Kn.mc[1], slash(W0, S_E));
        sp<R> X1;
        [[maybe_unused]] sp<R> Y0_1__E;  // Jslash(0,1) psi(E)
        if constexpr (true) Y0_1__E = slash(WJ0_1, S_E);
        if constexpr (true) X1 = spneg(Y0_1__E); else X1 = slash(J1_0, S_E);
        slash_acc(X1, W1, S_0);  // single-gluon term, fused
        const cx<R> A1_0 = rowcol(X.ub[0], X1), A1_1 = rowcol(X.ub[1], X1);
        sp<R> tS_1 = slash(W1, S_E);
        const sp<R> S_1 = fprop(Kn.qc[2], Kn.mc[2], tS_1);
        sp<R> X0;
        if constexpr (true) X0 = Y0_1__E; else X0 = slash(J0_1, S_E);
        slash_acc(X0, W0, S_1);  // single-gluon term, fused
        const cx<R> A0_0 = rowcol(X.ub[0], X0), A0_1 = rowcol(X.ub[1], X0);
        if constexpr (CM != CM_FMA) {
          const cx<float> Aa0[K] = {A0_0, A1_0};
          const cx<float> Aa1[K] = {A0_1, A1_1};
          if constexpr (MMA) {
            acc += R(2) * (cmma.sum(Aa0) + cmma.sum(Aa1));  // x2 helicity flip
          } else {
            sink->put(Aa0);
            sink->put(Aa1);
          }
        } else {
          cc0_0 = fmadd(A0_0.r, A0_0.r, fmadd(A0_0.i, A0_0.i, cc0_0));
          cc1_0 = fmadd(A0_0.r, A1_0.r, fmadd(A0_0.i, A1_0.i, cc1_0));
          cc0_0 = fmadd(A1_0.r, A1_0.r, fmadd(A1_0.i, A1_0.i, cc0_0));
          cc0_1 = fmadd(A0_1.r, A0_1.r, fmadd(A0_1.i, A0_1.i, cc0_1));
          cc1_1 = fmadd(A0_1.r, A1_1.r, fmadd(A0_1.i, A1_1.i, cc1_1));
          cc0_1 = fmadd(A1_1.r, A1_1.r, fmadd(A1_1.i, A1_1.i, cc0_1));
        }
      }
    }
  }
  if constexpr (CM == CM_FMA) acc = R(2) * (R(16) * (cc0_0 + cc0_1) + R(-4) * (cc1_0 + cc1_1));  // x2 helicity flip
  return acc;
}

// floating-point operations of one full helicity sum (all levels, all loop trips)
constexpr long FLOPS_HEL_SUM = 2355;
}}  // namespace
