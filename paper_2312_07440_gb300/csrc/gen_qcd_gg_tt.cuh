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
        const sp<R> S_E = h2 ? X.v[1] : X.v[0];
        sp<R> tS_0 = slash(E0, S_E);
        const sp<R> S_0 = fprop(Kn.qc[1], Kn.mc[1], tS_0);
        sp<R> X1 = slash(E1, S_0);
        slash_acc(X1, J1_0, S_E);
        const cx<R> A1_0 = rowcol(X.ub[0], X1), A1_1 = rowcol(X.ub[1], X1);
        sp<R> tS_1 = slash(E1, S_E);
        const sp<R> S_1 = fprop(Kn.qc[2], Kn.mc[2], tS_1);
        sp<R> X0 = slash(E0, S_1);
        slash_acc(X0, J0_1, S_E);
        const cx<R> A0_0 = rowcol(X.ub[0], X0), A0_1 = rowcol(X.ub[1], X0);
        if constexpr (CM != CM_FMA) {
          const cx<float> Aa0[K] = {A0_0, A1_0};
          const cx<float> Aa1[K] = {A0_1, A1_1};
          acc += R(2) * (cmma.sum(Aa0) + cmma.sum(Aa1));  // x2 helicity flip
        } else {
          R cs = R(0);
          { const R zr = R(16) * R(0.5) * A0_0.r + R(-2) * A1_0.r; const R zi = R(16) * R(0.5) * A0_0.i + R(-2) * A1_0.i;
            cs += A0_0.r * zr + A0_0.i * zi; }
          { const R zr = R(16) * R(0.5) * A1_0.r; const R zi = R(16) * R(0.5) * A1_0.i;
            cs += A1_0.r * zr + A1_0.i * zi; }
          { const R zr = R(16) * R(0.5) * A0_1.r + R(-2) * A1_1.r; const R zi = R(16) * R(0.5) * A0_1.i + R(-2) * A1_1.i;
            cs += A0_1.r * zr + A0_1.i * zi; }
          { const R zr = R(16) * R(0.5) * A1_1.r; const R zi = R(16) * R(0.5) * A1_1.i;
            cs += A1_1.r * zr + A1_1.i * zi; }
          acc += R(4) * cs;  // x2 symmetric colour sum, x2 helicity flip
        }
      }
    }
  }
  return acc;
}

// floating-point operations of one full helicity sum (all levels, all loop trips)
constexpr long FLOPS_HEL_SUM = 3016;
}}  // namespace
