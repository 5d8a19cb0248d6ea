// ---- generated by gen/qcd_gen.py: gg_ttgg (g g -> t tbar + 2 g), do not edit ----
// 123 Feynman diagrams, 24 colour orderings, 64 helicities.
// colour matrix C = Cint / 54
#pragma once
#include "colour_mma.cuh"
#include "qcd.cuh"

namespace rw { namespace gg_ttgg {
constexpr int NG = 4;
constexpr int NEXT = 6;
constexpr int K = 24;
constexpr int NHEL = 64;
constexpr int NDIAG = 123;
constexpr int MAX_LB = 5;  // helicity levels that can be spread over lanes
constexpr int CDEN = 54;
constexpr int IDENT = 2;  // identical outgoing gluons (1/IDENT!)
constexpr unsigned OUTGOING_GLUONS = 12u;  // bit g: gluon g outgoing
__host__ __device__ constexpr int cint(int i, int j) { constexpr int c[K * K] = {512, -64, -64, 8, 8, 80, -64, 8, 8, -1, -1, -10, 8, -1, 80, -10, 71, 62, -1, -10, -10, 62, 62, -28, -64, 512, 8, 80, -64, 8, 8, -64, -1, -10, 8, -1, -1, -10, -10, 62, 62, -28, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, 80, -10, 71, 62, -64, 8, 8, -1, -1, -10, -10, -1, 62, -28, -10, 62, 8, 80, -64, 512, 8, -64, -1, -10, -10, 62, 62, -28, 8, -64, -1, -10, 8, -1, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, -1, 8, 71, 62, 80, -10, -10, -1, 62, -28, -10, 62, -64, 8, 8, -1, -1, -10, 80, 8, 8, -64, -64, 512, -10, -1, 62, -28, -10, 62, -1, 8, 71, 62, 80, -10, 8, -64, -1, -10, 8, -1, -64, 8, 8, -1, -1, -10, 512, -64, -64, 8, 8, 80, 80, -10, 8, -1, 62, 71, -10, 62, -1, -10, -28, 62, 8, -64, -1, -10, 8, -1, -64, 512, 8, 80, -64, 8, -10, 62, -1, -10, -28, 62, 80, -10, 8, -1, 62, 71, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, -64, 8, -10, -1, 62, -28, -10, -1, 62, -10, -1, -10, -10, 62, 62, -28, 8, 80, -64, 512, 8, -64, -1, -10, 8, -64, -1, 8, 71, 62, -1, 8, -10, 80, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, 62, -28, -10, -1, 62, -10, 8, -1, -64, 8, -10, -1, -10, -1, 62, -28, -10, 62, 80, 8, 8, -64, -64, 512, 71, 62, -1, 8, -10, 80, -1, -10, 8, -64, -1, 8, 8, -1, -64, 8, -10, -1, 80, -10, 8, -1, 62, 71, 512, -64, -64, 8, 8, 80, 62, -10, -28, 62, -1, -10, -1, -10, 8, -64, -1, 8, -10, 62, -1, -10, -28, 62, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, 80, -10, 8, -1, 62, 71, 8, -1, -64, 8, -10, -1, -64, 8, 512, -64, 80, 8, -28, 62, 62, -10, -10, -1, -10, 62, -1, -10, -28, 62, -1, -10, 8, -64, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, 71, 62, -1, 8, -10, 80, 62, -28, -10, -1, 62, -10, 8, -64, 80, 8, 512, -64, -1, 8, -10, -1, -64, 8, 62, -28, -10, -1, 62, -10, 71, 62, -1, 8, -10, 80, 80, 8, 8, -64, -64, 512, -10, -1, -1, 8, 8, -64, -1, 8, -10, -1, -64, 8, -10, 80, 62, 71, 8, -1, 62, -10, -28, 62, -1, -10, 512, -64, -64, 8, 8, 80, -10, -1, -1, 8, 8, -64, 62, -10, -28, 62, -1, -10, -10, 80, 62, 71, 8, -1, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, -1, 8, -10, -1, -64, 8, -28, 62, 62, -10, -10, -1, -64, 8, 512, -64, 80, 8, 62, -10, -28, 62, -1, -10, -10, -1, -1, 8, 8, -64, 62, 71, -10, 80, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, -28, 62, 62, -10, -10, -1, -1, 8, -10, -1, -64, 8, 8, -64, 80, 8, 512, -64, -28, 62, 62, -10, -10, -1, 62, 71, -10, 80, -1, 8, -10, -1, -1, 8, 8, -64, 80, 8, 8, -64, -64, 512}; return c[i * K + j]; }
constexpr int ORDER[K][NG] = {{0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 1, 3}, {0, 2, 3, 1}, {0, 3, 1, 2}, {0, 3, 2, 1}, {1, 0, 2, 3}, {1, 0, 3, 2}, {1, 2, 0, 3}, {1, 2, 3, 0}, {1, 3, 0, 2}, {1, 3, 2, 0}, {2, 0, 1, 3}, {2, 0, 3, 1}, {2, 1, 0, 3}, {2, 1, 3, 0}, {2, 3, 0, 1}, {2, 3, 1, 0}, {3, 0, 1, 2}, {3, 0, 2, 1}, {3, 1, 0, 2}, {3, 1, 2, 0}, {3, 2, 0, 1}, {3, 2, 1, 0}};
static __device__ const short CI[K * K] = {512, -64, -64, 8, 8, 80, -64, 8, 8, -1, -1, -10, 8, -1, 80, -10, 71, 62, -1, -10, -10, 62, 62, -28, -64, 512, 8, 80, -64, 8, 8, -64, -1, -10, 8, -1, -1, -10, -10, 62, 62, -28, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, 80, -10, 71, 62, -64, 8, 8, -1, -1, -10, -10, -1, 62, -28, -10, 62, 8, 80, -64, 512, 8, -64, -1, -10, -10, 62, 62, -28, 8, -64, -1, -10, 8, -1, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, -1, 8, 71, 62, 80, -10, -10, -1, 62, -28, -10, 62, -64, 8, 8, -1, -1, -10, 80, 8, 8, -64, -64, 512, -10, -1, 62, -28, -10, 62, -1, 8, 71, 62, 80, -10, 8, -64, -1, -10, 8, -1, -64, 8, 8, -1, -1, -10, 512, -64, -64, 8, 8, 80, 80, -10, 8, -1, 62, 71, -10, 62, -1, -10, -28, 62, 8, -64, -1, -10, 8, -1, -64, 512, 8, 80, -64, 8, -10, 62, -1, -10, -28, 62, 80, -10, 8, -1, 62, 71, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, -64, 8, -10, -1, 62, -28, -10, -1, 62, -10, -1, -10, -10, 62, 62, -28, 8, 80, -64, 512, 8, -64, -1, -10, 8, -64, -1, 8, 71, 62, -1, 8, -10, 80, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, 62, -28, -10, -1, 62, -10, 8, -1, -64, 8, -10, -1, -10, -1, 62, -28, -10, 62, 80, 8, 8, -64, -64, 512, 71, 62, -1, 8, -10, 80, -1, -10, 8, -64, -1, 8, 8, -1, -64, 8, -10, -1, 80, -10, 8, -1, 62, 71, 512, -64, -64, 8, 8, 80, 62, -10, -28, 62, -1, -10, -1, -10, 8, -64, -1, 8, -10, 62, -1, -10, -28, 62, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, 80, -10, 8, -1, 62, 71, 8, -1, -64, 8, -10, -1, -64, 8, 512, -64, 80, 8, -28, 62, 62, -10, -10, -1, -10, 62, -1, -10, -28, 62, -1, -10, 8, -64, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, 71, 62, -1, 8, -10, 80, 62, -28, -10, -1, 62, -10, 8, -64, 80, 8, 512, -64, -1, 8, -10, -1, -64, 8, 62, -28, -10, -1, 62, -10, 71, 62, -1, 8, -10, 80, 80, 8, 8, -64, -64, 512, -10, -1, -1, 8, 8, -64, -1, 8, -10, -1, -64, 8, -10, 80, 62, 71, 8, -1, 62, -10, -28, 62, -1, -10, 512, -64, -64, 8, 8, 80, -10, -1, -1, 8, 8, -64, 62, -10, -28, 62, -1, -10, -10, 80, 62, 71, 8, -1, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, -1, 8, -10, -1, -64, 8, -28, 62, 62, -10, -10, -1, -64, 8, 512, -64, 80, 8, 62, -10, -28, 62, -1, -10, -10, -1, -1, 8, 8, -64, 62, 71, -10, 80, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, -28, 62, 62, -10, -10, -1, -1, 8, -10, -1, -64, 8, 8, -64, 80, 8, 512, -64, -28, 62, 62, -10, -10, -1, 62, 71, -10, 80, -1, 8, -10, -1, -1, 8, 8, -64, 80, 8, 8, -64, -64, 512};  // row-major C_int for the tensor-core sum

// Sum over this lane's helicities of sum_{s,t} Cint_st Re(A_s^* A_t), g = 1;
// helicities with gluon 0 at +1 only, doubled (J^dagger C J(h) = J^dagger C J(-h)).
// CM: colour sum by FMA (CM_FMA, any R) or on the tensor cores (CM_FP16/CM_BF16, R = float).
template <class R, int LB, int CM = CM_FMA>
__device__ __forceinline__ R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& Kn, int lane) {
  static_assert(CM == CM_FMA || sizeof(R) == 4, "tensor-core colour sum takes FP32 amplitudes");
  const ColourMma<K, CM == CM_FMA ? CM_FP16 : CM> cmma(CM == CM_FMA ? nullptr : CI);
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
        cv<R> J0_2_1 = vvv(E0, Kn.P[1], J2_1, Kn.P[6], Kn.cg[7]);
        vvv_acc(J0_2_1, J0_2, Kn.P[5], E1, Kn.P[2], Kn.cg[7]);
        vvvv_acc(J0_2_1, E0, E2, E1, Kn.c4[7]);
        cv<R> J1_0_2 = vvv(E1, Kn.P[2], J0_2, Kn.P[5], Kn.cg[7]);
        vvv_acc(J1_0_2, J1_0, Kn.P[3], E2, Kn.P[4], Kn.cg[7]);
        vvvv_acc(J1_0_2, E1, E0, E2, Kn.c4[7]);
        const cv<R> J1_2_0 = J0_2_1;
        const cv<R> J2_0_1 = J1_0_2;
        const cv<R> J2_1_0 = J0_1_2;
        #pragma unroll 1
        for (int i3 = 0; i3 < (LB >= 3 ? 1 : 2); ++i3) {
          const int h3 = LB >= 3 ? ((lane >> (LB - 3)) & 1) : i3;
          const cv<R> E3 = h3 ? X.eps[3][1] : X.eps[3][0];
          cv<R> J0_3 = vvv(E0, Kn.P[1], E3, Kn.P[8], Kn.cg[9]);
          cv<R> J1_3 = vvv(E1, Kn.P[2], E3, Kn.P[8], Kn.cg[10]);
          cv<R> J2_3 = vvv(E2, Kn.P[4], E3, Kn.P[8], Kn.cg[12]);
          const cv<R> J3_0 = neg(J0_3);
          const cv<R> J3_1 = neg(J1_3);
          const cv<R> J3_2 = neg(J2_3);
          cv<R> J0_1_3 = vvv(E0, Kn.P[1], J1_3, Kn.P[10], Kn.cg[11]);
          vvv_acc(J0_1_3, J0_1, Kn.P[3], E3, Kn.P[8], Kn.cg[11]);
          vvvv_acc(J0_1_3, E0, E1, E3, Kn.c4[11]);
          cv<R> J0_2_3 = vvv(E0, Kn.P[1], J2_3, Kn.P[12], Kn.cg[13]);
          vvv_acc(J0_2_3, J0_2, Kn.P[5], E3, Kn.P[8], Kn.cg[13]);
          vvvv_acc(J0_2_3, E0, E2, E3, Kn.c4[13]);
          cv<R> J0_3_1 = vvv(E0, Kn.P[1], J3_1, Kn.P[10], Kn.cg[11]);
          vvv_acc(J0_3_1, J0_3, Kn.P[9], E1, Kn.P[2], Kn.cg[11]);
          vvvv_acc(J0_3_1, E0, E3, E1, Kn.c4[11]);
          cv<R> J0_3_2 = vvv(E0, Kn.P[1], J3_2, Kn.P[12], Kn.cg[13]);
          vvv_acc(J0_3_2, J0_3, Kn.P[9], E2, Kn.P[4], Kn.cg[13]);
          vvvv_acc(J0_3_2, E0, E3, E2, Kn.c4[13]);
          cv<R> J1_0_3 = vvv(E1, Kn.P[2], J0_3, Kn.P[9], Kn.cg[11]);
          vvv_acc(J1_0_3, J1_0, Kn.P[3], E3, Kn.P[8], Kn.cg[11]);
          vvvv_acc(J1_0_3, E1, E0, E3, Kn.c4[11]);
          cv<R> J1_2_3 = vvv(E1, Kn.P[2], J2_3, Kn.P[12], Kn.cg[14]);
          vvv_acc(J1_2_3, J1_2, Kn.P[6], E3, Kn.P[8], Kn.cg[14]);
          vvvv_acc(J1_2_3, E1, E2, E3, Kn.c4[14]);
          const cv<R> J1_3_0 = J0_3_1;
          cv<R> J1_3_2 = vvv(E1, Kn.P[2], J3_2, Kn.P[12], Kn.cg[14]);
          vvv_acc(J1_3_2, J1_3, Kn.P[10], E2, Kn.P[4], Kn.cg[14]);
          vvvv_acc(J1_3_2, E1, E3, E2, Kn.c4[14]);
          cv<R> J2_0_3 = vvv(E2, Kn.P[4], J0_3, Kn.P[9], Kn.cg[13]);
          vvv_acc(J2_0_3, J2_0, Kn.P[5], E3, Kn.P[8], Kn.cg[13]);
          vvvv_acc(J2_0_3, E2, E0, E3, Kn.c4[13]);
          cv<R> J2_1_3 = vvv(E2, Kn.P[4], J1_3, Kn.P[10], Kn.cg[14]);
          vvv_acc(J2_1_3, J2_1, Kn.P[6], E3, Kn.P[8], Kn.cg[14]);
          vvvv_acc(J2_1_3, E2, E1, E3, Kn.c4[14]);
          const cv<R> J2_3_0 = J0_3_2;
          const cv<R> J2_3_1 = J1_3_2;
          const cv<R> J3_0_1 = J1_0_3;
          const cv<R> J3_0_2 = J2_0_3;
          const cv<R> J3_1_0 = J0_1_3;
          const cv<R> J3_1_2 = J2_1_3;
          const cv<R> J3_2_0 = J0_2_3;
          const cv<R> J3_2_1 = J1_2_3;
          cv<R> J0_1_2_3 = vvv(E0, Kn.P[1], J1_2_3, Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_1_2_3, J0_1, Kn.P[3], J2_3, Kn.P[12], Kn.cg[15]);
          vvv_acc(J0_1_2_3, J0_1_2, Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J0_1_2_3, E0, E1, J2_3, Kn.c4[15]);
          vvvv_acc(J0_1_2_3, E0, J1_2, E3, Kn.c4[15]);
          vvvv_acc(J0_1_2_3, J0_1, E2, E3, Kn.c4[15]);
          cv<R> J0_1_3_2 = vvv(E0, Kn.P[1], J1_3_2, Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_1_3_2, J0_1, Kn.P[3], J3_2, Kn.P[12], Kn.cg[15]);
          vvv_acc(J0_1_3_2, J0_1_3, Kn.P[11], E2, Kn.P[4], Kn.cg[15]);
          vvvv_acc(J0_1_3_2, E0, E1, J3_2, Kn.c4[15]);
          vvvv_acc(J0_1_3_2, E0, J1_3, E2, Kn.c4[15]);
          vvvv_acc(J0_1_3_2, J0_1, E3, E2, Kn.c4[15]);
          cv<R> J0_2_1_3 = vvv(E0, Kn.P[1], J2_1_3, Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_2_1_3, J0_2, Kn.P[5], J1_3, Kn.P[10], Kn.cg[15]);
          vvv_acc(J0_2_1_3, J0_2_1, Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J0_2_1_3, E0, E2, J1_3, Kn.c4[15]);
          vvvv_acc(J0_2_1_3, E0, J2_1, E3, Kn.c4[15]);
          vvvv_acc(J0_2_1_3, J0_2, E1, E3, Kn.c4[15]);
          cv<R> J0_2_3_1 = vvv(E0, Kn.P[1], J2_3_1, Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_2_3_1, J0_2, Kn.P[5], J3_1, Kn.P[10], Kn.cg[15]);
          vvv_acc(J0_2_3_1, J0_2_3, Kn.P[13], E1, Kn.P[2], Kn.cg[15]);
          vvvv_acc(J0_2_3_1, E0, E2, J3_1, Kn.c4[15]);
          vvvv_acc(J0_2_3_1, E0, J2_3, E1, Kn.c4[15]);
          vvvv_acc(J0_2_3_1, J0_2, E3, E1, Kn.c4[15]);
          cv<R> J0_3_1_2 = vvv(E0, Kn.P[1], J3_1_2, Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_3_1_2, J0_3, Kn.P[9], J1_2, Kn.P[6], Kn.cg[15]);
          vvv_acc(J0_3_1_2, J0_3_1, Kn.P[11], E2, Kn.P[4], Kn.cg[15]);
          vvvv_acc(J0_3_1_2, E0, E3, J1_2, Kn.c4[15]);
          vvvv_acc(J0_3_1_2, E0, J3_1, E2, Kn.c4[15]);
          vvvv_acc(J0_3_1_2, J0_3, E1, E2, Kn.c4[15]);
          cv<R> J0_3_2_1 = vvv(E0, Kn.P[1], J3_2_1, Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_3_2_1, J0_3, Kn.P[9], J2_1, Kn.P[6], Kn.cg[15]);
          vvv_acc(J0_3_2_1, J0_3_2, Kn.P[13], E1, Kn.P[2], Kn.cg[15]);
          vvvv_acc(J0_3_2_1, E0, E3, J2_1, Kn.c4[15]);
          vvvv_acc(J0_3_2_1, E0, J3_2, E1, Kn.c4[15]);
          vvvv_acc(J0_3_2_1, J0_3, E2, E1, Kn.c4[15]);
          cv<R> J1_0_2_3 = vvv(E1, Kn.P[2], J0_2_3, Kn.P[13], Kn.cg[15]);
          vvv_acc(J1_0_2_3, J1_0, Kn.P[3], J2_3, Kn.P[12], Kn.cg[15]);
          vvv_acc(J1_0_2_3, J1_0_2, Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J1_0_2_3, E1, E0, J2_3, Kn.c4[15]);
          vvvv_acc(J1_0_2_3, E1, J0_2, E3, Kn.c4[15]);
          vvvv_acc(J1_0_2_3, J1_0, E2, E3, Kn.c4[15]);
          cv<R> J1_0_3_2 = vvv(E1, Kn.P[2], J0_3_2, Kn.P[13], Kn.cg[15]);
          vvv_acc(J1_0_3_2, J1_0, Kn.P[3], J3_2, Kn.P[12], Kn.cg[15]);
          vvv_acc(J1_0_3_2, J1_0_3, Kn.P[11], E2, Kn.P[4], Kn.cg[15]);
          vvvv_acc(J1_0_3_2, E1, E0, J3_2, Kn.c4[15]);
          vvvv_acc(J1_0_3_2, E1, J0_3, E2, Kn.c4[15]);
          vvvv_acc(J1_0_3_2, J1_0, E3, E2, Kn.c4[15]);
          cv<R> J1_2_0_3 = vvv(E1, Kn.P[2], J2_0_3, Kn.P[13], Kn.cg[15]);
          vvv_acc(J1_2_0_3, J1_2, Kn.P[6], J0_3, Kn.P[9], Kn.cg[15]);
          vvv_acc(J1_2_0_3, J1_2_0, Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J1_2_0_3, E1, E2, J0_3, Kn.c4[15]);
          vvvv_acc(J1_2_0_3, E1, J2_0, E3, Kn.c4[15]);
          vvvv_acc(J1_2_0_3, J1_2, E0, E3, Kn.c4[15]);
          const cv<R> J1_2_3_0 = neg(J0_3_2_1);
          cv<R> J1_3_0_2 = vvv(E1, Kn.P[2], J3_0_2, Kn.P[13], Kn.cg[15]);
          vvv_acc(J1_3_0_2, J1_3, Kn.P[10], J0_2, Kn.P[5], Kn.cg[15]);
          vvv_acc(J1_3_0_2, J1_3_0, Kn.P[11], E2, Kn.P[4], Kn.cg[15]);
          vvvv_acc(J1_3_0_2, E1, E3, J0_2, Kn.c4[15]);
          vvvv_acc(J1_3_0_2, E1, J3_0, E2, Kn.c4[15]);
          vvvv_acc(J1_3_0_2, J1_3, E0, E2, Kn.c4[15]);
          const cv<R> J1_3_2_0 = neg(J0_2_3_1);
          cv<R> J2_0_1_3 = vvv(E2, Kn.P[4], J0_1_3, Kn.P[11], Kn.cg[15]);
          vvv_acc(J2_0_1_3, J2_0, Kn.P[5], J1_3, Kn.P[10], Kn.cg[15]);
          vvv_acc(J2_0_1_3, J2_0_1, Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J2_0_1_3, E2, E0, J1_3, Kn.c4[15]);
          vvvv_acc(J2_0_1_3, E2, J0_1, E3, Kn.c4[15]);
          vvvv_acc(J2_0_1_3, J2_0, E1, E3, Kn.c4[15]);
          const cv<R> J2_0_3_1 = neg(J1_3_0_2);
          cv<R> J2_1_0_3 = vvv(E2, Kn.P[4], J1_0_3, Kn.P[11], Kn.cg[15]);
          vvv_acc(J2_1_0_3, J2_1, Kn.P[6], J0_3, Kn.P[9], Kn.cg[15]);
          vvv_acc(J2_1_0_3, J2_1_0, Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J2_1_0_3, E2, E1, J0_3, Kn.c4[15]);
          vvvv_acc(J2_1_0_3, E2, J1_0, E3, Kn.c4[15]);
          vvvv_acc(J2_1_0_3, J2_1, E0, E3, Kn.c4[15]);
          const cv<R> J2_1_3_0 = neg(J0_3_1_2);
          const cv<R> J2_3_0_1 = neg(J1_0_3_2);
          const cv<R> J2_3_1_0 = neg(J0_1_3_2);
          const cv<R> J3_0_1_2 = neg(J2_1_0_3);
          const cv<R> J3_0_2_1 = neg(J1_2_0_3);
          const cv<R> J3_1_0_2 = neg(J2_0_1_3);
          const cv<R> J3_1_2_0 = neg(J0_2_1_3);
          const cv<R> J3_2_0_1 = neg(J1_0_2_3);
          const cv<R> J3_2_1_0 = neg(J0_1_2_3);
          #pragma unroll 1
          for (int i4 = 0; i4 < (LB >= 4 ? 1 : 2); ++i4) {
            const int h4 = LB >= 4 ? ((lane >> (LB - 4)) & 1) : i4;
            const sp<R> S_E = h4 ? X.v[1] : X.v[0];
            sp<R> tS_0 = slash(E0, S_E);
            const sp<R> S_0 = fprop(Kn.qc[1], Kn.mc[1], tS_0);
            sp<R> tS_1 = slash(E1, S_E);
            const sp<R> S_1 = fprop(Kn.qc[2], Kn.mc[2], tS_1);
            sp<R> tS_2 = slash(E2, S_E);
            const sp<R> S_2 = fprop(Kn.qc[4], Kn.mc[4], tS_2);
            sp<R> tS_3 = slash(E3, S_E);
            const sp<R> S_3 = fprop(Kn.qc[8], Kn.mc[8], tS_3);
            sp<R> tS_0_1 = slash(E0, S_1);
            slash_acc(tS_0_1, J0_1, S_E);
            const sp<R> S_0_1 = fprop(Kn.qc[3], Kn.mc[3], tS_0_1);
            sp<R> tS_0_2 = slash(E0, S_2);
            slash_acc(tS_0_2, J0_2, S_E);
            const sp<R> S_0_2 = fprop(Kn.qc[5], Kn.mc[5], tS_0_2);
            sp<R> tS_0_3 = slash(E0, S_3);
            slash_acc(tS_0_3, J0_3, S_E);
            const sp<R> S_0_3 = fprop(Kn.qc[9], Kn.mc[9], tS_0_3);
            sp<R> tS_1_0 = slash(E1, S_0);
            slash_acc(tS_1_0, J1_0, S_E);
            const sp<R> S_1_0 = fprop(Kn.qc[3], Kn.mc[3], tS_1_0);
            sp<R> tS_1_2 = slash(E1, S_2);
            slash_acc(tS_1_2, J1_2, S_E);
            const sp<R> S_1_2 = fprop(Kn.qc[6], Kn.mc[6], tS_1_2);
            sp<R> tS_1_3 = slash(E1, S_3);
            slash_acc(tS_1_3, J1_3, S_E);
            const sp<R> S_1_3 = fprop(Kn.qc[10], Kn.mc[10], tS_1_3);
            sp<R> tS_2_0 = slash(E2, S_0);
            slash_acc(tS_2_0, J2_0, S_E);
            const sp<R> S_2_0 = fprop(Kn.qc[5], Kn.mc[5], tS_2_0);
            sp<R> tS_2_1 = slash(E2, S_1);
            slash_acc(tS_2_1, J2_1, S_E);
            const sp<R> S_2_1 = fprop(Kn.qc[6], Kn.mc[6], tS_2_1);
            sp<R> tS_2_3 = slash(E2, S_3);
            slash_acc(tS_2_3, J2_3, S_E);
            const sp<R> S_2_3 = fprop(Kn.qc[12], Kn.mc[12], tS_2_3);
            sp<R> tS_3_0 = slash(E3, S_0);
            slash_acc(tS_3_0, J3_0, S_E);
            const sp<R> S_3_0 = fprop(Kn.qc[9], Kn.mc[9], tS_3_0);
            sp<R> tS_3_1 = slash(E3, S_1);
            slash_acc(tS_3_1, J3_1, S_E);
            const sp<R> S_3_1 = fprop(Kn.qc[10], Kn.mc[10], tS_3_1);
            sp<R> tS_3_2 = slash(E3, S_2);
            slash_acc(tS_3_2, J3_2, S_E);
            const sp<R> S_3_2 = fprop(Kn.qc[12], Kn.mc[12], tS_3_2);
            sp<R> tS_0_1_2 = slash(E0, S_1_2);
            slash_acc(tS_0_1_2, J0_1, S_2);
            slash_acc(tS_0_1_2, J0_1_2, S_E);
            const sp<R> S_0_1_2 = fprop(Kn.qc[7], Kn.mc[7], tS_0_1_2);
            sp<R> tS_0_1_3 = slash(E0, S_1_3);
            slash_acc(tS_0_1_3, J0_1, S_3);
            slash_acc(tS_0_1_3, J0_1_3, S_E);
            const sp<R> S_0_1_3 = fprop(Kn.qc[11], Kn.mc[11], tS_0_1_3);
            sp<R> tS_0_2_1 = slash(E0, S_2_1);
            slash_acc(tS_0_2_1, J0_2, S_1);
            slash_acc(tS_0_2_1, J0_2_1, S_E);
            const sp<R> S_0_2_1 = fprop(Kn.qc[7], Kn.mc[7], tS_0_2_1);
            sp<R> tS_0_2_3 = slash(E0, S_2_3);
            slash_acc(tS_0_2_3, J0_2, S_3);
            slash_acc(tS_0_2_3, J0_2_3, S_E);
            const sp<R> S_0_2_3 = fprop(Kn.qc[13], Kn.mc[13], tS_0_2_3);
            sp<R> tS_0_3_1 = slash(E0, S_3_1);
            slash_acc(tS_0_3_1, J0_3, S_1);
            slash_acc(tS_0_3_1, J0_3_1, S_E);
            const sp<R> S_0_3_1 = fprop(Kn.qc[11], Kn.mc[11], tS_0_3_1);
            sp<R> tS_0_3_2 = slash(E0, S_3_2);
            slash_acc(tS_0_3_2, J0_3, S_2);
            slash_acc(tS_0_3_2, J0_3_2, S_E);
            const sp<R> S_0_3_2 = fprop(Kn.qc[13], Kn.mc[13], tS_0_3_2);
            sp<R> tS_1_0_2 = slash(E1, S_0_2);
            slash_acc(tS_1_0_2, J1_0, S_2);
            slash_acc(tS_1_0_2, J1_0_2, S_E);
            const sp<R> S_1_0_2 = fprop(Kn.qc[7], Kn.mc[7], tS_1_0_2);
            sp<R> tS_1_0_3 = slash(E1, S_0_3);
            slash_acc(tS_1_0_3, J1_0, S_3);
            slash_acc(tS_1_0_3, J1_0_3, S_E);
            const sp<R> S_1_0_3 = fprop(Kn.qc[11], Kn.mc[11], tS_1_0_3);
            sp<R> tS_1_2_0 = slash(E1, S_2_0);
            slash_acc(tS_1_2_0, J1_2, S_0);
            slash_acc(tS_1_2_0, J1_2_0, S_E);
            const sp<R> S_1_2_0 = fprop(Kn.qc[7], Kn.mc[7], tS_1_2_0);
            sp<R> tS_1_2_3 = slash(E1, S_2_3);
            slash_acc(tS_1_2_3, J1_2, S_3);
            slash_acc(tS_1_2_3, J1_2_3, S_E);
            const sp<R> S_1_2_3 = fprop(Kn.qc[14], Kn.mc[14], tS_1_2_3);
            sp<R> tS_1_3_0 = slash(E1, S_3_0);
            slash_acc(tS_1_3_0, J1_3, S_0);
            slash_acc(tS_1_3_0, J1_3_0, S_E);
            const sp<R> S_1_3_0 = fprop(Kn.qc[11], Kn.mc[11], tS_1_3_0);
            sp<R> tS_1_3_2 = slash(E1, S_3_2);
            slash_acc(tS_1_3_2, J1_3, S_2);
            slash_acc(tS_1_3_2, J1_3_2, S_E);
            const sp<R> S_1_3_2 = fprop(Kn.qc[14], Kn.mc[14], tS_1_3_2);
            sp<R> tS_2_0_1 = slash(E2, S_0_1);
            slash_acc(tS_2_0_1, J2_0, S_1);
            slash_acc(tS_2_0_1, J2_0_1, S_E);
            const sp<R> S_2_0_1 = fprop(Kn.qc[7], Kn.mc[7], tS_2_0_1);
            sp<R> tS_2_0_3 = slash(E2, S_0_3);
            slash_acc(tS_2_0_3, J2_0, S_3);
            slash_acc(tS_2_0_3, J2_0_3, S_E);
            const sp<R> S_2_0_3 = fprop(Kn.qc[13], Kn.mc[13], tS_2_0_3);
            sp<R> tS_2_1_0 = slash(E2, S_1_0);
            slash_acc(tS_2_1_0, J2_1, S_0);
            slash_acc(tS_2_1_0, J2_1_0, S_E);
            const sp<R> S_2_1_0 = fprop(Kn.qc[7], Kn.mc[7], tS_2_1_0);
            sp<R> tS_2_1_3 = slash(E2, S_1_3);
            slash_acc(tS_2_1_3, J2_1, S_3);
            slash_acc(tS_2_1_3, J2_1_3, S_E);
            const sp<R> S_2_1_3 = fprop(Kn.qc[14], Kn.mc[14], tS_2_1_3);
            sp<R> tS_2_3_0 = slash(E2, S_3_0);
            slash_acc(tS_2_3_0, J2_3, S_0);
            slash_acc(tS_2_3_0, J2_3_0, S_E);
            const sp<R> S_2_3_0 = fprop(Kn.qc[13], Kn.mc[13], tS_2_3_0);
            sp<R> tS_2_3_1 = slash(E2, S_3_1);
            slash_acc(tS_2_3_1, J2_3, S_1);
            slash_acc(tS_2_3_1, J2_3_1, S_E);
            const sp<R> S_2_3_1 = fprop(Kn.qc[14], Kn.mc[14], tS_2_3_1);
            sp<R> tS_3_0_1 = slash(E3, S_0_1);
            slash_acc(tS_3_0_1, J3_0, S_1);
            slash_acc(tS_3_0_1, J3_0_1, S_E);
            const sp<R> S_3_0_1 = fprop(Kn.qc[11], Kn.mc[11], tS_3_0_1);
            sp<R> tS_3_0_2 = slash(E3, S_0_2);
            slash_acc(tS_3_0_2, J3_0, S_2);
            slash_acc(tS_3_0_2, J3_0_2, S_E);
            const sp<R> S_3_0_2 = fprop(Kn.qc[13], Kn.mc[13], tS_3_0_2);
            sp<R> tS_3_1_0 = slash(E3, S_1_0);
            slash_acc(tS_3_1_0, J3_1, S_0);
            slash_acc(tS_3_1_0, J3_1_0, S_E);
            const sp<R> S_3_1_0 = fprop(Kn.qc[11], Kn.mc[11], tS_3_1_0);
            sp<R> tS_3_1_2 = slash(E3, S_1_2);
            slash_acc(tS_3_1_2, J3_1, S_2);
            slash_acc(tS_3_1_2, J3_1_2, S_E);
            const sp<R> S_3_1_2 = fprop(Kn.qc[14], Kn.mc[14], tS_3_1_2);
            sp<R> tS_3_2_0 = slash(E3, S_2_0);
            slash_acc(tS_3_2_0, J3_2, S_0);
            slash_acc(tS_3_2_0, J3_2_0, S_E);
            const sp<R> S_3_2_0 = fprop(Kn.qc[13], Kn.mc[13], tS_3_2_0);
            sp<R> tS_3_2_1 = slash(E3, S_2_1);
            slash_acc(tS_3_2_1, J3_2, S_1);
            slash_acc(tS_3_2_1, J3_2_1, S_E);
            const sp<R> S_3_2_1 = fprop(Kn.qc[14], Kn.mc[14], tS_3_2_1);
            sp<R> X0 = slash(E0, S_1_2_3);
            slash_acc(X0, J0_1, S_2_3);
            slash_acc(X0, J0_1_2, S_3);
            slash_acc(X0, J0_1_2_3, S_E);
            sp<R> X1 = slash(E0, S_1_3_2);
            slash_acc(X1, J0_1, S_3_2);
            slash_acc(X1, J0_1_3, S_2);
            slash_acc(X1, J0_1_3_2, S_E);
            sp<R> X2 = slash(E0, S_2_1_3);
            slash_acc(X2, J0_2, S_1_3);
            slash_acc(X2, J0_2_1, S_3);
            slash_acc(X2, J0_2_1_3, S_E);
            sp<R> X3 = slash(E0, S_2_3_1);
            slash_acc(X3, J0_2, S_3_1);
            slash_acc(X3, J0_2_3, S_1);
            slash_acc(X3, J0_2_3_1, S_E);
            sp<R> X4 = slash(E0, S_3_1_2);
            slash_acc(X4, J0_3, S_1_2);
            slash_acc(X4, J0_3_1, S_2);
            slash_acc(X4, J0_3_1_2, S_E);
            sp<R> X5 = slash(E0, S_3_2_1);
            slash_acc(X5, J0_3, S_2_1);
            slash_acc(X5, J0_3_2, S_1);
            slash_acc(X5, J0_3_2_1, S_E);
            sp<R> X6 = slash(E1, S_0_2_3);
            slash_acc(X6, J1_0, S_2_3);
            slash_acc(X6, J1_0_2, S_3);
            slash_acc(X6, J1_0_2_3, S_E);
            sp<R> X7 = slash(E1, S_0_3_2);
            slash_acc(X7, J1_0, S_3_2);
            slash_acc(X7, J1_0_3, S_2);
            slash_acc(X7, J1_0_3_2, S_E);
            sp<R> X8 = slash(E1, S_2_0_3);
            slash_acc(X8, J1_2, S_0_3);
            slash_acc(X8, J1_2_0, S_3);
            slash_acc(X8, J1_2_0_3, S_E);
            sp<R> X9 = slash(E1, S_2_3_0);
            slash_acc(X9, J1_2, S_3_0);
            slash_acc(X9, J1_2_3, S_0);
            slash_acc(X9, J1_2_3_0, S_E);
            sp<R> X10 = slash(E1, S_3_0_2);
            slash_acc(X10, J1_3, S_0_2);
            slash_acc(X10, J1_3_0, S_2);
            slash_acc(X10, J1_3_0_2, S_E);
            sp<R> X11 = slash(E1, S_3_2_0);
            slash_acc(X11, J1_3, S_2_0);
            slash_acc(X11, J1_3_2, S_0);
            slash_acc(X11, J1_3_2_0, S_E);
            sp<R> X12 = slash(E2, S_0_1_3);
            slash_acc(X12, J2_0, S_1_3);
            slash_acc(X12, J2_0_1, S_3);
            slash_acc(X12, J2_0_1_3, S_E);
            sp<R> X13 = slash(E2, S_0_3_1);
            slash_acc(X13, J2_0, S_3_1);
            slash_acc(X13, J2_0_3, S_1);
            slash_acc(X13, J2_0_3_1, S_E);
            sp<R> X14 = slash(E2, S_1_0_3);
            slash_acc(X14, J2_1, S_0_3);
            slash_acc(X14, J2_1_0, S_3);
            slash_acc(X14, J2_1_0_3, S_E);
            sp<R> X15 = slash(E2, S_1_3_0);
            slash_acc(X15, J2_1, S_3_0);
            slash_acc(X15, J2_1_3, S_0);
            slash_acc(X15, J2_1_3_0, S_E);
            sp<R> X16 = slash(E2, S_3_0_1);
            slash_acc(X16, J2_3, S_0_1);
            slash_acc(X16, J2_3_0, S_1);
            slash_acc(X16, J2_3_0_1, S_E);
            sp<R> X17 = slash(E2, S_3_1_0);
            slash_acc(X17, J2_3, S_1_0);
            slash_acc(X17, J2_3_1, S_0);
            slash_acc(X17, J2_3_1_0, S_E);
            sp<R> X18 = slash(E3, S_0_1_2);
            slash_acc(X18, J3_0, S_1_2);
            slash_acc(X18, J3_0_1, S_2);
            slash_acc(X18, J3_0_1_2, S_E);
            sp<R> X19 = slash(E3, S_0_2_1);
            slash_acc(X19, J3_0, S_2_1);
            slash_acc(X19, J3_0_2, S_1);
            slash_acc(X19, J3_0_2_1, S_E);
            sp<R> X20 = slash(E3, S_1_0_2);
            slash_acc(X20, J3_1, S_0_2);
            slash_acc(X20, J3_1_0, S_2);
            slash_acc(X20, J3_1_0_2, S_E);
            sp<R> X21 = slash(E3, S_1_2_0);
            slash_acc(X21, J3_1, S_2_0);
            slash_acc(X21, J3_1_2, S_0);
            slash_acc(X21, J3_1_2_0, S_E);
            sp<R> X22 = slash(E3, S_2_0_1);
            slash_acc(X22, J3_2, S_0_1);
            slash_acc(X22, J3_2_0, S_1);
            slash_acc(X22, J3_2_0_1, S_E);
            sp<R> X23 = slash(E3, S_2_1_0);
            slash_acc(X23, J3_2, S_1_0);
            slash_acc(X23, J3_2_1, S_0);
            slash_acc(X23, J3_2_1_0, S_E);
            #pragma unroll 1
            for (int i5 = 0; i5 < (LB >= 5 ? 1 : 2); ++i5) {
              const int h5 = LB >= 5 ? ((lane >> (LB - 5)) & 1) : i5;
              const sp<R> UB = h5 ? X.ub[1] : X.ub[0];
              const cx<R> A0 = rowcol(UB, X0);
              const cx<R> A1 = rowcol(UB, X1);
              const cx<R> A2 = rowcol(UB, X2);
              const cx<R> A3 = rowcol(UB, X3);
              const cx<R> A4 = rowcol(UB, X4);
              const cx<R> A5 = rowcol(UB, X5);
              const cx<R> A6 = rowcol(UB, X6);
              const cx<R> A7 = rowcol(UB, X7);
              const cx<R> A8 = rowcol(UB, X8);
              const cx<R> A9 = rowcol(UB, X9);
              const cx<R> A10 = rowcol(UB, X10);
              const cx<R> A11 = rowcol(UB, X11);
              const cx<R> A12 = rowcol(UB, X12);
              const cx<R> A13 = rowcol(UB, X13);
              const cx<R> A14 = rowcol(UB, X14);
              const cx<R> A15 = rowcol(UB, X15);
              const cx<R> A16 = rowcol(UB, X16);
              const cx<R> A17 = rowcol(UB, X17);
              const cx<R> A18 = rowcol(UB, X18);
              const cx<R> A19 = rowcol(UB, X19);
              const cx<R> A20 = rowcol(UB, X20);
              const cx<R> A21 = rowcol(UB, X21);
              const cx<R> A22 = rowcol(UB, X22);
              const cx<R> A23 = rowcol(UB, X23);
              if constexpr (CM != CM_FMA) {
                const cx<float> Aa[K] = {A0, A1, A2, A3, A4, A5, A6, A7, A8, A9, A10, A11, A12, A13, A14, A15, A16, A17, A18, A19, A20, A21, A22, A23};
                acc += R(2) * cmma.sum(Aa);  // x2 helicity flip
              } else {
                R cs = R(0);
                { const R zr = R(512) * R(0.5) * A0.r + R(-64) * A1.r + R(-64) * A2.r + R(8) * A3.r + R(8) * A4.r + R(80) * A5.r + R(-64) * A6.r + R(8) * A7.r + R(8) * A8.r + R(-1) * A9.r + R(-1) * A10.r + R(-10) * A11.r + R(8) * A12.r + R(-1) * A13.r + R(80) * A14.r + R(-10) * A15.r + R(71) * A16.r + R(62) * A17.r + R(-1) * A18.r + R(-10) * A19.r + R(-10) * A20.r + R(62) * A21.r + R(62) * A22.r + R(-28) * A23.r; const R zi = R(512) * R(0.5) * A0.i + R(-64) * A1.i + R(-64) * A2.i + R(8) * A3.i + R(8) * A4.i + R(80) * A5.i + R(-64) * A6.i + R(8) * A7.i + R(8) * A8.i + R(-1) * A9.i + R(-1) * A10.i + R(-10) * A11.i + R(8) * A12.i + R(-1) * A13.i + R(80) * A14.i + R(-10) * A15.i + R(71) * A16.i + R(62) * A17.i + R(-1) * A18.i + R(-10) * A19.i + R(-10) * A20.i + R(62) * A21.i + R(62) * A22.i + R(-28) * A23.i;
                  cs += A0.r * zr + A0.i * zi; }
                { const R zr = R(512) * R(0.5) * A1.r + R(8) * A2.r + R(80) * A3.r + R(-64) * A4.r + R(8) * A5.r + R(8) * A6.r + R(-64) * A7.r + R(-1) * A8.r + R(-10) * A9.r + R(8) * A10.r + R(-1) * A11.r + R(-1) * A12.r + R(-10) * A13.r + R(-10) * A14.r + R(62) * A15.r + R(62) * A16.r + R(-28) * A17.r + R(8) * A18.r + R(-1) * A19.r + R(80) * A20.r + R(-10) * A21.r + R(71) * A22.r + R(62) * A23.r; const R zi = R(512) * R(0.5) * A1.i + R(8) * A2.i + R(80) * A3.i + R(-64) * A4.i + R(8) * A5.i + R(8) * A6.i + R(-64) * A7.i + R(-1) * A8.i + R(-10) * A9.i + R(8) * A10.i + R(-1) * A11.i + R(-1) * A12.i + R(-10) * A13.i + R(-10) * A14.i + R(62) * A15.i + R(62) * A16.i + R(-28) * A17.i + R(8) * A18.i + R(-1) * A19.i + R(80) * A20.i + R(-10) * A21.i + R(71) * A22.i + R(62) * A23.i;
                  cs += A1.r * zr + A1.i * zi; }
                { const R zr = R(512) * R(0.5) * A2.r + R(-64) * A3.r + R(80) * A4.r + R(8) * A5.r + R(8) * A6.r + R(-1) * A7.r + R(80) * A8.r + R(-10) * A9.r + R(71) * A10.r + R(62) * A11.r + R(-64) * A12.r + R(8) * A13.r + R(8) * A14.r + R(-1) * A15.r + R(-1) * A16.r + R(-10) * A17.r + R(-10) * A18.r + R(-1) * A19.r + R(62) * A20.r + R(-28) * A21.r + R(-10) * A22.r + R(62) * A23.r; const R zi = R(512) * R(0.5) * A2.i + R(-64) * A3.i + R(80) * A4.i + R(8) * A5.i + R(8) * A6.i + R(-1) * A7.i + R(80) * A8.i + R(-10) * A9.i + R(71) * A10.i + R(62) * A11.i + R(-64) * A12.i + R(8) * A13.i + R(8) * A14.i + R(-1) * A15.i + R(-1) * A16.i + R(-10) * A17.i + R(-10) * A18.i + R(-1) * A19.i + R(62) * A20.i + R(-28) * A21.i + R(-10) * A22.i + R(62) * A23.i;
                  cs += A2.r * zr + A2.i * zi; }
                { const R zr = R(512) * R(0.5) * A3.r + R(8) * A4.r + R(-64) * A5.r + R(-1) * A6.r + R(-10) * A7.r + R(-10) * A8.r + R(62) * A9.r + R(62) * A10.r + R(-28) * A11.r + R(8) * A12.r + R(-64) * A13.r + R(-1) * A14.r + R(-10) * A15.r + R(8) * A16.r + R(-1) * A17.r + R(-1) * A18.r + R(8) * A19.r + R(71) * A20.r + R(62) * A21.r + R(80) * A22.r + R(-10) * A23.r; const R zi = R(512) * R(0.5) * A3.i + R(8) * A4.i + R(-64) * A5.i + R(-1) * A6.i + R(-10) * A7.i + R(-10) * A8.i + R(62) * A9.i + R(62) * A10.i + R(-28) * A11.i + R(8) * A12.i + R(-64) * A13.i + R(-1) * A14.i + R(-10) * A15.i + R(8) * A16.i + R(-1) * A17.i + R(-1) * A18.i + R(8) * A19.i + R(71) * A20.i + R(62) * A21.i + R(80) * A22.i + R(-10) * A23.i;
                  cs += A3.r * zr + A3.i * zi; }
                { const R zr = R(512) * R(0.5) * A4.r + R(-64) * A5.r + R(-1) * A6.r + R(8) * A7.r + R(71) * A8.r + R(62) * A9.r + R(80) * A10.r + R(-10) * A11.r + R(-10) * A12.r + R(-1) * A13.r + R(62) * A14.r + R(-28) * A15.r + R(-10) * A16.r + R(62) * A17.r + R(-64) * A18.r + R(8) * A19.r + R(8) * A20.r + R(-1) * A21.r + R(-1) * A22.r + R(-10) * A23.r; const R zi = R(512) * R(0.5) * A4.i + R(-64) * A5.i + R(-1) * A6.i + R(8) * A7.i + R(71) * A8.i + R(62) * A9.i + R(80) * A10.i + R(-10) * A11.i + R(-10) * A12.i + R(-1) * A13.i + R(62) * A14.i + R(-28) * A15.i + R(-10) * A16.i + R(62) * A17.i + R(-64) * A18.i + R(8) * A19.i + R(8) * A20.i + R(-1) * A21.i + R(-1) * A22.i + R(-10) * A23.i;
                  cs += A4.r * zr + A4.i * zi; }
                { const R zr = R(512) * R(0.5) * A5.r + R(-10) * A6.r + R(-1) * A7.r + R(62) * A8.r + R(-28) * A9.r + R(-10) * A10.r + R(62) * A11.r + R(-1) * A12.r + R(8) * A13.r + R(71) * A14.r + R(62) * A15.r + R(80) * A16.r + R(-10) * A17.r + R(8) * A18.r + R(-64) * A19.r + R(-1) * A20.r + R(-10) * A21.r + R(8) * A22.r + R(-1) * A23.r; const R zi = R(512) * R(0.5) * A5.i + R(-10) * A6.i + R(-1) * A7.i + R(62) * A8.i + R(-28) * A9.i + R(-10) * A10.i + R(62) * A11.i + R(-1) * A12.i + R(8) * A13.i + R(71) * A14.i + R(62) * A15.i + R(80) * A16.i + R(-10) * A17.i + R(8) * A18.i + R(-64) * A19.i + R(-1) * A20.i + R(-10) * A21.i + R(8) * A22.i + R(-1) * A23.i;
                  cs += A5.r * zr + A5.i * zi; }
                { const R zr = R(512) * R(0.5) * A6.r + R(-64) * A7.r + R(-64) * A8.r + R(8) * A9.r + R(8) * A10.r + R(80) * A11.r + R(80) * A12.r + R(-10) * A13.r + R(8) * A14.r + R(-1) * A15.r + R(62) * A16.r + R(71) * A17.r + R(-10) * A18.r + R(62) * A19.r + R(-1) * A20.r + R(-10) * A21.r + R(-28) * A22.r + R(62) * A23.r; const R zi = R(512) * R(0.5) * A6.i + R(-64) * A7.i + R(-64) * A8.i + R(8) * A9.i + R(8) * A10.i + R(80) * A11.i + R(80) * A12.i + R(-10) * A13.i + R(8) * A14.i + R(-1) * A15.i + R(62) * A16.i + R(71) * A17.i + R(-10) * A18.i + R(62) * A19.i + R(-1) * A20.i + R(-10) * A21.i + R(-28) * A22.i + R(62) * A23.i;
                  cs += A6.r * zr + A6.i * zi; }
                { const R zr = R(512) * R(0.5) * A7.r + R(8) * A8.r + R(80) * A9.r + R(-64) * A10.r + R(8) * A11.r + R(-10) * A12.r + R(62) * A13.r + R(-1) * A14.r + R(-10) * A15.r + R(-28) * A16.r + R(62) * A17.r + R(80) * A18.r + R(-10) * A19.r + R(8) * A20.r + R(-1) * A21.r + R(62) * A22.r + R(71) * A23.r; const R zi = R(512) * R(0.5) * A7.i + R(8) * A8.i + R(80) * A9.i + R(-64) * A10.i + R(8) * A11.i + R(-10) * A12.i + R(62) * A13.i + R(-1) * A14.i + R(-10) * A15.i + R(-28) * A16.i + R(62) * A17.i + R(80) * A18.i + R(-10) * A19.i + R(8) * A20.i + R(-1) * A21.i + R(62) * A22.i + R(71) * A23.i;
                  cs += A7.r * zr + A7.i * zi; }
                { const R zr = R(512) * R(0.5) * A8.r + R(-64) * A9.r + R(80) * A10.r + R(8) * A11.r + R(8) * A12.r + R(-1) * A13.r + R(-64) * A14.r + R(8) * A15.r + R(-10) * A16.r + R(-1) * A17.r + R(62) * A18.r + R(-28) * A19.r + R(-10) * A20.r + R(-1) * A21.r + R(62) * A22.r + R(-10) * A23.r; const R zi = R(512) * R(0.5) * A8.i + R(-64) * A9.i + R(80) * A10.i + R(8) * A11.i + R(8) * A12.i + R(-1) * A13.i + R(-64) * A14.i + R(8) * A15.i + R(-10) * A16.i + R(-1) * A17.i + R(62) * A18.i + R(-28) * A19.i + R(-10) * A20.i + R(-1) * A21.i + R(62) * A22.i + R(-10) * A23.i;
                  cs += A8.r * zr + A8.i * zi; }
                { const R zr = R(512) * R(0.5) * A9.r + R(8) * A10.r + R(-64) * A11.r + R(-1) * A12.r + R(-10) * A13.r + R(8) * A14.r + R(-64) * A15.r + R(-1) * A16.r + R(8) * A17.r + R(71) * A18.r + R(62) * A19.r + R(-1) * A20.r + R(8) * A21.r + R(-10) * A22.r + R(80) * A23.r; const R zi = R(512) * R(0.5) * A9.i + R(8) * A10.i + R(-64) * A11.i + R(-1) * A12.i + R(-10) * A13.i + R(8) * A14.i + R(-64) * A15.i + R(-1) * A16.i + R(8) * A17.i + R(71) * A18.i + R(62) * A19.i + R(-1) * A20.i + R(8) * A21.i + R(-10) * A22.i + R(80) * A23.i;
                  cs += A9.r * zr + A9.i * zi; }
                { const R zr = R(512) * R(0.5) * A10.r + R(-64) * A11.r + R(62) * A12.r + R(-28) * A13.r + R(-10) * A14.r + R(-1) * A15.r + R(62) * A16.r + R(-10) * A17.r + R(8) * A18.r + R(-1) * A19.r + R(-64) * A20.r + R(8) * A21.r + R(-10) * A22.r + R(-1) * A23.r; const R zi = R(512) * R(0.5) * A10.i + R(-64) * A11.i + R(62) * A12.i + R(-28) * A13.i + R(-10) * A14.i + R(-1) * A15.i + R(62) * A16.i + R(-10) * A17.i + R(8) * A18.i + R(-1) * A19.i + R(-64) * A20.i + R(8) * A21.i + R(-10) * A22.i + R(-1) * A23.i;
                  cs += A10.r * zr + A10.i * zi; }
                { const R zr = R(512) * R(0.5) * A11.r + R(71) * A12.r + R(62) * A13.r + R(-1) * A14.r + R(8) * A15.r + R(-10) * A16.r + R(80) * A17.r + R(-1) * A18.r + R(-10) * A19.r + R(8) * A20.r + R(-64) * A21.r + R(-1) * A22.r + R(8) * A23.r; const R zi = R(512) * R(0.5) * A11.i + R(71) * A12.i + R(62) * A13.i + R(-1) * A14.i + R(8) * A15.i + R(-10) * A16.i + R(80) * A17.i + R(-1) * A18.i + R(-10) * A19.i + R(8) * A20.i + R(-64) * A21.i + R(-1) * A22.i + R(8) * A23.i;
                  cs += A11.r * zr + A11.i * zi; }
                { const R zr = R(512) * R(0.5) * A12.r + R(-64) * A13.r + R(-64) * A14.r + R(8) * A15.r + R(8) * A16.r + R(80) * A17.r + R(62) * A18.r + R(-10) * A19.r + R(-28) * A20.r + R(62) * A21.r + R(-1) * A22.r + R(-10) * A23.r; const R zi = R(512) * R(0.5) * A12.i + R(-64) * A13.i + R(-64) * A14.i + R(8) * A15.i + R(8) * A16.i + R(80) * A17.i + R(62) * A18.i + R(-10) * A19.i + R(-28) * A20.i + R(62) * A21.i + R(-1) * A22.i + R(-10) * A23.i;
                  cs += A12.r * zr + A12.i * zi; }
                { const R zr = R(512) * R(0.5) * A13.r + R(8) * A14.r + R(80) * A15.r + R(-64) * A16.r + R(8) * A17.r + R(-10) * A18.r + R(80) * A19.r + R(62) * A20.r + R(71) * A21.r + R(8) * A22.r + R(-1) * A23.r; const R zi = R(512) * R(0.5) * A13.i + R(8) * A14.i + R(80) * A15.i + R(-64) * A16.i + R(8) * A17.i + R(-10) * A18.i + R(80) * A19.i + R(62) * A20.i + R(71) * A21.i + R(8) * A22.i + R(-1) * A23.i;
                  cs += A13.r * zr + A13.i * zi; }
                { const R zr = R(512) * R(0.5) * A14.r + R(-64) * A15.r + R(80) * A16.r + R(8) * A17.r + R(-28) * A18.r + R(62) * A19.r + R(62) * A20.r + R(-10) * A21.r + R(-10) * A22.r + R(-1) * A23.r; const R zi = R(512) * R(0.5) * A14.i + R(-64) * A15.i + R(80) * A16.i + R(8) * A17.i + R(-28) * A18.i + R(62) * A19.i + R(62) * A20.i + R(-10) * A21.i + R(-10) * A22.i + R(-1) * A23.i;
                  cs += A14.r * zr + A14.i * zi; }
                { const R zr = R(512) * R(0.5) * A15.r + R(8) * A16.r + R(-64) * A17.r + R(62) * A18.r + R(71) * A19.r + R(-10) * A20.r + R(80) * A21.r + R(-1) * A22.r + R(8) * A23.r; const R zi = R(512) * R(0.5) * A15.i + R(8) * A16.i + R(-64) * A17.i + R(62) * A18.i + R(71) * A19.i + R(-10) * A20.i + R(80) * A21.i + R(-1) * A22.i + R(8) * A23.i;
                  cs += A15.r * zr + A15.i * zi; }
                { const R zr = R(512) * R(0.5) * A16.r + R(-64) * A17.r + R(-1) * A18.r + R(8) * A19.r + R(-10) * A20.r + R(-1) * A21.r + R(-64) * A22.r + R(8) * A23.r; const R zi = R(512) * R(0.5) * A16.i + R(-64) * A17.i + R(-1) * A18.i + R(8) * A19.i + R(-10) * A20.i + R(-1) * A21.i + R(-64) * A22.i + R(8) * A23.i;
                  cs += A16.r * zr + A16.i * zi; }
                { const R zr = R(512) * R(0.5) * A17.r + R(-10) * A18.r + R(-1) * A19.r + R(-1) * A20.r + R(8) * A21.r + R(8) * A22.r + R(-64) * A23.r; const R zi = R(512) * R(0.5) * A17.i + R(-10) * A18.i + R(-1) * A19.i + R(-1) * A20.i + R(8) * A21.i + R(8) * A22.i + R(-64) * A23.i;
                  cs += A17.r * zr + A17.i * zi; }
                { const R zr = R(512) * R(0.5) * A18.r + R(-64) * A19.r + R(-64) * A20.r + R(8) * A21.r + R(8) * A22.r + R(80) * A23.r; const R zi = R(512) * R(0.5) * A18.i + R(-64) * A19.i + R(-64) * A20.i + R(8) * A21.i + R(8) * A22.i + R(80) * A23.i;
                  cs += A18.r * zr + A18.i * zi; }
                { const R zr = R(512) * R(0.5) * A19.r + R(8) * A20.r + R(80) * A21.r + R(-64) * A22.r + R(8) * A23.r; const R zi = R(512) * R(0.5) * A19.i + R(8) * A20.i + R(80) * A21.i + R(-64) * A22.i + R(8) * A23.i;
                  cs += A19.r * zr + A19.i * zi; }
                { const R zr = R(512) * R(0.5) * A20.r + R(-64) * A21.r + R(80) * A22.r + R(8) * A23.r; const R zi = R(512) * R(0.5) * A20.i + R(-64) * A21.i + R(80) * A22.i + R(8) * A23.i;
                  cs += A20.r * zr + A20.i * zi; }
                { const R zr = R(512) * R(0.5) * A21.r + R(8) * A22.r + R(-64) * A23.r; const R zi = R(512) * R(0.5) * A21.i + R(8) * A22.i + R(-64) * A23.i;
                  cs += A21.r * zr + A21.i * zi; }
                { const R zr = R(512) * R(0.5) * A22.r + R(-64) * A23.r; const R zi = R(512) * R(0.5) * A22.i + R(-64) * A23.i;
                  cs += A22.r * zr + A22.i * zi; }
                { const R zr = R(512) * R(0.5) * A23.r; const R zi = R(512) * R(0.5) * A23.i;
                  cs += A23.r * zr + A23.i * zi; }
                acc += R(4) * cs;  // x2 symmetric colour sum, x2 helicity flip
              }
            }
          }
        }
      }
    }
  }
  return acc;
}

// floating-point operations of one full helicity sum (all levels, all loop trips)
constexpr long FLOPS_HEL_SUM = 471884;
}}  // namespace
