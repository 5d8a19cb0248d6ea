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
constexpr int MAX_LB = 4;  // helicity levels that can be spread over lanes
constexpr int NJS = 24;  // currents of 3+ gluons, one JStore slot each
constexpr int CDEN = 54;
constexpr int IDENT = 2;  // identical outgoing gluons (1/IDENT!)
constexpr unsigned OUTGOING_GLUONS = 12u;  // bit g: gluon g outgoing
__host__ __device__ constexpr int cint(int i, int j) { constexpr int c[K * K] = {512, -64, -64, 8, 8, 80, -64, 8, 8, -1, -1, -10, 8, -1, 80, -10, 71, 62, -1, -10, -10, 62, 62, -28, -64, 512, 8, 80, -64, 8, 8, -64, -1, -10, 8, -1, -1, -10, -10, 62, 62, -28, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, 80, -10, 71, 62, -64, 8, 8, -1, -1, -10, -10, -1, 62, -28, -10, 62, 8, 80, -64, 512, 8, -64, -1, -10, -10, 62, 62, -28, 8, -64, -1, -10, 8, -1, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, -1, 8, 71, 62, 80, -10, -10, -1, 62, -28, -10, 62, -64, 8, 8, -1, -1, -10, 80, 8, 8, -64, -64, 512, -10, -1, 62, -28, -10, 62, -1, 8, 71, 62, 80, -10, 8, -64, -1, -10, 8, -1, -64, 8, 8, -1, -1, -10, 512, -64, -64, 8, 8, 80, 80, -10, 8, -1, 62, 71, -10, 62, -1, -10, -28, 62, 8, -64, -1, -10, 8, -1, -64, 512, 8, 80, -64, 8, -10, 62, -1, -10, -28, 62, 80, -10, 8, -1, 62, 71, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, -64, 8, -10, -1, 62, -28, -10, -1, 62, -10, -1, -10, -10, 62, 62, -28, 8, 80, -64, 512, 8, -64, -1, -10, 8, -64, -1, 8, 71, 62, -1, 8, -10, 80, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, 62, -28, -10, -1, 62, -10, 8, -1, -64, 8, -10, -1, -10, -1, 62, -28, -10, 62, 80, 8, 8, -64, -64, 512, 71, 62, -1, 8, -10, 80, -1, -10, 8, -64, -1, 8, 8, -1, -64, 8, -10, -1, 80, -10, 8, -1, 62, 71, 512, -64, -64, 8, 8, 80, 62, -10, -28, 62, -1, -10, -1, -10, 8, -64, -1, 8, -10, 62, -1, -10, -28, 62, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, 80, -10, 8, -1, 62, 71, 8, -1, -64, 8, -10, -1, -64, 8, 512, -64, 80, 8, -28, 62, 62, -10, -10, -1, -10, 62, -1, -10, -28, 62, -1, -10, 8, -64, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, 71, 62, -1, 8, -10, 80, 62, -28, -10, -1, 62, -10, 8, -64, 80, 8, 512, -64, -1, 8, -10, -1, -64, 8, 62, -28, -10, -1, 62, -10, 71, 62, -1, 8, -10, 80, 80, 8, 8, -64, -64, 512, -10, -1, -1, 8, 8, -64, -1, 8, -10, -1, -64, 8, -10, 80, 62, 71, 8, -1, 62, -10, -28, 62, -1, -10, 512, -64, -64, 8, 8, 80, -10, -1, -1, 8, 8, -64, 62, -10, -28, 62, -1, -10, -10, 80, 62, 71, 8, -1, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, -1, 8, -10, -1, -64, 8, -28, 62, 62, -10, -10, -1, -64, 8, 512, -64, 80, 8, 62, -10, -28, 62, -1, -10, -10, -1, -1, 8, 8, -64, 62, 71, -10, 80, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, -28, 62, 62, -10, -10, -1, -1, 8, -10, -1, -64, 8, 8, -64, 80, 8, 512, -64, -28, 62, 62, -10, -10, -1, 62, 71, -10, 80, -1, 8, -10, -1, -1, 8, 8, -64, 80, 8, 8, -64, -64, 512}; return c[i * K + j]; }
constexpr int ORDER[K][NG] = {{0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 1, 3}, {0, 2, 3, 1}, {0, 3, 1, 2}, {0, 3, 2, 1}, {1, 0, 2, 3}, {1, 0, 3, 2}, {1, 2, 0, 3}, {1, 2, 3, 0}, {1, 3, 0, 2}, {1, 3, 2, 0}, {2, 0, 1, 3}, {2, 0, 3, 1}, {2, 1, 0, 3}, {2, 1, 3, 0}, {2, 3, 0, 1}, {2, 3, 1, 0}, {3, 0, 1, 2}, {3, 0, 2, 1}, {3, 1, 0, 2}, {3, 1, 2, 0}, {3, 2, 0, 1}, {3, 2, 1, 0}};
static __device__ const short CI[K * K] = {512, -64, -64, 8, 8, 80, -64, 8, 8, -1, -1, -10, 8, -1, 80, -10, 71, 62, -1, -10, -10, 62, 62, -28, -64, 512, 8, 80, -64, 8, 8, -64, -1, -10, 8, -1, -1, -10, -10, 62, 62, -28, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, 80, -10, 71, 62, -64, 8, 8, -1, -1, -10, -10, -1, 62, -28, -10, 62, 8, 80, -64, 512, 8, -64, -1, -10, -10, 62, 62, -28, 8, -64, -1, -10, 8, -1, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, -1, 8, 71, 62, 80, -10, -10, -1, 62, -28, -10, 62, -64, 8, 8, -1, -1, -10, 80, 8, 8, -64, -64, 512, -10, -1, 62, -28, -10, 62, -1, 8, 71, 62, 80, -10, 8, -64, -1, -10, 8, -1, -64, 8, 8, -1, -1, -10, 512, -64, -64, 8, 8, 80, 80, -10, 8, -1, 62, 71, -10, 62, -1, -10, -28, 62, 8, -64, -1, -10, 8, -1, -64, 512, 8, 80, -64, 8, -10, 62, -1, -10, -28, 62, 80, -10, 8, -1, 62, 71, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, -64, 8, -10, -1, 62, -28, -10, -1, 62, -10, -1, -10, -10, 62, 62, -28, 8, 80, -64, 512, 8, -64, -1, -10, 8, -64, -1, 8, 71, 62, -1, 8, -10, 80, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, 62, -28, -10, -1, 62, -10, 8, -1, -64, 8, -10, -1, -10, -1, 62, -28, -10, 62, 80, 8, 8, -64, -64, 512, 71, 62, -1, 8, -10, 80, -1, -10, 8, -64, -1, 8, 8, -1, -64, 8, -10, -1, 80, -10, 8, -1, 62, 71, 512, -64, -64, 8, 8, 80, 62, -10, -28, 62, -1, -10, -1, -10, 8, -64, -1, 8, -10, 62, -1, -10, -28, 62, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, 80, -10, 8, -1, 62, 71, 8, -1, -64, 8, -10, -1, -64, 8, 512, -64, 80, 8, -28, 62, 62, -10, -10, -1, -10, 62, -1, -10, -28, 62, -1, -10, 8, -64, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, 71, 62, -1, 8, -10, 80, 62, -28, -10, -1, 62, -10, 8, -64, 80, 8, 512, -64, -1, 8, -10, -1, -64, 8, 62, -28, -10, -1, 62, -10, 71, 62, -1, 8, -10, 80, 80, 8, 8, -64, -64, 512, -10, -1, -1, 8, 8, -64, -1, 8, -10, -1, -64, 8, -10, 80, 62, 71, 8, -1, 62, -10, -28, 62, -1, -10, 512, -64, -64, 8, 8, 80, -10, -1, -1, 8, 8, -64, 62, -10, -28, 62, -1, -10, -10, 80, 62, 71, 8, -1, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, -1, 8, -10, -1, -64, 8, -28, 62, 62, -10, -10, -1, -64, 8, 512, -64, 80, 8, 62, -10, -28, 62, -1, -10, -10, -1, -1, 8, 8, -64, 62, 71, -10, 80, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, -28, 62, 62, -10, -10, -1, -1, 8, -10, -1, -64, 8, 8, -64, 80, 8, 512, -64, -28, 62, 62, -10, -10, -1, 62, 71, -10, 80, -1, 8, -10, -1, -1, 8, 8, -64, 80, 8, 8, -64, -64, 512};  // row-major C_int for the tensor-core sum

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
  [[maybe_unused]] R cz0_0 = R(0), cz0_1 = R(0), cz0_2 = R(0), cz0_3 = R(0), cz1_0 = R(0), cz1_1 = R(0), cz1_2 = R(0), cz1_3 = R(0);
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
          js.put(3, J0_1_3);
          cv<R> J0_2_3 = vvv(E0, Kn.P[1], J2_3, Kn.P[12], Kn.cg[13]);
          vvv_acc(J0_2_3, J0_2, Kn.P[5], E3, Kn.P[8], Kn.cg[13]);
          vvvv_acc(J0_2_3, E0, E2, E3, Kn.c4[13]);
          js.put(4, J0_2_3);
          cv<R> J0_3_1 = vvv(E0, Kn.P[1], J3_1, Kn.P[10], Kn.cg[11]);
          vvv_acc(J0_3_1, J0_3, Kn.P[9], E1, Kn.P[2], Kn.cg[11]);
          vvvv_acc(J0_3_1, E0, E3, E1, Kn.c4[11]);
          js.put(5, J0_3_1);
          cv<R> J0_3_2 = vvv(E0, Kn.P[1], J3_2, Kn.P[12], Kn.cg[13]);
          vvv_acc(J0_3_2, J0_3, Kn.P[9], E2, Kn.P[4], Kn.cg[13]);
          vvvv_acc(J0_3_2, E0, E3, E2, Kn.c4[13]);
          js.put(6, J0_3_2);
          cv<R> J1_0_3 = vvv(E1, Kn.P[2], J0_3, Kn.P[9], Kn.cg[11]);
          vvv_acc(J1_0_3, J1_0, Kn.P[3], E3, Kn.P[8], Kn.cg[11]);
          vvvv_acc(J1_0_3, E1, E0, E3, Kn.c4[11]);
          js.put(7, J1_0_3);
          cv<R> J1_2_3 = vvv(E1, Kn.P[2], J2_3, Kn.P[12], Kn.cg[14]);
          vvv_acc(J1_2_3, J1_2, Kn.P[6], E3, Kn.P[8], Kn.cg[14]);
          vvvv_acc(J1_2_3, E1, E2, E3, Kn.c4[14]);
          js.put(8, J1_2_3);
          cv<R> J1_3_2 = vvv(E1, Kn.P[2], J3_2, Kn.P[12], Kn.cg[14]);
          vvv_acc(J1_3_2, J1_3, Kn.P[10], E2, Kn.P[4], Kn.cg[14]);
          vvvv_acc(J1_3_2, E1, E3, E2, Kn.c4[14]);
          js.put(9, J1_3_2);
          cv<R> J2_0_3 = vvv(E2, Kn.P[4], J0_3, Kn.P[9], Kn.cg[13]);
          vvv_acc(J2_0_3, J2_0, Kn.P[5], E3, Kn.P[8], Kn.cg[13]);
          vvvv_acc(J2_0_3, E2, E0, E3, Kn.c4[13]);
          js.put(10, J2_0_3);
          cv<R> J2_1_3 = vvv(E2, Kn.P[4], J1_3, Kn.P[10], Kn.cg[14]);
          vvv_acc(J2_1_3, J2_1, Kn.P[6], E3, Kn.P[8], Kn.cg[14]);
          vvvv_acc(J2_1_3, E2, E1, E3, Kn.c4[14]);
          js.put(11, J2_1_3);
          cv<R> J0_1_2_3 = vvv(E0, Kn.P[1], js.get(8), Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_1_2_3, J0_1, Kn.P[3], J2_3, Kn.P[12], Kn.cg[15]);
          vvv_acc(J0_1_2_3, js.get(0), Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J0_1_2_3, E0, E1, J2_3, Kn.c4[15]);
          vvvv_acc(J0_1_2_3, E0, J1_2, E3, Kn.c4[15]);
          vvvv_acc(J0_1_2_3, J0_1, E2, E3, Kn.c4[15]);
          js.put(12, J0_1_2_3);
          cv<R> J0_1_3_2 = vvv(E0, Kn.P[1], js.get(9), Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_1_3_2, J0_1, Kn.P[3], J3_2, Kn.P[12], Kn.cg[15]);
          vvv_acc(J0_1_3_2, js.get(3), Kn.P[11], E2, Kn.P[4], Kn.cg[15]);
          vvvv_acc(J0_1_3_2, E0, E1, J3_2, Kn.c4[15]);
          vvvv_acc(J0_1_3_2, E0, J1_3, E2, Kn.c4[15]);
          vvvv_acc(J0_1_3_2, J0_1, E3, E2, Kn.c4[15]);
          js.put(13, J0_1_3_2);
          cv<R> J0_2_1_3 = vvv(E0, Kn.P[1], js.get(11), Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_2_1_3, J0_2, Kn.P[5], J1_3, Kn.P[10], Kn.cg[15]);
          vvv_acc(J0_2_1_3, js.get(1), Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J0_2_1_3, E0, E2, J1_3, Kn.c4[15]);
          vvvv_acc(J0_2_1_3, E0, J2_1, E3, Kn.c4[15]);
          vvvv_acc(J0_2_1_3, J0_2, E1, E3, Kn.c4[15]);
          js.put(14, J0_2_1_3);
          cv<R> J0_2_3_1 = vvv(E0, Kn.P[1], js.get(9), Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_2_3_1, J0_2, Kn.P[5], J3_1, Kn.P[10], Kn.cg[15]);
          vvv_acc(J0_2_3_1, js.get(4), Kn.P[13], E1, Kn.P[2], Kn.cg[15]);
          vvvv_acc(J0_2_3_1, E0, E2, J3_1, Kn.c4[15]);
          vvvv_acc(J0_2_3_1, E0, J2_3, E1, Kn.c4[15]);
          vvvv_acc(J0_2_3_1, J0_2, E3, E1, Kn.c4[15]);
          js.put(15, J0_2_3_1);
          cv<R> J0_3_1_2 = vvv(E0, Kn.P[1], js.get(11), Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_3_1_2, J0_3, Kn.P[9], J1_2, Kn.P[6], Kn.cg[15]);
          vvv_acc(J0_3_1_2, js.get(5), Kn.P[11], E2, Kn.P[4], Kn.cg[15]);
          vvvv_acc(J0_3_1_2, E0, E3, J1_2, Kn.c4[15]);
          vvvv_acc(J0_3_1_2, E0, J3_1, E2, Kn.c4[15]);
          vvvv_acc(J0_3_1_2, J0_3, E1, E2, Kn.c4[15]);
          js.put(16, J0_3_1_2);
          cv<R> J0_3_2_1 = vvv(E0, Kn.P[1], js.get(8), Kn.P[14], Kn.cg[15]);
          vvv_acc(J0_3_2_1, J0_3, Kn.P[9], J2_1, Kn.P[6], Kn.cg[15]);
          vvv_acc(J0_3_2_1, js.get(6), Kn.P[13], E1, Kn.P[2], Kn.cg[15]);
          vvvv_acc(J0_3_2_1, E0, E3, J2_1, Kn.c4[15]);
          vvvv_acc(J0_3_2_1, E0, J3_2, E1, Kn.c4[15]);
          vvvv_acc(J0_3_2_1, J0_3, E2, E1, Kn.c4[15]);
          js.put(17, J0_3_2_1);
          cv<R> J1_0_2_3 = vvv(E1, Kn.P[2], js.get(4), Kn.P[13], Kn.cg[15]);
          vvv_acc(J1_0_2_3, J1_0, Kn.P[3], J2_3, Kn.P[12], Kn.cg[15]);
          vvv_acc(J1_0_2_3, js.get(2), Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J1_0_2_3, E1, E0, J2_3, Kn.c4[15]);
          vvvv_acc(J1_0_2_3, E1, J0_2, E3, Kn.c4[15]);
          vvvv_acc(J1_0_2_3, J1_0, E2, E3, Kn.c4[15]);
          js.put(18, J1_0_2_3);
          cv<R> J1_0_3_2 = vvv(E1, Kn.P[2], js.get(6), Kn.P[13], Kn.cg[15]);
          vvv_acc(J1_0_3_2, J1_0, Kn.P[3], J3_2, Kn.P[12], Kn.cg[15]);
          vvv_acc(J1_0_3_2, js.get(7), Kn.P[11], E2, Kn.P[4], Kn.cg[15]);
          vvvv_acc(J1_0_3_2, E1, E0, J3_2, Kn.c4[15]);
          vvvv_acc(J1_0_3_2, E1, J0_3, E2, Kn.c4[15]);
          vvvv_acc(J1_0_3_2, J1_0, E3, E2, Kn.c4[15]);
          js.put(19, J1_0_3_2);
          cv<R> J1_2_0_3 = vvv(E1, Kn.P[2], js.get(10), Kn.P[13], Kn.cg[15]);
          vvv_acc(J1_2_0_3, J1_2, Kn.P[6], J0_3, Kn.P[9], Kn.cg[15]);
          vvv_acc(J1_2_0_3, js.get(1), Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J1_2_0_3, E1, E2, J0_3, Kn.c4[15]);
          vvvv_acc(J1_2_0_3, E1, J2_0, E3, Kn.c4[15]);
          vvvv_acc(J1_2_0_3, J1_2, E0, E3, Kn.c4[15]);
          js.put(20, J1_2_0_3);
          cv<R> J1_3_0_2 = vvv(E1, Kn.P[2], js.get(10), Kn.P[13], Kn.cg[15]);
          vvv_acc(J1_3_0_2, J1_3, Kn.P[10], J0_2, Kn.P[5], Kn.cg[15]);
          vvv_acc(J1_3_0_2, js.get(5), Kn.P[11], E2, Kn.P[4], Kn.cg[15]);
          vvvv_acc(J1_3_0_2, E1, E3, J0_2, Kn.c4[15]);
          vvvv_acc(J1_3_0_2, E1, J3_0, E2, Kn.c4[15]);
          vvvv_acc(J1_3_0_2, J1_3, E0, E2, Kn.c4[15]);
          js.put(21, J1_3_0_2);
          cv<R> J2_0_1_3 = vvv(E2, Kn.P[4], js.get(3), Kn.P[11], Kn.cg[15]);
          vvv_acc(J2_0_1_3, J2_0, Kn.P[5], J1_3, Kn.P[10], Kn.cg[15]);
          vvv_acc(J2_0_1_3, js.get(2), Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J2_0_1_3, E2, E0, J1_3, Kn.c4[15]);
          vvvv_acc(J2_0_1_3, E2, J0_1, E3, Kn.c4[15]);
          vvvv_acc(J2_0_1_3, J2_0, E1, E3, Kn.c4[15]);
          js.put(22, J2_0_1_3);
          cv<R> J2_1_0_3 = vvv(E2, Kn.P[4], js.get(7), Kn.P[11], Kn.cg[15]);
          vvv_acc(J2_1_0_3, J2_1, Kn.P[6], J0_3, Kn.P[9], Kn.cg[15]);
          vvv_acc(J2_1_0_3, js.get(0), Kn.P[7], E3, Kn.P[8], Kn.cg[15]);
          vvvv_acc(J2_1_0_3, E2, E1, J0_3, Kn.c4[15]);
          vvvv_acc(J2_1_0_3, E2, J1_0, E3, Kn.c4[15]);
          vvvv_acc(J2_1_0_3, J2_1, E0, E3, Kn.c4[15]);
          js.put(23, J2_1_0_3);
          #pragma unroll 1
          for (int i4 = 0; i4 < (LB >= 4 ? 1 : 2); ++i4) {
            const int h4 = LB >= 4 ? ((lane >> (LB - 4)) & 1) : i4;
            const sp<R> S_E = h4 ? X.v[1] : X.v[0];
            constexpr bool SH = sizeof(R) == 8;  // share every repeated slash (FP64)
            sp<R> tS_0 = slash(E0, S_E);
            const sp<R> S_0 = fprop(Kn.qc[1], Kn.mc[1], tS_0);
            sp<R> tS_1_0;
            [[maybe_unused]] sp<R> Y0_1__E;  // Jslash(0,1) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y0_1__E = slash(J0_1, S_E);
              if constexpr (true) tS_1_0 = spneg(Y0_1__E); else tS_1_0 = slash(J1_0, S_E);
              slash_acc(tS_1_0, E1, S_0);  // single-gluon term, fused
            } else {
              tS_1_0 = slash(E1, S_0);
              slash_acc(tS_1_0, J1_0, S_E);
            }
            const sp<R> S_1_0 = fprop(Kn.qc[3], Kn.mc[3], tS_1_0);
            sp<R> tS_2_1_0;
            [[maybe_unused]] sp<R> Y1_2__0;  // Jslash(1,2) psi(0)
            [[maybe_unused]] sp<R> Y0_1_2__E;  // Jslash(0,1,2) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y1_2__0 = slash(J1_2, S_0);
              if constexpr (true) tS_2_1_0 = spneg(Y1_2__0); else tS_2_1_0 = slash(J2_1, S_0);
              if constexpr (true) Y0_1_2__E = slash(js.get(0), S_E);
              if constexpr (true) spadd(tS_2_1_0, Y0_1_2__E); else slash_acc(tS_2_1_0, js.get(0), S_E);
              slash_acc(tS_2_1_0, E2, S_1_0);  // single-gluon term, fused
            } else {
              tS_2_1_0 = slash(E2, S_1_0);
              slash_acc(tS_2_1_0, J2_1, S_0);
              slash_acc(tS_2_1_0, js.get(0), S_E);
            }
            const sp<R> S_2_1_0 = fprop(Kn.qc[7], Kn.mc[7], tS_2_1_0);
            sp<R> X23;
            [[maybe_unused]] sp<R> Y2_3__1_0;  // Jslash(2,3) psi(1_0)
            [[maybe_unused]] sp<R> Y1_2_3__0;  // Jslash(1,2,3) psi(0)
            [[maybe_unused]] sp<R> Y0_1_2_3__E;  // Jslash(0,1,2,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y2_3__1_0 = slash(J2_3, S_1_0);
              if constexpr (true) X23 = spneg(Y2_3__1_0); else X23 = slash(J3_2, S_1_0);
              if constexpr (true) Y1_2_3__0 = slash(js.get(8), S_0);
              if constexpr (true) spadd(X23, Y1_2_3__0); else slash_acc(X23, js.get(8), S_0);
              if constexpr (true) Y0_1_2_3__E = slash(js.get(12), S_E);
              if constexpr (true) spsub(X23, Y0_1_2_3__E); else slash_acc(X23, neg(js.get(12)), S_E);
              slash_acc(X23, E3, S_2_1_0);  // single-gluon term, fused
            } else {
              X23 = slash(E3, S_2_1_0);
              slash_acc(X23, J3_2, S_1_0);
              slash_acc(X23, js.get(8), S_0);
              slash_acc(X23, neg(js.get(12)), S_E);
            }
            const cx<R> A23_0 = rowcol(X.ub[0], X23), A23_1 = rowcol(X.ub[1], X23);
            sp<R> tS_3_1_0;
            [[maybe_unused]] sp<R> Y1_3__0;  // Jslash(1,3) psi(0)
            [[maybe_unused]] sp<R> Y0_1_3__E;  // Jslash(0,1,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y1_3__0 = slash(J1_3, S_0);
              if constexpr (true) tS_3_1_0 = spneg(Y1_3__0); else tS_3_1_0 = slash(J3_1, S_0);
              if constexpr (true) Y0_1_3__E = slash(js.get(3), S_E);
              if constexpr (true) spadd(tS_3_1_0, Y0_1_3__E); else slash_acc(tS_3_1_0, js.get(3), S_E);
              slash_acc(tS_3_1_0, E3, S_1_0);  // single-gluon term, fused
            } else {
              tS_3_1_0 = slash(E3, S_1_0);
              slash_acc(tS_3_1_0, J3_1, S_0);
              slash_acc(tS_3_1_0, js.get(3), S_E);
            }
            const sp<R> S_3_1_0 = fprop(Kn.qc[11], Kn.mc[11], tS_3_1_0);
            sp<R> X17;
            [[maybe_unused]] sp<R> Y1_3_2__0;  // Jslash(1,3,2) psi(0)
            [[maybe_unused]] sp<R> Y0_1_3_2__E;  // Jslash(0,1,3,2) psi(E)
            if constexpr (SH) {
              if constexpr (true) X17 = Y2_3__1_0; else X17 = slash(J2_3, S_1_0);
              if constexpr (true) Y1_3_2__0 = slash(js.get(9), S_0);
              if constexpr (true) spadd(X17, Y1_3_2__0); else slash_acc(X17, js.get(9), S_0);
              if constexpr (true) Y0_1_3_2__E = slash(js.get(13), S_E);
              if constexpr (true) spsub(X17, Y0_1_3_2__E); else slash_acc(X17, neg(js.get(13)), S_E);
              slash_acc(X17, E2, S_3_1_0);  // single-gluon term, fused
            } else {
              X17 = slash(E2, S_3_1_0);
              slash_acc(X17, J2_3, S_1_0);
              slash_acc(X17, js.get(9), S_0);
              slash_acc(X17, neg(js.get(13)), S_E);
            }
            const cx<R> A17_0 = rowcol(X.ub[0], X17), A17_1 = rowcol(X.ub[1], X17);
            sp<R> tS_2_0;
            [[maybe_unused]] sp<R> Y0_2__E;  // Jslash(0,2) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y0_2__E = slash(J0_2, S_E);
              if constexpr (true) tS_2_0 = spneg(Y0_2__E); else tS_2_0 = slash(J2_0, S_E);
              slash_acc(tS_2_0, E2, S_0);  // single-gluon term, fused
            } else {
              tS_2_0 = slash(E2, S_0);
              slash_acc(tS_2_0, J2_0, S_E);
            }
            const sp<R> S_2_0 = fprop(Kn.qc[5], Kn.mc[5], tS_2_0);
            sp<R> tS_1_2_0;
            [[maybe_unused]] sp<R> Y0_2_1__E;  // Jslash(0,2,1) psi(E)
            if constexpr (SH) {
              if constexpr (true) tS_1_2_0 = Y1_2__0; else tS_1_2_0 = slash(J1_2, S_0);
              if constexpr (true) Y0_2_1__E = slash(js.get(1), S_E);
              if constexpr (true) spadd(tS_1_2_0, Y0_2_1__E); else slash_acc(tS_1_2_0, js.get(1), S_E);
              slash_acc(tS_1_2_0, E1, S_2_0);  // single-gluon term, fused
            } else {
              tS_1_2_0 = slash(E1, S_2_0);
              slash_acc(tS_1_2_0, J1_2, S_0);
              slash_acc(tS_1_2_0, js.get(1), S_E);
            }
            const sp<R> S_1_2_0 = fprop(Kn.qc[7], Kn.mc[7], tS_1_2_0);
            sp<R> X21;
            [[maybe_unused]] sp<R> Y1_3__2_0;  // Jslash(1,3) psi(2_0)
            [[maybe_unused]] sp<R> Y2_1_3__0;  // Jslash(2,1,3) psi(0)
            [[maybe_unused]] sp<R> Y0_2_1_3__E;  // Jslash(0,2,1,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y1_3__2_0 = slash(J1_3, S_2_0);
              if constexpr (true) X21 = spneg(Y1_3__2_0); else X21 = slash(J3_1, S_2_0);
              if constexpr (true) Y2_1_3__0 = slash(js.get(11), S_0);
              if constexpr (true) spadd(X21, Y2_1_3__0); else slash_acc(X21, js.get(11), S_0);
              if constexpr (true) Y0_2_1_3__E = slash(js.get(14), S_E);
              if constexpr (true) spsub(X21, Y0_2_1_3__E); else slash_acc(X21, neg(js.get(14)), S_E);
              slash_acc(X21, E3, S_1_2_0);  // single-gluon term, fused
            } else {
              X21 = slash(E3, S_1_2_0);
              slash_acc(X21, J3_1, S_2_0);
              slash_acc(X21, js.get(11), S_0);
              slash_acc(X21, neg(js.get(14)), S_E);
            }
            const cx<R> A21_0 = rowcol(X.ub[0], X21), A21_1 = rowcol(X.ub[1], X21);
            sp<R> tS_3_2_0;
            [[maybe_unused]] sp<R> Y2_3__0;  // Jslash(2,3) psi(0)
            [[maybe_unused]] sp<R> Y0_2_3__E;  // Jslash(0,2,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y2_3__0 = slash(J2_3, S_0);
              if constexpr (true) tS_3_2_0 = spneg(Y2_3__0); else tS_3_2_0 = slash(J3_2, S_0);
              if constexpr (true) Y0_2_3__E = slash(js.get(4), S_E);
              if constexpr (true) spadd(tS_3_2_0, Y0_2_3__E); else slash_acc(tS_3_2_0, js.get(4), S_E);
              slash_acc(tS_3_2_0, E3, S_2_0);  // single-gluon term, fused
            } else {
              tS_3_2_0 = slash(E3, S_2_0);
              slash_acc(tS_3_2_0, J3_2, S_0);
              slash_acc(tS_3_2_0, js.get(4), S_E);
            }
            const sp<R> S_3_2_0 = fprop(Kn.qc[13], Kn.mc[13], tS_3_2_0);
            sp<R> X11;
            [[maybe_unused]] sp<R> Y0_2_3_1__E;  // Jslash(0,2,3,1) psi(E)
            if constexpr (SH) {
              if constexpr (true) X11 = Y1_3__2_0; else X11 = slash(J1_3, S_2_0);
              if constexpr (true) spadd(X11, Y1_3_2__0); else slash_acc(X11, js.get(9), S_0);
              if constexpr (true) Y0_2_3_1__E = slash(js.get(15), S_E);
              if constexpr (true) spsub(X11, Y0_2_3_1__E); else slash_acc(X11, neg(js.get(15)), S_E);
              slash_acc(X11, E1, S_3_2_0);  // single-gluon term, fused
            } else {
              X11 = slash(E1, S_3_2_0);
              slash_acc(X11, J1_3, S_2_0);
              slash_acc(X11, js.get(9), S_0);
              slash_acc(X11, neg(js.get(15)), S_E);
            }
            const cx<R> A11_0 = rowcol(X.ub[0], X11), A11_1 = rowcol(X.ub[1], X11);
            sp<R> tS_3_0;
            [[maybe_unused]] sp<R> Y0_3__E;  // Jslash(0,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y0_3__E = slash(J0_3, S_E);
              if constexpr (true) tS_3_0 = spneg(Y0_3__E); else tS_3_0 = slash(J3_0, S_E);
              slash_acc(tS_3_0, E3, S_0);  // single-gluon term, fused
            } else {
              tS_3_0 = slash(E3, S_0);
              slash_acc(tS_3_0, J3_0, S_E);
            }
            const sp<R> S_3_0 = fprop(Kn.qc[9], Kn.mc[9], tS_3_0);
            sp<R> tS_1_3_0;
            [[maybe_unused]] sp<R> Y0_3_1__E;  // Jslash(0,3,1) psi(E)
            if constexpr (SH) {
              if constexpr (true) tS_1_3_0 = Y1_3__0; else tS_1_3_0 = slash(J1_3, S_0);
              if constexpr (true) Y0_3_1__E = slash(js.get(5), S_E);
              if constexpr (true) spadd(tS_1_3_0, Y0_3_1__E); else slash_acc(tS_1_3_0, js.get(5), S_E);
              slash_acc(tS_1_3_0, E1, S_3_0);  // single-gluon term, fused
            } else {
              tS_1_3_0 = slash(E1, S_3_0);
              slash_acc(tS_1_3_0, J1_3, S_0);
              slash_acc(tS_1_3_0, js.get(5), S_E);
            }
            const sp<R> S_1_3_0 = fprop(Kn.qc[11], Kn.mc[11], tS_1_3_0);
            sp<R> X15;
            [[maybe_unused]] sp<R> Y1_2__3_0;  // Jslash(1,2) psi(3_0)
            [[maybe_unused]] sp<R> Y0_3_1_2__E;  // Jslash(0,3,1,2) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y1_2__3_0 = slash(J1_2, S_3_0);
              if constexpr (true) X15 = spneg(Y1_2__3_0); else X15 = slash(J2_1, S_3_0);
              if constexpr (true) spadd(X15, Y2_1_3__0); else slash_acc(X15, js.get(11), S_0);
              if constexpr (true) Y0_3_1_2__E = slash(js.get(16), S_E);
              if constexpr (true) spsub(X15, Y0_3_1_2__E); else slash_acc(X15, neg(js.get(16)), S_E);
              slash_acc(X15, E2, S_1_3_0);  // single-gluon term, fused
            } else {
              X15 = slash(E2, S_1_3_0);
              slash_acc(X15, J2_1, S_3_0);
              slash_acc(X15, js.get(11), S_0);
              slash_acc(X15, neg(js.get(16)), S_E);
            }
            const cx<R> A15_0 = rowcol(X.ub[0], X15), A15_1 = rowcol(X.ub[1], X15);
            sp<R> tS_2_3_0;
            [[maybe_unused]] sp<R> Y0_3_2__E;  // Jslash(0,3,2) psi(E)
            if constexpr (SH) {
              if constexpr (true) tS_2_3_0 = Y2_3__0; else tS_2_3_0 = slash(J2_3, S_0);
              if constexpr (true) Y0_3_2__E = slash(js.get(6), S_E);
              if constexpr (true) spadd(tS_2_3_0, Y0_3_2__E); else slash_acc(tS_2_3_0, js.get(6), S_E);
              slash_acc(tS_2_3_0, E2, S_3_0);  // single-gluon term, fused
            } else {
              tS_2_3_0 = slash(E2, S_3_0);
              slash_acc(tS_2_3_0, J2_3, S_0);
              slash_acc(tS_2_3_0, js.get(6), S_E);
            }
            const sp<R> S_2_3_0 = fprop(Kn.qc[13], Kn.mc[13], tS_2_3_0);
            sp<R> X9;
            [[maybe_unused]] sp<R> Y0_3_2_1__E;  // Jslash(0,3,2,1) psi(E)
            if constexpr (SH) {
              if constexpr (true) X9 = Y1_2__3_0; else X9 = slash(J1_2, S_3_0);
              if constexpr (true) spadd(X9, Y1_2_3__0); else slash_acc(X9, js.get(8), S_0);
              if constexpr (true) Y0_3_2_1__E = slash(js.get(17), S_E);
              if constexpr (true) spsub(X9, Y0_3_2_1__E); else slash_acc(X9, neg(js.get(17)), S_E);
              slash_acc(X9, E1, S_2_3_0);  // single-gluon term, fused
            } else {
              X9 = slash(E1, S_2_3_0);
              slash_acc(X9, J1_2, S_3_0);
              slash_acc(X9, js.get(8), S_0);
              slash_acc(X9, neg(js.get(17)), S_E);
            }
            const cx<R> A9_0 = rowcol(X.ub[0], X9), A9_1 = rowcol(X.ub[1], X9);
            sp<R> tS_1 = slash(E1, S_E);
            const sp<R> S_1 = fprop(Kn.qc[2], Kn.mc[2], tS_1);
            sp<R> tS_0_1;
            if constexpr (SH) {
              if constexpr (true) tS_0_1 = Y0_1__E; else tS_0_1 = slash(J0_1, S_E);
              slash_acc(tS_0_1, E0, S_1);  // single-gluon term, fused
            } else {
              tS_0_1 = slash(E0, S_1);
              slash_acc(tS_0_1, J0_1, S_E);
            }
            const sp<R> S_0_1 = fprop(Kn.qc[3], Kn.mc[3], tS_0_1);
            sp<R> tS_2_0_1;
            [[maybe_unused]] sp<R> Y0_2__1;  // Jslash(0,2) psi(1)
            [[maybe_unused]] sp<R> Y1_0_2__E;  // Jslash(1,0,2) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y0_2__1 = slash(J0_2, S_1);
              if constexpr (true) tS_2_0_1 = spneg(Y0_2__1); else tS_2_0_1 = slash(J2_0, S_1);
              if constexpr (true) Y1_0_2__E = slash(js.get(2), S_E);
              if constexpr (true) spadd(tS_2_0_1, Y1_0_2__E); else slash_acc(tS_2_0_1, js.get(2), S_E);
              slash_acc(tS_2_0_1, E2, S_0_1);  // single-gluon term, fused
            } else {
              tS_2_0_1 = slash(E2, S_0_1);
              slash_acc(tS_2_0_1, J2_0, S_1);
              slash_acc(tS_2_0_1, js.get(2), S_E);
            }
            const sp<R> S_2_0_1 = fprop(Kn.qc[7], Kn.mc[7], tS_2_0_1);
            sp<R> X22;
            [[maybe_unused]] sp<R> Y2_3__0_1;  // Jslash(2,3) psi(0_1)
            [[maybe_unused]] sp<R> Y0_2_3__1;  // Jslash(0,2,3) psi(1)
            [[maybe_unused]] sp<R> Y1_0_2_3__E;  // Jslash(1,0,2,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y2_3__0_1 = slash(J2_3, S_0_1);
              if constexpr (true) X22 = spneg(Y2_3__0_1); else X22 = slash(J3_2, S_0_1);
              if constexpr (true) Y0_2_3__1 = slash(js.get(4), S_1);
              if constexpr (true) spadd(X22, Y0_2_3__1); else slash_acc(X22, js.get(4), S_1);
              if constexpr (true) Y1_0_2_3__E = slash(js.get(18), S_E);
              if constexpr (true) spsub(X22, Y1_0_2_3__E); else slash_acc(X22, neg(js.get(18)), S_E);
              slash_acc(X22, E3, S_2_0_1);  // single-gluon term, fused
            } else {
              X22 = slash(E3, S_2_0_1);
              slash_acc(X22, J3_2, S_0_1);
              slash_acc(X22, js.get(4), S_1);
              slash_acc(X22, neg(js.get(18)), S_E);
            }
            const cx<R> A22_0 = rowcol(X.ub[0], X22), A22_1 = rowcol(X.ub[1], X22);
            sp<R> tS_3_0_1;
            [[maybe_unused]] sp<R> Y0_3__1;  // Jslash(0,3) psi(1)
            [[maybe_unused]] sp<R> Y1_0_3__E;  // Jslash(1,0,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y0_3__1 = slash(J0_3, S_1);
              if constexpr (true) tS_3_0_1 = spneg(Y0_3__1); else tS_3_0_1 = slash(J3_0, S_1);
              if constexpr (true) Y1_0_3__E = slash(js.get(7), S_E);
              if constexpr (true) spadd(tS_3_0_1, Y1_0_3__E); else slash_acc(tS_3_0_1, js.get(7), S_E);
              slash_acc(tS_3_0_1, E3, S_0_1);  // single-gluon term, fused
            } else {
              tS_3_0_1 = slash(E3, S_0_1);
              slash_acc(tS_3_0_1, J3_0, S_1);
              slash_acc(tS_3_0_1, js.get(7), S_E);
            }
            const sp<R> S_3_0_1 = fprop(Kn.qc[11], Kn.mc[11], tS_3_0_1);
            sp<R> X16;
            [[maybe_unused]] sp<R> Y0_3_2__1;  // Jslash(0,3,2) psi(1)
            [[maybe_unused]] sp<R> Y1_0_3_2__E;  // Jslash(1,0,3,2) psi(E)
            if constexpr (SH) {
              if constexpr (true) X16 = Y2_3__0_1; else X16 = slash(J2_3, S_0_1);
              if constexpr (true) Y0_3_2__1 = slash(js.get(6), S_1);
              if constexpr (true) spadd(X16, Y0_3_2__1); else slash_acc(X16, js.get(6), S_1);
              if constexpr (true) Y1_0_3_2__E = slash(js.get(19), S_E);
              if constexpr (true) spsub(X16, Y1_0_3_2__E); else slash_acc(X16, neg(js.get(19)), S_E);
              slash_acc(X16, E2, S_3_0_1);  // single-gluon term, fused
            } else {
              X16 = slash(E2, S_3_0_1);
              slash_acc(X16, J2_3, S_0_1);
              slash_acc(X16, js.get(6), S_1);
              slash_acc(X16, neg(js.get(19)), S_E);
            }
            const cx<R> A16_0 = rowcol(X.ub[0], X16), A16_1 = rowcol(X.ub[1], X16);
            sp<R> tS_2_1;
            [[maybe_unused]] sp<R> Y1_2__E;  // Jslash(1,2) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y1_2__E = slash(J1_2, S_E);
              if constexpr (true) tS_2_1 = spneg(Y1_2__E); else tS_2_1 = slash(J2_1, S_E);
              slash_acc(tS_2_1, E2, S_1);  // single-gluon term, fused
            } else {
              tS_2_1 = slash(E2, S_1);
              slash_acc(tS_2_1, J2_1, S_E);
            }
            const sp<R> S_2_1 = fprop(Kn.qc[6], Kn.mc[6], tS_2_1);
            sp<R> tS_0_2_1;
            if constexpr (SH) {
              if constexpr (true) tS_0_2_1 = Y0_2__1; else tS_0_2_1 = slash(J0_2, S_1);
              if constexpr (true) spadd(tS_0_2_1, Y0_2_1__E); else slash_acc(tS_0_2_1, js.get(1), S_E);
              slash_acc(tS_0_2_1, E0, S_2_1);  // single-gluon term, fused
            } else {
              tS_0_2_1 = slash(E0, S_2_1);
              slash_acc(tS_0_2_1, J0_2, S_1);
              slash_acc(tS_0_2_1, js.get(1), S_E);
            }
            const sp<R> S_0_2_1 = fprop(Kn.qc[7], Kn.mc[7], tS_0_2_1);
            sp<R> X19;
            [[maybe_unused]] sp<R> Y0_3__2_1;  // Jslash(0,3) psi(2_1)
            [[maybe_unused]] sp<R> Y2_0_3__1;  // Jslash(2,0,3) psi(1)
            [[maybe_unused]] sp<R> Y1_2_0_3__E;  // Jslash(1,2,0,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y0_3__2_1 = slash(J0_3, S_2_1);
              if constexpr (true) X19 = spneg(Y0_3__2_1); else X19 = slash(J3_0, S_2_1);
              if constexpr (true) Y2_0_3__1 = slash(js.get(10), S_1);
              if constexpr (true) spadd(X19, Y2_0_3__1); else slash_acc(X19, js.get(10), S_1);
              if constexpr (true) Y1_2_0_3__E = slash(js.get(20), S_E);
              if constexpr (true) spsub(X19, Y1_2_0_3__E); else slash_acc(X19, neg(js.get(20)), S_E);
              slash_acc(X19, E3, S_0_2_1);  // single-gluon term, fused
            } else {
              X19 = slash(E3, S_0_2_1);
              slash_acc(X19, J3_0, S_2_1);
              slash_acc(X19, js.get(10), S_1);
              slash_acc(X19, neg(js.get(20)), S_E);
            }
            const cx<R> A19_0 = rowcol(X.ub[0], X19), A19_1 = rowcol(X.ub[1], X19);
            sp<R> tS_3_2_1;
            [[maybe_unused]] sp<R> Y2_3__1;  // Jslash(2,3) psi(1)
            [[maybe_unused]] sp<R> Y1_2_3__E;  // Jslash(1,2,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y2_3__1 = slash(J2_3, S_1);
              if constexpr (true) tS_3_2_1 = spneg(Y2_3__1); else tS_3_2_1 = slash(J3_2, S_1);
              if constexpr (true) Y1_2_3__E = slash(js.get(8), S_E);
              if constexpr (true) spadd(tS_3_2_1, Y1_2_3__E); else slash_acc(tS_3_2_1, js.get(8), S_E);
              slash_acc(tS_3_2_1, E3, S_2_1);  // single-gluon term, fused
            } else {
              tS_3_2_1 = slash(E3, S_2_1);
              slash_acc(tS_3_2_1, J3_2, S_1);
              slash_acc(tS_3_2_1, js.get(8), S_E);
            }
            const sp<R> S_3_2_1 = fprop(Kn.qc[14], Kn.mc[14], tS_3_2_1);
            sp<R> X5;
            if constexpr (SH) {
              if constexpr (true) X5 = Y0_3__2_1; else X5 = slash(J0_3, S_2_1);
              if constexpr (true) spadd(X5, Y0_3_2__1); else slash_acc(X5, js.get(6), S_1);
              if constexpr (true) spadd(X5, Y0_3_2_1__E); else slash_acc(X5, js.get(17), S_E);
              slash_acc(X5, E0, S_3_2_1);  // single-gluon term, fused
            } else {
              X5 = slash(E0, S_3_2_1);
              slash_acc(X5, J0_3, S_2_1);
              slash_acc(X5, js.get(6), S_1);
              slash_acc(X5, js.get(17), S_E);
            }
            const cx<R> A5_0 = rowcol(X.ub[0], X5), A5_1 = rowcol(X.ub[1], X5);
            sp<R> tS_3_1;
            [[maybe_unused]] sp<R> Y1_3__E;  // Jslash(1,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y1_3__E = slash(J1_3, S_E);
              if constexpr (true) tS_3_1 = spneg(Y1_3__E); else tS_3_1 = slash(J3_1, S_E);
              slash_acc(tS_3_1, E3, S_1);  // single-gluon term, fused
            } else {
              tS_3_1 = slash(E3, S_1);
              slash_acc(tS_3_1, J3_1, S_E);
            }
            const sp<R> S_3_1 = fprop(Kn.qc[10], Kn.mc[10], tS_3_1);
            sp<R> tS_0_3_1;
            if constexpr (SH) {
              if constexpr (true) tS_0_3_1 = Y0_3__1; else tS_0_3_1 = slash(J0_3, S_1);
              if constexpr (true) spadd(tS_0_3_1, Y0_3_1__E); else slash_acc(tS_0_3_1, js.get(5), S_E);
              slash_acc(tS_0_3_1, E0, S_3_1);  // single-gluon term, fused
            } else {
              tS_0_3_1 = slash(E0, S_3_1);
              slash_acc(tS_0_3_1, J0_3, S_1);
              slash_acc(tS_0_3_1, js.get(5), S_E);
            }
            const sp<R> S_0_3_1 = fprop(Kn.qc[11], Kn.mc[11], tS_0_3_1);
            sp<R> X13;
            [[maybe_unused]] sp<R> Y0_2__3_1;  // Jslash(0,2) psi(3_1)
            [[maybe_unused]] sp<R> Y1_3_0_2__E;  // Jslash(1,3,0,2) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y0_2__3_1 = slash(J0_2, S_3_1);
              if constexpr (true) X13 = spneg(Y0_2__3_1); else X13 = slash(J2_0, S_3_1);
              if constexpr (true) spadd(X13, Y2_0_3__1); else slash_acc(X13, js.get(10), S_1);
              if constexpr (true) Y1_3_0_2__E = slash(js.get(21), S_E);
              if constexpr (true) spsub(X13, Y1_3_0_2__E); else slash_acc(X13, neg(js.get(21)), S_E);
              slash_acc(X13, E2, S_0_3_1);  // single-gluon term, fused
            } else {
              X13 = slash(E2, S_0_3_1);
              slash_acc(X13, J2_0, S_3_1);
              slash_acc(X13, js.get(10), S_1);
              slash_acc(X13, neg(js.get(21)), S_E);
            }
            const cx<R> A13_0 = rowcol(X.ub[0], X13), A13_1 = rowcol(X.ub[1], X13);
            sp<R> tS_2_3_1;
            [[maybe_unused]] sp<R> Y1_3_2__E;  // Jslash(1,3,2) psi(E)
            if constexpr (SH) {
              if constexpr (true) tS_2_3_1 = Y2_3__1; else tS_2_3_1 = slash(J2_3, S_1);
              if constexpr (true) Y1_3_2__E = slash(js.get(9), S_E);
              if constexpr (true) spadd(tS_2_3_1, Y1_3_2__E); else slash_acc(tS_2_3_1, js.get(9), S_E);
              slash_acc(tS_2_3_1, E2, S_3_1);  // single-gluon term, fused
            } else {
              tS_2_3_1 = slash(E2, S_3_1);
              slash_acc(tS_2_3_1, J2_3, S_1);
              slash_acc(tS_2_3_1, js.get(9), S_E);
            }
            const sp<R> S_2_3_1 = fprop(Kn.qc[14], Kn.mc[14], tS_2_3_1);
            sp<R> X3;
            if constexpr (SH) {
              if constexpr (true) X3 = Y0_2__3_1; else X3 = slash(J0_2, S_3_1);
              if constexpr (true) spadd(X3, Y0_2_3__1); else slash_acc(X3, js.get(4), S_1);
              if constexpr (true) spadd(X3, Y0_2_3_1__E); else slash_acc(X3, js.get(15), S_E);
              slash_acc(X3, E0, S_2_3_1);  // single-gluon term, fused
            } else {
              X3 = slash(E0, S_2_3_1);
              slash_acc(X3, J0_2, S_3_1);
              slash_acc(X3, js.get(4), S_1);
              slash_acc(X3, js.get(15), S_E);
            }
            const cx<R> A3_0 = rowcol(X.ub[0], X3), A3_1 = rowcol(X.ub[1], X3);
            sp<R> tS_2 = slash(E2, S_E);
            const sp<R> S_2 = fprop(Kn.qc[4], Kn.mc[4], tS_2);
            sp<R> tS_0_2;
            if constexpr (SH) {
              if constexpr (true) tS_0_2 = Y0_2__E; else tS_0_2 = slash(J0_2, S_E);
              slash_acc(tS_0_2, E0, S_2);  // single-gluon term, fused
            } else {
              tS_0_2 = slash(E0, S_2);
              slash_acc(tS_0_2, J0_2, S_E);
            }
            const sp<R> S_0_2 = fprop(Kn.qc[5], Kn.mc[5], tS_0_2);
            sp<R> tS_1_0_2;
            [[maybe_unused]] sp<R> Y0_1__2;  // Jslash(0,1) psi(2)
            if constexpr (SH) {
              if constexpr (true) Y0_1__2 = slash(J0_1, S_2);
              if constexpr (true) tS_1_0_2 = spneg(Y0_1__2); else tS_1_0_2 = slash(J1_0, S_2);
              if constexpr (true) spadd(tS_1_0_2, Y1_0_2__E); else slash_acc(tS_1_0_2, js.get(2), S_E);
              slash_acc(tS_1_0_2, E1, S_0_2);  // single-gluon term, fused
            } else {
              tS_1_0_2 = slash(E1, S_0_2);
              slash_acc(tS_1_0_2, J1_0, S_2);
              slash_acc(tS_1_0_2, js.get(2), S_E);
            }
            const sp<R> S_1_0_2 = fprop(Kn.qc[7], Kn.mc[7], tS_1_0_2);
            sp<R> X20;
            [[maybe_unused]] sp<R> Y1_3__0_2;  // Jslash(1,3) psi(0_2)
            [[maybe_unused]] sp<R> Y0_1_3__2;  // Jslash(0,1,3) psi(2)
            [[maybe_unused]] sp<R> Y2_0_1_3__E;  // Jslash(2,0,1,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y1_3__0_2 = slash(J1_3, S_0_2);
              if constexpr (true) X20 = spneg(Y1_3__0_2); else X20 = slash(J3_1, S_0_2);
              if constexpr (true) Y0_1_3__2 = slash(js.get(3), S_2);
              if constexpr (true) spadd(X20, Y0_1_3__2); else slash_acc(X20, js.get(3), S_2);
              if constexpr (true) Y2_0_1_3__E = slash(js.get(22), S_E);
              if constexpr (true) spsub(X20, Y2_0_1_3__E); else slash_acc(X20, neg(js.get(22)), S_E);
              slash_acc(X20, E3, S_1_0_2);  // single-gluon term, fused
            } else {
              X20 = slash(E3, S_1_0_2);
              slash_acc(X20, J3_1, S_0_2);
              slash_acc(X20, js.get(3), S_2);
              slash_acc(X20, neg(js.get(22)), S_E);
            }
            const cx<R> A20_0 = rowcol(X.ub[0], X20), A20_1 = rowcol(X.ub[1], X20);
            sp<R> tS_3_0_2;
            [[maybe_unused]] sp<R> Y0_3__2;  // Jslash(0,3) psi(2)
            [[maybe_unused]] sp<R> Y2_0_3__E;  // Jslash(2,0,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y0_3__2 = slash(J0_3, S_2);
              if constexpr (true) tS_3_0_2 = spneg(Y0_3__2); else tS_3_0_2 = slash(J3_0, S_2);
              if constexpr (true) Y2_0_3__E = slash(js.get(10), S_E);
              if constexpr (true) spadd(tS_3_0_2, Y2_0_3__E); else slash_acc(tS_3_0_2, js.get(10), S_E);
              slash_acc(tS_3_0_2, E3, S_0_2);  // single-gluon term, fused
            } else {
              tS_3_0_2 = slash(E3, S_0_2);
              slash_acc(tS_3_0_2, J3_0, S_2);
              slash_acc(tS_3_0_2, js.get(10), S_E);
            }
            const sp<R> S_3_0_2 = fprop(Kn.qc[13], Kn.mc[13], tS_3_0_2);
            sp<R> X10;
            [[maybe_unused]] sp<R> Y0_3_1__2;  // Jslash(0,3,1) psi(2)
            if constexpr (SH) {
              if constexpr (true) X10 = Y1_3__0_2; else X10 = slash(J1_3, S_0_2);
              if constexpr (true) Y0_3_1__2 = slash(js.get(5), S_2);
              if constexpr (true) spadd(X10, Y0_3_1__2); else slash_acc(X10, js.get(5), S_2);
              if constexpr (true) spadd(X10, Y1_3_0_2__E); else slash_acc(X10, js.get(21), S_E);
              slash_acc(X10, E1, S_3_0_2);  // single-gluon term, fused
            } else {
              X10 = slash(E1, S_3_0_2);
              slash_acc(X10, J1_3, S_0_2);
              slash_acc(X10, js.get(5), S_2);
              slash_acc(X10, js.get(21), S_E);
            }
            const cx<R> A10_0 = rowcol(X.ub[0], X10), A10_1 = rowcol(X.ub[1], X10);
            sp<R> tS_1_2;
            if constexpr (SH) {
              if constexpr (true) tS_1_2 = Y1_2__E; else tS_1_2 = slash(J1_2, S_E);
              slash_acc(tS_1_2, E1, S_2);  // single-gluon term, fused
            } else {
              tS_1_2 = slash(E1, S_2);
              slash_acc(tS_1_2, J1_2, S_E);
            }
            const sp<R> S_1_2 = fprop(Kn.qc[6], Kn.mc[6], tS_1_2);
            sp<R> tS_0_1_2;
            if constexpr (SH) {
              if constexpr (true) tS_0_1_2 = Y0_1__2; else tS_0_1_2 = slash(J0_1, S_2);
              if constexpr (true) spadd(tS_0_1_2, Y0_1_2__E); else slash_acc(tS_0_1_2, js.get(0), S_E);
              slash_acc(tS_0_1_2, E0, S_1_2);  // single-gluon term, fused
            } else {
              tS_0_1_2 = slash(E0, S_1_2);
              slash_acc(tS_0_1_2, J0_1, S_2);
              slash_acc(tS_0_1_2, js.get(0), S_E);
            }
            const sp<R> S_0_1_2 = fprop(Kn.qc[7], Kn.mc[7], tS_0_1_2);
            sp<R> X18;
            [[maybe_unused]] sp<R> Y0_3__1_2;  // Jslash(0,3) psi(1_2)
            [[maybe_unused]] sp<R> Y1_0_3__2;  // Jslash(1,0,3) psi(2)
            [[maybe_unused]] sp<R> Y2_1_0_3__E;  // Jslash(2,1,0,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y0_3__1_2 = slash(J0_3, S_1_2);
              if constexpr (true) X18 = spneg(Y0_3__1_2); else X18 = slash(J3_0, S_1_2);
              if constexpr (true) Y1_0_3__2 = slash(js.get(7), S_2);
              if constexpr (true) spadd(X18, Y1_0_3__2); else slash_acc(X18, js.get(7), S_2);
              if constexpr (true) Y2_1_0_3__E = slash(js.get(23), S_E);
              if constexpr (true) spsub(X18, Y2_1_0_3__E); else slash_acc(X18, neg(js.get(23)), S_E);
              slash_acc(X18, E3, S_0_1_2);  // single-gluon term, fused
            } else {
              X18 = slash(E3, S_0_1_2);
              slash_acc(X18, J3_0, S_1_2);
              slash_acc(X18, js.get(7), S_2);
              slash_acc(X18, neg(js.get(23)), S_E);
            }
            const cx<R> A18_0 = rowcol(X.ub[0], X18), A18_1 = rowcol(X.ub[1], X18);
            sp<R> tS_3_1_2;
            [[maybe_unused]] sp<R> Y1_3__2;  // Jslash(1,3) psi(2)
            [[maybe_unused]] sp<R> Y2_1_3__E;  // Jslash(2,1,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y1_3__2 = slash(J1_3, S_2);
              if constexpr (true) tS_3_1_2 = spneg(Y1_3__2); else tS_3_1_2 = slash(J3_1, S_2);
              if constexpr (true) Y2_1_3__E = slash(js.get(11), S_E);
              if constexpr (true) spadd(tS_3_1_2, Y2_1_3__E); else slash_acc(tS_3_1_2, js.get(11), S_E);
              slash_acc(tS_3_1_2, E3, S_1_2);  // single-gluon term, fused
            } else {
              tS_3_1_2 = slash(E3, S_1_2);
              slash_acc(tS_3_1_2, J3_1, S_2);
              slash_acc(tS_3_1_2, js.get(11), S_E);
            }
            const sp<R> S_3_1_2 = fprop(Kn.qc[14], Kn.mc[14], tS_3_1_2);
            sp<R> X4;
            if constexpr (SH) {
              if constexpr (true) X4 = Y0_3__1_2; else X4 = slash(J0_3, S_1_2);
              if constexpr (true) spadd(X4, Y0_3_1__2); else slash_acc(X4, js.get(5), S_2);
              if constexpr (true) spadd(X4, Y0_3_1_2__E); else slash_acc(X4, js.get(16), S_E);
              slash_acc(X4, E0, S_3_1_2);  // single-gluon term, fused
            } else {
              X4 = slash(E0, S_3_1_2);
              slash_acc(X4, J0_3, S_1_2);
              slash_acc(X4, js.get(5), S_2);
              slash_acc(X4, js.get(16), S_E);
            }
            const cx<R> A4_0 = rowcol(X.ub[0], X4), A4_1 = rowcol(X.ub[1], X4);
            sp<R> tS_3_2;
            [[maybe_unused]] sp<R> Y2_3__E;  // Jslash(2,3) psi(E)
            if constexpr (SH) {
              if constexpr (true) Y2_3__E = slash(J2_3, S_E);
              if constexpr (true) tS_3_2 = spneg(Y2_3__E); else tS_3_2 = slash(J3_2, S_E);
              slash_acc(tS_3_2, E3, S_2);  // single-gluon term, fused
            } else {
              tS_3_2 = slash(E3, S_2);
              slash_acc(tS_3_2, J3_2, S_E);
            }
            const sp<R> S_3_2 = fprop(Kn.qc[12], Kn.mc[12], tS_3_2);
            sp<R> tS_0_3_2;
            if constexpr (SH) {
              if constexpr (true) tS_0_3_2 = Y0_3__2; else tS_0_3_2 = slash(J0_3, S_2);
              if constexpr (true) spadd(tS_0_3_2, Y0_3_2__E); else slash_acc(tS_0_3_2, js.get(6), S_E);
              slash_acc(tS_0_3_2, E0, S_3_2);  // single-gluon term, fused
            } else {
              tS_0_3_2 = slash(E0, S_3_2);
              slash_acc(tS_0_3_2, J0_3, S_2);
              slash_acc(tS_0_3_2, js.get(6), S_E);
            }
            const sp<R> S_0_3_2 = fprop(Kn.qc[13], Kn.mc[13], tS_0_3_2);
            sp<R> X7;
            [[maybe_unused]] sp<R> Y0_1__3_2;  // Jslash(0,1) psi(3_2)
            if constexpr (SH) {
              if constexpr (true) Y0_1__3_2 = slash(J0_1, S_3_2);
              if constexpr (true) X7 = spneg(Y0_1__3_2); else X7 = slash(J1_0, S_3_2);
              if constexpr (true) spadd(X7, Y1_0_3__2); else slash_acc(X7, js.get(7), S_2);
              if constexpr (true) spadd(X7, Y1_0_3_2__E); else slash_acc(X7, js.get(19), S_E);
              slash_acc(X7, E1, S_0_3_2);  // single-gluon term, fused
            } else {
              X7 = slash(E1, S_0_3_2);
              slash_acc(X7, J1_0, S_3_2);
              slash_acc(X7, js.get(7), S_2);
              slash_acc(X7, js.get(19), S_E);
            }
            const cx<R> A7_0 = rowcol(X.ub[0], X7), A7_1 = rowcol(X.ub[1], X7);
            sp<R> tS_1_3_2;
            if constexpr (SH) {
              if constexpr (true) tS_1_3_2 = Y1_3__2; else tS_1_3_2 = slash(J1_3, S_2);
              if constexpr (true) spadd(tS_1_3_2, Y1_3_2__E); else slash_acc(tS_1_3_2, js.get(9), S_E);
              slash_acc(tS_1_3_2, E1, S_3_2);  // single-gluon term, fused
            } else {
              tS_1_3_2 = slash(E1, S_3_2);
              slash_acc(tS_1_3_2, J1_3, S_2);
              slash_acc(tS_1_3_2, js.get(9), S_E);
            }
            const sp<R> S_1_3_2 = fprop(Kn.qc[14], Kn.mc[14], tS_1_3_2);
            sp<R> X1;
            if constexpr (SH) {
              if constexpr (true) X1 = Y0_1__3_2; else X1 = slash(J0_1, S_3_2);
              if constexpr (true) spadd(X1, Y0_1_3__2); else slash_acc(X1, js.get(3), S_2);
              if constexpr (true) spadd(X1, Y0_1_3_2__E); else slash_acc(X1, js.get(13), S_E);
              slash_acc(X1, E0, S_1_3_2);  // single-gluon term, fused
            } else {
              X1 = slash(E0, S_1_3_2);
              slash_acc(X1, J0_1, S_3_2);
              slash_acc(X1, js.get(3), S_2);
              slash_acc(X1, js.get(13), S_E);
            }
            const cx<R> A1_0 = rowcol(X.ub[0], X1), A1_1 = rowcol(X.ub[1], X1);
            sp<R> tS_3 = slash(E3, S_E);
            const sp<R> S_3 = fprop(Kn.qc[8], Kn.mc[8], tS_3);
            sp<R> tS_0_3;
            if constexpr (SH) {
              if constexpr (true) tS_0_3 = Y0_3__E; else tS_0_3 = slash(J0_3, S_E);
              slash_acc(tS_0_3, E0, S_3);  // single-gluon term, fused
            } else {
              tS_0_3 = slash(E0, S_3);
              slash_acc(tS_0_3, J0_3, S_E);
            }
            const sp<R> S_0_3 = fprop(Kn.qc[9], Kn.mc[9], tS_0_3);
            sp<R> tS_1_0_3;
            [[maybe_unused]] sp<R> Y0_1__3;  // Jslash(0,1) psi(3)
            if constexpr (SH) {
              if constexpr (true) Y0_1__3 = slash(J0_1, S_3);
              if constexpr (true) tS_1_0_3 = spneg(Y0_1__3); else tS_1_0_3 = slash(J1_0, S_3);
              if constexpr (true) spadd(tS_1_0_3, Y1_0_3__E); else slash_acc(tS_1_0_3, js.get(7), S_E);
              slash_acc(tS_1_0_3, E1, S_0_3);  // single-gluon term, fused
            } else {
              tS_1_0_3 = slash(E1, S_0_3);
              slash_acc(tS_1_0_3, J1_0, S_3);
              slash_acc(tS_1_0_3, js.get(7), S_E);
            }
            const sp<R> S_1_0_3 = fprop(Kn.qc[11], Kn.mc[11], tS_1_0_3);
            sp<R> X14;
            [[maybe_unused]] sp<R> Y1_2__0_3;  // Jslash(1,2) psi(0_3)
            [[maybe_unused]] sp<R> Y0_1_2__3;  // Jslash(0,1,2) psi(3)
            if constexpr (SH) {
              if constexpr (true) Y1_2__0_3 = slash(J1_2, S_0_3);
              if constexpr (true) X14 = spneg(Y1_2__0_3); else X14 = slash(J2_1, S_0_3);
              if constexpr (true) Y0_1_2__3 = slash(js.get(0), S_3);
              if constexpr (true) spadd(X14, Y0_1_2__3); else slash_acc(X14, js.get(0), S_3);
              if constexpr (true) spadd(X14, Y2_1_0_3__E); else slash_acc(X14, js.get(23), S_E);
              slash_acc(X14, E2, S_1_0_3);  // single-gluon term, fused
            } else {
              X14 = slash(E2, S_1_0_3);
              slash_acc(X14, J2_1, S_0_3);
              slash_acc(X14, js.get(0), S_3);
              slash_acc(X14, js.get(23), S_E);
            }
            const cx<R> A14_0 = rowcol(X.ub[0], X14), A14_1 = rowcol(X.ub[1], X14);
            sp<R> tS_2_0_3;
            [[maybe_unused]] sp<R> Y0_2__3;  // Jslash(0,2) psi(3)
            if constexpr (SH) {
              if constexpr (true) Y0_2__3 = slash(J0_2, S_3);
              if constexpr (true) tS_2_0_3 = spneg(Y0_2__3); else tS_2_0_3 = slash(J2_0, S_3);
              if constexpr (true) spadd(tS_2_0_3, Y2_0_3__E); else slash_acc(tS_2_0_3, js.get(10), S_E);
              slash_acc(tS_2_0_3, E2, S_0_3);  // single-gluon term, fused
            } else {
              tS_2_0_3 = slash(E2, S_0_3);
              slash_acc(tS_2_0_3, J2_0, S_3);
              slash_acc(tS_2_0_3, js.get(10), S_E);
            }
            const sp<R> S_2_0_3 = fprop(Kn.qc[13], Kn.mc[13], tS_2_0_3);
            sp<R> X8;
            [[maybe_unused]] sp<R> Y0_2_1__3;  // Jslash(0,2,1) psi(3)
            if constexpr (SH) {
              if constexpr (true) X8 = Y1_2__0_3; else X8 = slash(J1_2, S_0_3);
              if constexpr (true) Y0_2_1__3 = slash(js.get(1), S_3);
              if constexpr (true) spadd(X8, Y0_2_1__3); else slash_acc(X8, js.get(1), S_3);
              if constexpr (true) spadd(X8, Y1_2_0_3__E); else slash_acc(X8, js.get(20), S_E);
              slash_acc(X8, E1, S_2_0_3);  // single-gluon term, fused
            } else {
              X8 = slash(E1, S_2_0_3);
              slash_acc(X8, J1_2, S_0_3);
              slash_acc(X8, js.get(1), S_3);
              slash_acc(X8, js.get(20), S_E);
            }
            const cx<R> A8_0 = rowcol(X.ub[0], X8), A8_1 = rowcol(X.ub[1], X8);
            sp<R> tS_1_3;
            if constexpr (SH) {
              if constexpr (true) tS_1_3 = Y1_3__E; else tS_1_3 = slash(J1_3, S_E);
              slash_acc(tS_1_3, E1, S_3);  // single-gluon term, fused
            } else {
              tS_1_3 = slash(E1, S_3);
              slash_acc(tS_1_3, J1_3, S_E);
            }
            const sp<R> S_1_3 = fprop(Kn.qc[10], Kn.mc[10], tS_1_3);
            sp<R> tS_0_1_3;
            if constexpr (SH) {
              if constexpr (true) tS_0_1_3 = Y0_1__3; else tS_0_1_3 = slash(J0_1, S_3);
              if constexpr (true) spadd(tS_0_1_3, Y0_1_3__E); else slash_acc(tS_0_1_3, js.get(3), S_E);
              slash_acc(tS_0_1_3, E0, S_1_3);  // single-gluon term, fused
            } else {
              tS_0_1_3 = slash(E0, S_1_3);
              slash_acc(tS_0_1_3, J0_1, S_3);
              slash_acc(tS_0_1_3, js.get(3), S_E);
            }
            const sp<R> S_0_1_3 = fprop(Kn.qc[11], Kn.mc[11], tS_0_1_3);
            sp<R> X12;
            [[maybe_unused]] sp<R> Y0_2__1_3;  // Jslash(0,2) psi(1_3)
            [[maybe_unused]] sp<R> Y1_0_2__3;  // Jslash(1,0,2) psi(3)
            if constexpr (SH) {
              if constexpr (true) Y0_2__1_3 = slash(J0_2, S_1_3);
              if constexpr (true) X12 = spneg(Y0_2__1_3); else X12 = slash(J2_0, S_1_3);
              if constexpr (true) Y1_0_2__3 = slash(js.get(2), S_3);
              if constexpr (true) spadd(X12, Y1_0_2__3); else slash_acc(X12, js.get(2), S_3);
              if constexpr (true) spadd(X12, Y2_0_1_3__E); else slash_acc(X12, js.get(22), S_E);
              slash_acc(X12, E2, S_0_1_3);  // single-gluon term, fused
            } else {
              X12 = slash(E2, S_0_1_3);
              slash_acc(X12, J2_0, S_1_3);
              slash_acc(X12, js.get(2), S_3);
              slash_acc(X12, js.get(22), S_E);
            }
            const cx<R> A12_0 = rowcol(X.ub[0], X12), A12_1 = rowcol(X.ub[1], X12);
            sp<R> tS_2_1_3;
            [[maybe_unused]] sp<R> Y1_2__3;  // Jslash(1,2) psi(3)
            if constexpr (SH) {
              if constexpr (true) Y1_2__3 = slash(J1_2, S_3);
              if constexpr (true) tS_2_1_3 = spneg(Y1_2__3); else tS_2_1_3 = slash(J2_1, S_3);
              if constexpr (true) spadd(tS_2_1_3, Y2_1_3__E); else slash_acc(tS_2_1_3, js.get(11), S_E);
              slash_acc(tS_2_1_3, E2, S_1_3);  // single-gluon term, fused
            } else {
              tS_2_1_3 = slash(E2, S_1_3);
              slash_acc(tS_2_1_3, J2_1, S_3);
              slash_acc(tS_2_1_3, js.get(11), S_E);
            }
            const sp<R> S_2_1_3 = fprop(Kn.qc[14], Kn.mc[14], tS_2_1_3);
            sp<R> X2;
            if constexpr (SH) {
              if constexpr (true) X2 = Y0_2__1_3; else X2 = slash(J0_2, S_1_3);
              if constexpr (true) spadd(X2, Y0_2_1__3); else slash_acc(X2, js.get(1), S_3);
              if constexpr (true) spadd(X2, Y0_2_1_3__E); else slash_acc(X2, js.get(14), S_E);
              slash_acc(X2, E0, S_2_1_3);  // single-gluon term, fused
            } else {
              X2 = slash(E0, S_2_1_3);
              slash_acc(X2, J0_2, S_1_3);
              slash_acc(X2, js.get(1), S_3);
              slash_acc(X2, js.get(14), S_E);
            }
            const cx<R> A2_0 = rowcol(X.ub[0], X2), A2_1 = rowcol(X.ub[1], X2);
            sp<R> tS_2_3;
            if constexpr (SH) {
              if constexpr (true) tS_2_3 = Y2_3__E; else tS_2_3 = slash(J2_3, S_E);
              slash_acc(tS_2_3, E2, S_3);  // single-gluon term, fused
            } else {
              tS_2_3 = slash(E2, S_3);
              slash_acc(tS_2_3, J2_3, S_E);
            }
            const sp<R> S_2_3 = fprop(Kn.qc[12], Kn.mc[12], tS_2_3);
            sp<R> tS_0_2_3;
            if constexpr (SH) {
              if constexpr (true) tS_0_2_3 = Y0_2__3; else tS_0_2_3 = slash(J0_2, S_3);
              if constexpr (true) spadd(tS_0_2_3, Y0_2_3__E); else slash_acc(tS_0_2_3, js.get(4), S_E);
              slash_acc(tS_0_2_3, E0, S_2_3);  // single-gluon term, fused
            } else {
              tS_0_2_3 = slash(E0, S_2_3);
              slash_acc(tS_0_2_3, J0_2, S_3);
              slash_acc(tS_0_2_3, js.get(4), S_E);
            }
            const sp<R> S_0_2_3 = fprop(Kn.qc[13], Kn.mc[13], tS_0_2_3);
            sp<R> X6;
            [[maybe_unused]] sp<R> Y0_1__2_3;  // Jslash(0,1) psi(2_3)
            if constexpr (SH) {
              if constexpr (true) Y0_1__2_3 = slash(J0_1, S_2_3);
              if constexpr (true) X6 = spneg(Y0_1__2_3); else X6 = slash(J1_0, S_2_3);
              if constexpr (true) spadd(X6, Y1_0_2__3); else slash_acc(X6, js.get(2), S_3);
              if constexpr (true) spadd(X6, Y1_0_2_3__E); else slash_acc(X6, js.get(18), S_E);
              slash_acc(X6, E1, S_0_2_3);  // single-gluon term, fused
            } else {
              X6 = slash(E1, S_0_2_3);
              slash_acc(X6, J1_0, S_2_3);
              slash_acc(X6, js.get(2), S_3);
              slash_acc(X6, js.get(18), S_E);
            }
            const cx<R> A6_0 = rowcol(X.ub[0], X6), A6_1 = rowcol(X.ub[1], X6);
            sp<R> tS_1_2_3;
            if constexpr (SH) {
              if constexpr (true) tS_1_2_3 = Y1_2__3; else tS_1_2_3 = slash(J1_2, S_3);
              if constexpr (true) spadd(tS_1_2_3, Y1_2_3__E); else slash_acc(tS_1_2_3, js.get(8), S_E);
              slash_acc(tS_1_2_3, E1, S_2_3);  // single-gluon term, fused
            } else {
              tS_1_2_3 = slash(E1, S_2_3);
              slash_acc(tS_1_2_3, J1_2, S_3);
              slash_acc(tS_1_2_3, js.get(8), S_E);
            }
            const sp<R> S_1_2_3 = fprop(Kn.qc[14], Kn.mc[14], tS_1_2_3);
            sp<R> X0;
            if constexpr (SH) {
              if constexpr (true) X0 = Y0_1__2_3; else X0 = slash(J0_1, S_2_3);
              if constexpr (true) spadd(X0, Y0_1_2__3); else slash_acc(X0, js.get(0), S_3);
              if constexpr (true) spadd(X0, Y0_1_2_3__E); else slash_acc(X0, js.get(12), S_E);
              slash_acc(X0, E0, S_1_2_3);  // single-gluon term, fused
            } else {
              X0 = slash(E0, S_1_2_3);
              slash_acc(X0, J0_1, S_2_3);
              slash_acc(X0, js.get(0), S_3);
              slash_acc(X0, js.get(12), S_E);
            }
            const cx<R> A0_0 = rowcol(X.ub[0], X0), A0_1 = rowcol(X.ub[1], X0);
            if constexpr (CM != CM_FMA) {
              const cx<float> Aa0[K] = {A0_0, A1_0, A2_0, A3_0, A4_0, A5_0, A6_0, A7_0, A8_0, A9_0, A10_0, A11_0, A12_0, A13_0, A14_0, A15_0, A16_0, A17_0, A18_0, A19_0, A20_0, A21_0, A22_0, A23_0};
              const cx<float> Aa1[K] = {A0_1, A1_1, A2_1, A3_1, A4_1, A5_1, A6_1, A7_1, A8_1, A9_1, A10_1, A11_1, A12_1, A13_1, A14_1, A15_1, A16_1, A17_1, A18_1, A19_1, A20_1, A21_1, A22_1, A23_1};
              if constexpr (MMA) {
                acc += R(2) * (cmma.sum(Aa0) + cmma.sum(Aa1));  // x2 helicity flip
              } else {
                sink->put(Aa0);
                sink->put(Aa1);
              }
            } else {
              { const R zr = R(1024) * A0_0.r + R(-256) * A1_0.r + R(-256) * A2_0.r + R(32) * A3_0.r + R(32) * A4_0.r + R(320) * A5_0.r + R(-256) * A6_0.r + R(32) * A7_0.r + R(32) * A8_0.r + R(-4) * A9_0.r + R(-4) * A10_0.r + R(-40) * A11_0.r + R(32) * A12_0.r + R(-4) * A13_0.r + R(320) * A14_0.r + R(-40) * A15_0.r + R(284) * A16_0.r + R(248) * A17_0.r + R(-4) * A18_0.r + R(-40) * A19_0.r + R(-40) * A20_0.r + R(248) * A21_0.r + R(248) * A22_0.r + R(-112) * A23_0.r; const R zi = R(1024) * A0_0.i + R(-256) * A1_0.i + R(-256) * A2_0.i + R(32) * A3_0.i + R(32) * A4_0.i + R(320) * A5_0.i + R(-256) * A6_0.i + R(32) * A7_0.i + R(32) * A8_0.i + R(-4) * A9_0.i + R(-4) * A10_0.i + R(-40) * A11_0.i + R(32) * A12_0.i + R(-4) * A13_0.i + R(320) * A14_0.i + R(-40) * A15_0.i + R(284) * A16_0.i + R(248) * A17_0.i + R(-4) * A18_0.i + R(-40) * A19_0.i + R(-40) * A20_0.i + R(248) * A21_0.i + R(248) * A22_0.i + R(-112) * A23_0.i;
                cz0_0 = fmadd(A0_0.r, zr, fmadd(A0_0.i, zi, cz0_0)); }
              { const R zr = R(1024) * A1_0.r + R(32) * A2_0.r + R(320) * A3_0.r + R(-256) * A4_0.r + R(32) * A5_0.r + R(32) * A6_0.r + R(-256) * A7_0.r + R(-4) * A8_0.r + R(-40) * A9_0.r + R(32) * A10_0.r + R(-4) * A11_0.r + R(-4) * A12_0.r + R(-40) * A13_0.r + R(-40) * A14_0.r + R(248) * A15_0.r + R(248) * A16_0.r + R(-112) * A17_0.r + R(32) * A18_0.r + R(-4) * A19_0.r + R(320) * A20_0.r + R(-40) * A21_0.r + R(284) * A22_0.r + R(248) * A23_0.r; const R zi = R(1024) * A1_0.i + R(32) * A2_0.i + R(320) * A3_0.i + R(-256) * A4_0.i + R(32) * A5_0.i + R(32) * A6_0.i + R(-256) * A7_0.i + R(-4) * A8_0.i + R(-40) * A9_0.i + R(32) * A10_0.i + R(-4) * A11_0.i + R(-4) * A12_0.i + R(-40) * A13_0.i + R(-40) * A14_0.i + R(248) * A15_0.i + R(248) * A16_0.i + R(-112) * A17_0.i + R(32) * A18_0.i + R(-4) * A19_0.i + R(320) * A20_0.i + R(-40) * A21_0.i + R(284) * A22_0.i + R(248) * A23_0.i;
                cz0_1 = fmadd(A1_0.r, zr, fmadd(A1_0.i, zi, cz0_1)); }
              { const R zr = R(1024) * A2_0.r + R(-256) * A3_0.r + R(320) * A4_0.r + R(32) * A5_0.r + R(32) * A6_0.r + R(-4) * A7_0.r + R(320) * A8_0.r + R(-40) * A9_0.r + R(284) * A10_0.r + R(248) * A11_0.r + R(-256) * A12_0.r + R(32) * A13_0.r + R(32) * A14_0.r + R(-4) * A15_0.r + R(-4) * A16_0.r + R(-40) * A17_0.r + R(-40) * A18_0.r + R(-4) * A19_0.r + R(248) * A20_0.r + R(-112) * A21_0.r + R(-40) * A22_0.r + R(248) * A23_0.r; const R zi = R(1024) * A2_0.i + R(-256) * A3_0.i + R(320) * A4_0.i + R(32) * A5_0.i + R(32) * A6_0.i + R(-4) * A7_0.i + R(320) * A8_0.i + R(-40) * A9_0.i + R(284) * A10_0.i + R(248) * A11_0.i + R(-256) * A12_0.i + R(32) * A13_0.i + R(32) * A14_0.i + R(-4) * A15_0.i + R(-4) * A16_0.i + R(-40) * A17_0.i + R(-40) * A18_0.i + R(-4) * A19_0.i + R(248) * A20_0.i + R(-112) * A21_0.i + R(-40) * A22_0.i + R(248) * A23_0.i;
                cz0_2 = fmadd(A2_0.r, zr, fmadd(A2_0.i, zi, cz0_2)); }
              { const R zr = R(1024) * A3_0.r + R(32) * A4_0.r + R(-256) * A5_0.r + R(-4) * A6_0.r + R(-40) * A7_0.r + R(-40) * A8_0.r + R(248) * A9_0.r + R(248) * A10_0.r + R(-112) * A11_0.r + R(32) * A12_0.r + R(-256) * A13_0.r + R(-4) * A14_0.r + R(-40) * A15_0.r + R(32) * A16_0.r + R(-4) * A17_0.r + R(-4) * A18_0.r + R(32) * A19_0.r + R(284) * A20_0.r + R(248) * A21_0.r + R(320) * A22_0.r + R(-40) * A23_0.r; const R zi = R(1024) * A3_0.i + R(32) * A4_0.i + R(-256) * A5_0.i + R(-4) * A6_0.i + R(-40) * A7_0.i + R(-40) * A8_0.i + R(248) * A9_0.i + R(248) * A10_0.i + R(-112) * A11_0.i + R(32) * A12_0.i + R(-256) * A13_0.i + R(-4) * A14_0.i + R(-40) * A15_0.i + R(32) * A16_0.i + R(-4) * A17_0.i + R(-4) * A18_0.i + R(32) * A19_0.i + R(284) * A20_0.i + R(248) * A21_0.i + R(320) * A22_0.i + R(-40) * A23_0.i;
                cz0_3 = fmadd(A3_0.r, zr, fmadd(A3_0.i, zi, cz0_3)); }
              { const R zr = R(1024) * A4_0.r + R(-256) * A5_0.r + R(-4) * A6_0.r + R(32) * A7_0.r + R(284) * A8_0.r + R(248) * A9_0.r + R(320) * A10_0.r + R(-40) * A11_0.r + R(-40) * A12_0.r + R(-4) * A13_0.r + R(248) * A14_0.r + R(-112) * A15_0.r + R(-40) * A16_0.r + R(248) * A17_0.r + R(-256) * A18_0.r + R(32) * A19_0.r + R(32) * A20_0.r + R(-4) * A21_0.r + R(-4) * A22_0.r + R(-40) * A23_0.r; const R zi = R(1024) * A4_0.i + R(-256) * A5_0.i + R(-4) * A6_0.i + R(32) * A7_0.i + R(284) * A8_0.i + R(248) * A9_0.i + R(320) * A10_0.i + R(-40) * A11_0.i + R(-40) * A12_0.i + R(-4) * A13_0.i + R(248) * A14_0.i + R(-112) * A15_0.i + R(-40) * A16_0.i + R(248) * A17_0.i + R(-256) * A18_0.i + R(32) * A19_0.i + R(32) * A20_0.i + R(-4) * A21_0.i + R(-4) * A22_0.i + R(-40) * A23_0.i;
                cz0_0 = fmadd(A4_0.r, zr, fmadd(A4_0.i, zi, cz0_0)); }
              { const R zr = R(1024) * A5_0.r + R(-40) * A6_0.r + R(-4) * A7_0.r + R(248) * A8_0.r + R(-112) * A9_0.r + R(-40) * A10_0.r + R(248) * A11_0.r + R(-4) * A12_0.r + R(32) * A13_0.r + R(284) * A14_0.r + R(248) * A15_0.r + R(320) * A16_0.r + R(-40) * A17_0.r + R(32) * A18_0.r + R(-256) * A19_0.r + R(-4) * A20_0.r + R(-40) * A21_0.r + R(32) * A22_0.r + R(-4) * A23_0.r; const R zi = R(1024) * A5_0.i + R(-40) * A6_0.i + R(-4) * A7_0.i + R(248) * A8_0.i + R(-112) * A9_0.i + R(-40) * A10_0.i + R(248) * A11_0.i + R(-4) * A12_0.i + R(32) * A13_0.i + R(284) * A14_0.i + R(248) * A15_0.i + R(320) * A16_0.i + R(-40) * A17_0.i + R(32) * A18_0.i + R(-256) * A19_0.i + R(-4) * A20_0.i + R(-40) * A21_0.i + R(32) * A22_0.i + R(-4) * A23_0.i;
                cz0_1 = fmadd(A5_0.r, zr, fmadd(A5_0.i, zi, cz0_1)); }
              { const R zr = R(1024) * A6_0.r + R(-256) * A7_0.r + R(-256) * A8_0.r + R(32) * A9_0.r + R(32) * A10_0.r + R(320) * A11_0.r + R(320) * A12_0.r + R(-40) * A13_0.r + R(32) * A14_0.r + R(-4) * A15_0.r + R(248) * A16_0.r + R(284) * A17_0.r + R(-40) * A18_0.r + R(248) * A19_0.r + R(-4) * A20_0.r + R(-40) * A21_0.r + R(-112) * A22_0.r + R(248) * A23_0.r; const R zi = R(1024) * A6_0.i + R(-256) * A7_0.i + R(-256) * A8_0.i + R(32) * A9_0.i + R(32) * A10_0.i + R(320) * A11_0.i + R(320) * A12_0.i + R(-40) * A13_0.i + R(32) * A14_0.i + R(-4) * A15_0.i + R(248) * A16_0.i + R(284) * A17_0.i + R(-40) * A18_0.i + R(248) * A19_0.i + R(-4) * A20_0.i + R(-40) * A21_0.i + R(-112) * A22_0.i + R(248) * A23_0.i;
                cz0_2 = fmadd(A6_0.r, zr, fmadd(A6_0.i, zi, cz0_2)); }
              { const R zr = R(1024) * A7_0.r + R(32) * A8_0.r + R(320) * A9_0.r + R(-256) * A10_0.r + R(32) * A11_0.r + R(-40) * A12_0.r + R(248) * A13_0.r + R(-4) * A14_0.r + R(-40) * A15_0.r + R(-112) * A16_0.r + R(248) * A17_0.r + R(320) * A18_0.r + R(-40) * A19_0.r + R(32) * A20_0.r + R(-4) * A21_0.r + R(248) * A22_0.r + R(284) * A23_0.r; const R zi = R(1024) * A7_0.i + R(32) * A8_0.i + R(320) * A9_0.i + R(-256) * A10_0.i + R(32) * A11_0.i + R(-40) * A12_0.i + R(248) * A13_0.i + R(-4) * A14_0.i + R(-40) * A15_0.i + R(-112) * A16_0.i + R(248) * A17_0.i + R(320) * A18_0.i + R(-40) * A19_0.i + R(32) * A20_0.i + R(-4) * A21_0.i + R(248) * A22_0.i + R(284) * A23_0.i;
                cz0_3 = fmadd(A7_0.r, zr, fmadd(A7_0.i, zi, cz0_3)); }
              { const R zr = R(1024) * A8_0.r + R(-256) * A9_0.r + R(320) * A10_0.r + R(32) * A11_0.r + R(32) * A12_0.r + R(-4) * A13_0.r + R(-256) * A14_0.r + R(32) * A15_0.r + R(-40) * A16_0.r + R(-4) * A17_0.r + R(248) * A18_0.r + R(-112) * A19_0.r + R(-40) * A20_0.r + R(-4) * A21_0.r + R(248) * A22_0.r + R(-40) * A23_0.r; const R zi = R(1024) * A8_0.i + R(-256) * A9_0.i + R(320) * A10_0.i + R(32) * A11_0.i + R(32) * A12_0.i + R(-4) * A13_0.i + R(-256) * A14_0.i + R(32) * A15_0.i + R(-40) * A16_0.i + R(-4) * A17_0.i + R(248) * A18_0.i + R(-112) * A19_0.i + R(-40) * A20_0.i + R(-4) * A21_0.i + R(248) * A22_0.i + R(-40) * A23_0.i;
                cz0_0 = fmadd(A8_0.r, zr, fmadd(A8_0.i, zi, cz0_0)); }
              { const R zr = R(1024) * A9_0.r + R(32) * A10_0.r + R(-256) * A11_0.r + R(-4) * A12_0.r + R(-40) * A13_0.r + R(32) * A14_0.r + R(-256) * A15_0.r + R(-4) * A16_0.r + R(32) * A17_0.r + R(284) * A18_0.r + R(248) * A19_0.r + R(-4) * A20_0.r + R(32) * A21_0.r + R(-40) * A22_0.r + R(320) * A23_0.r; const R zi = R(1024) * A9_0.i + R(32) * A10_0.i + R(-256) * A11_0.i + R(-4) * A12_0.i + R(-40) * A13_0.i + R(32) * A14_0.i + R(-256) * A15_0.i + R(-4) * A16_0.i + R(32) * A17_0.i + R(284) * A18_0.i + R(248) * A19_0.i + R(-4) * A20_0.i + R(32) * A21_0.i + R(-40) * A22_0.i + R(320) * A23_0.i;
                cz0_1 = fmadd(A9_0.r, zr, fmadd(A9_0.i, zi, cz0_1)); }
              { const R zr = R(1024) * A10_0.r + R(-256) * A11_0.r + R(248) * A12_0.r + R(-112) * A13_0.r + R(-40) * A14_0.r + R(-4) * A15_0.r + R(248) * A16_0.r + R(-40) * A17_0.r + R(32) * A18_0.r + R(-4) * A19_0.r + R(-256) * A20_0.r + R(32) * A21_0.r + R(-40) * A22_0.r + R(-4) * A23_0.r; const R zi = R(1024) * A10_0.i + R(-256) * A11_0.i + R(248) * A12_0.i + R(-112) * A13_0.i + R(-40) * A14_0.i + R(-4) * A15_0.i + R(248) * A16_0.i + R(-40) * A17_0.i + R(32) * A18_0.i + R(-4) * A19_0.i + R(-256) * A20_0.i + R(32) * A21_0.i + R(-40) * A22_0.i + R(-4) * A23_0.i;
                cz0_2 = fmadd(A10_0.r, zr, fmadd(A10_0.i, zi, cz0_2)); }
              { const R zr = R(1024) * A11_0.r + R(284) * A12_0.r + R(248) * A13_0.r + R(-4) * A14_0.r + R(32) * A15_0.r + R(-40) * A16_0.r + R(320) * A17_0.r + R(-4) * A18_0.r + R(-40) * A19_0.r + R(32) * A20_0.r + R(-256) * A21_0.r + R(-4) * A22_0.r + R(32) * A23_0.r; const R zi = R(1024) * A11_0.i + R(284) * A12_0.i + R(248) * A13_0.i + R(-4) * A14_0.i + R(32) * A15_0.i + R(-40) * A16_0.i + R(320) * A17_0.i + R(-4) * A18_0.i + R(-40) * A19_0.i + R(32) * A20_0.i + R(-256) * A21_0.i + R(-4) * A22_0.i + R(32) * A23_0.i;
                cz0_3 = fmadd(A11_0.r, zr, fmadd(A11_0.i, zi, cz0_3)); }
              { const R zr = R(1024) * A12_0.r + R(-256) * A13_0.r + R(-256) * A14_0.r + R(32) * A15_0.r + R(32) * A16_0.r + R(320) * A17_0.r + R(248) * A18_0.r + R(-40) * A19_0.r + R(-112) * A20_0.r + R(248) * A21_0.r + R(-4) * A22_0.r + R(-40) * A23_0.r; const R zi = R(1024) * A12_0.i + R(-256) * A13_0.i + R(-256) * A14_0.i + R(32) * A15_0.i + R(32) * A16_0.i + R(320) * A17_0.i + R(248) * A18_0.i + R(-40) * A19_0.i + R(-112) * A20_0.i + R(248) * A21_0.i + R(-4) * A22_0.i + R(-40) * A23_0.i;
                cz0_0 = fmadd(A12_0.r, zr, fmadd(A12_0.i, zi, cz0_0)); }
              { const R zr = R(1024) * A13_0.r + R(32) * A14_0.r + R(320) * A15_0.r + R(-256) * A16_0.r + R(32) * A17_0.r + R(-40) * A18_0.r + R(320) * A19_0.r + R(248) * A20_0.r + R(284) * A21_0.r + R(32) * A22_0.r + R(-4) * A23_0.r; const R zi = R(1024) * A13_0.i + R(32) * A14_0.i + R(320) * A15_0.i + R(-256) * A16_0.i + R(32) * A17_0.i + R(-40) * A18_0.i + R(320) * A19_0.i + R(248) * A20_0.i + R(284) * A21_0.i + R(32) * A22_0.i + R(-4) * A23_0.i;
                cz0_1 = fmadd(A13_0.r, zr, fmadd(A13_0.i, zi, cz0_1)); }
              { const R zr = R(1024) * A14_0.r + R(-256) * A15_0.r + R(320) * A16_0.r + R(32) * A17_0.r + R(-112) * A18_0.r + R(248) * A19_0.r + R(248) * A20_0.r + R(-40) * A21_0.r + R(-40) * A22_0.r + R(-4) * A23_0.r; const R zi = R(1024) * A14_0.i + R(-256) * A15_0.i + R(320) * A16_0.i + R(32) * A17_0.i + R(-112) * A18_0.i + R(248) * A19_0.i + R(248) * A20_0.i + R(-40) * A21_0.i + R(-40) * A22_0.i + R(-4) * A23_0.i;
                cz0_2 = fmadd(A14_0.r, zr, fmadd(A14_0.i, zi, cz0_2)); }
              { const R zr = R(1024) * A15_0.r + R(32) * A16_0.r + R(-256) * A17_0.r + R(248) * A18_0.r + R(284) * A19_0.r + R(-40) * A20_0.r + R(320) * A21_0.r + R(-4) * A22_0.r + R(32) * A23_0.r; const R zi = R(1024) * A15_0.i + R(32) * A16_0.i + R(-256) * A17_0.i + R(248) * A18_0.i + R(284) * A19_0.i + R(-40) * A20_0.i + R(320) * A21_0.i + R(-4) * A22_0.i + R(32) * A23_0.i;
                cz0_3 = fmadd(A15_0.r, zr, fmadd(A15_0.i, zi, cz0_3)); }
              { const R zr = R(1024) * A16_0.r + R(-256) * A17_0.r + R(-4) * A18_0.r + R(32) * A19_0.r + R(-40) * A20_0.r + R(-4) * A21_0.r + R(-256) * A22_0.r + R(32) * A23_0.r; const R zi = R(1024) * A16_0.i + R(-256) * A17_0.i + R(-4) * A18_0.i + R(32) * A19_0.i + R(-40) * A20_0.i + R(-4) * A21_0.i + R(-256) * A22_0.i + R(32) * A23_0.i;
                cz0_0 = fmadd(A16_0.r, zr, fmadd(A16_0.i, zi, cz0_0)); }
              { const R zr = R(1024) * A17_0.r + R(-40) * A18_0.r + R(-4) * A19_0.r + R(-4) * A20_0.r + R(32) * A21_0.r + R(32) * A22_0.r + R(-256) * A23_0.r; const R zi = R(1024) * A17_0.i + R(-40) * A18_0.i + R(-4) * A19_0.i + R(-4) * A20_0.i + R(32) * A21_0.i + R(32) * A22_0.i + R(-256) * A23_0.i;
                cz0_1 = fmadd(A17_0.r, zr, fmadd(A17_0.i, zi, cz0_1)); }
              { const R zr = R(1024) * A18_0.r + R(-256) * A19_0.r + R(-256) * A20_0.r + R(32) * A21_0.r + R(32) * A22_0.r + R(320) * A23_0.r; const R zi = R(1024) * A18_0.i + R(-256) * A19_0.i + R(-256) * A20_0.i + R(32) * A21_0.i + R(32) * A22_0.i + R(320) * A23_0.i;
                cz0_2 = fmadd(A18_0.r, zr, fmadd(A18_0.i, zi, cz0_2)); }
              { const R zr = R(1024) * A19_0.r + R(32) * A20_0.r + R(320) * A21_0.r + R(-256) * A22_0.r + R(32) * A23_0.r; const R zi = R(1024) * A19_0.i + R(32) * A20_0.i + R(320) * A21_0.i + R(-256) * A22_0.i + R(32) * A23_0.i;
                cz0_3 = fmadd(A19_0.r, zr, fmadd(A19_0.i, zi, cz0_3)); }
              { const R zr = R(1024) * A20_0.r + R(-256) * A21_0.r + R(320) * A22_0.r + R(32) * A23_0.r; const R zi = R(1024) * A20_0.i + R(-256) * A21_0.i + R(320) * A22_0.i + R(32) * A23_0.i;
                cz0_0 = fmadd(A20_0.r, zr, fmadd(A20_0.i, zi, cz0_0)); }
              { const R zr = R(1024) * A21_0.r + R(32) * A22_0.r + R(-256) * A23_0.r; const R zi = R(1024) * A21_0.i + R(32) * A22_0.i + R(-256) * A23_0.i;
                cz0_1 = fmadd(A21_0.r, zr, fmadd(A21_0.i, zi, cz0_1)); }
              { const R zr = R(1024) * A22_0.r + R(-256) * A23_0.r; const R zi = R(1024) * A22_0.i + R(-256) * A23_0.i;
                cz0_2 = fmadd(A22_0.r, zr, fmadd(A22_0.i, zi, cz0_2)); }
              { const R zr = R(1024) * A23_0.r; const R zi = R(1024) * A23_0.i;
                cz0_3 = fmadd(A23_0.r, zr, fmadd(A23_0.i, zi, cz0_3)); }
              { const R zr = R(1024) * A0_1.r + R(-256) * A1_1.r + R(-256) * A2_1.r + R(32) * A3_1.r + R(32) * A4_1.r + R(320) * A5_1.r + R(-256) * A6_1.r + R(32) * A7_1.r + R(32) * A8_1.r + R(-4) * A9_1.r + R(-4) * A10_1.r + R(-40) * A11_1.r + R(32) * A12_1.r + R(-4) * A13_1.r + R(320) * A14_1.r + R(-40) * A15_1.r + R(284) * A16_1.r + R(248) * A17_1.r + R(-4) * A18_1.r + R(-40) * A19_1.r + R(-40) * A20_1.r + R(248) * A21_1.r + R(248) * A22_1.r + R(-112) * A23_1.r; const R zi = R(1024) * A0_1.i + R(-256) * A1_1.i + R(-256) * A2_1.i + R(32) * A3_1.i + R(32) * A4_1.i + R(320) * A5_1.i + R(-256) * A6_1.i + R(32) * A7_1.i + R(32) * A8_1.i + R(-4) * A9_1.i + R(-4) * A10_1.i + R(-40) * A11_1.i + R(32) * A12_1.i + R(-4) * A13_1.i + R(320) * A14_1.i + R(-40) * A15_1.i + R(284) * A16_1.i + R(248) * A17_1.i + R(-4) * A18_1.i + R(-40) * A19_1.i + R(-40) * A20_1.i + R(248) * A21_1.i + R(248) * A22_1.i + R(-112) * A23_1.i;
                cz1_0 = fmadd(A0_1.r, zr, fmadd(A0_1.i, zi, cz1_0)); }
              { const R zr = R(1024) * A1_1.r + R(32) * A2_1.r + R(320) * A3_1.r + R(-256) * A4_1.r + R(32) * A5_1.r + R(32) * A6_1.r + R(-256) * A7_1.r + R(-4) * A8_1.r + R(-40) * A9_1.r + R(32) * A10_1.r + R(-4) * A11_1.r + R(-4) * A12_1.r + R(-40) * A13_1.r + R(-40) * A14_1.r + R(248) * A15_1.r + R(248) * A16_1.r + R(-112) * A17_1.r + R(32) * A18_1.r + R(-4) * A19_1.r + R(320) * A20_1.r + R(-40) * A21_1.r + R(284) * A22_1.r + R(248) * A23_1.r; const R zi = R(1024) * A1_1.i + R(32) * A2_1.i + R(320) * A3_1.i + R(-256) * A4_1.i + R(32) * A5_1.i + R(32) * A6_1.i + R(-256) * A7_1.i + R(-4) * A8_1.i + R(-40) * A9_1.i + R(32) * A10_1.i + R(-4) * A11_1.i + R(-4) * A12_1.i + R(-40) * A13_1.i + R(-40) * A14_1.i + R(248) * A15_1.i + R(248) * A16_1.i + R(-112) * A17_1.i + R(32) * A18_1.i + R(-4) * A19_1.i + R(320) * A20_1.i + R(-40) * A21_1.i + R(284) * A22_1.i + R(248) * A23_1.i;
                cz1_1 = fmadd(A1_1.r, zr, fmadd(A1_1.i, zi, cz1_1)); }
              { const R zr = R(1024) * A2_1.r + R(-256) * A3_1.r + R(320) * A4_1.r + R(32) * A5_1.r + R(32) * A6_1.r + R(-4) * A7_1.r + R(320) * A8_1.r + R(-40) * A9_1.r + R(284) * A10_1.r + R(248) * A11_1.r + R(-256) * A12_1.r + R(32) * A13_1.r + R(32) * A14_1.r + R(-4) * A15_1.r + R(-4) * A16_1.r + R(-40) * A17_1.r + R(-40) * A18_1.r + R(-4) * A19_1.r + R(248) * A20_1.r + R(-112) * A21_1.r + R(-40) * A22_1.r + R(248) * A23_1.r; const R zi = R(1024) * A2_1.i + R(-256) * A3_1.i + R(320) * A4_1.i + R(32) * A5_1.i + R(32) * A6_1.i + R(-4) * A7_1.i + R(320) * A8_1.i + R(-40) * A9_1.i + R(284) * A10_1.i + R(248) * A11_1.i + R(-256) * A12_1.i + R(32) * A13_1.i + R(32) * A14_1.i + R(-4) * A15_1.i + R(-4) * A16_1.i + R(-40) * A17_1.i + R(-40) * A18_1.i + R(-4) * A19_1.i + R(248) * A20_1.i + R(-112) * A21_1.i + R(-40) * A22_1.i + R(248) * A23_1.i;
                cz1_2 = fmadd(A2_1.r, zr, fmadd(A2_1.i, zi, cz1_2)); }
              { const R zr = R(1024) * A3_1.r + R(32) * A4_1.r + R(-256) * A5_1.r + R(-4) * A6_1.r + R(-40) * A7_1.r + R(-40) * A8_1.r + R(248) * A9_1.r + R(248) * A10_1.r + R(-112) * A11_1.r + R(32) * A12_1.r + R(-256) * A13_1.r + R(-4) * A14_1.r + R(-40) * A15_1.r + R(32) * A16_1.r + R(-4) * A17_1.r + R(-4) * A18_1.r + R(32) * A19_1.r + R(284) * A20_1.r + R(248) * A21_1.r + R(320) * A22_1.r + R(-40) * A23_1.r; const R zi = R(1024) * A3_1.i + R(32) * A4_1.i + R(-256) * A5_1.i + R(-4) * A6_1.i + R(-40) * A7_1.i + R(-40) * A8_1.i + R(248) * A9_1.i + R(248) * A10_1.i + R(-112) * A11_1.i + R(32) * A12_1.i + R(-256) * A13_1.i + R(-4) * A14_1.i + R(-40) * A15_1.i + R(32) * A16_1.i + R(-4) * A17_1.i + R(-4) * A18_1.i + R(32) * A19_1.i + R(284) * A20_1.i + R(248) * A21_1.i + R(320) * A22_1.i + R(-40) * A23_1.i;
                cz1_3 = fmadd(A3_1.r, zr, fmadd(A3_1.i, zi, cz1_3)); }
              { const R zr = R(1024) * A4_1.r + R(-256) * A5_1.r + R(-4) * A6_1.r + R(32) * A7_1.r + R(284) * A8_1.r + R(248) * A9_1.r + R(320) * A10_1.r + R(-40) * A11_1.r + R(-40) * A12_1.r + R(-4) * A13_1.r + R(248) * A14_1.r + R(-112) * A15_1.r + R(-40) * A16_1.r + R(248) * A17_1.r + R(-256) * A18_1.r + R(32) * A19_1.r + R(32) * A20_1.r + R(-4) * A21_1.r + R(-4) * A22_1.r + R(-40) * A23_1.r; const R zi = R(1024) * A4_1.i + R(-256) * A5_1.i + R(-4) * A6_1.i + R(32) * A7_1.i + R(284) * A8_1.i + R(248) * A9_1.i + R(320) * A10_1.i + R(-40) * A11_1.i + R(-40) * A12_1.i + R(-4) * A13_1.i + R(248) * A14_1.i + R(-112) * A15_1.i + R(-40) * A16_1.i + R(248) * A17_1.i + R(-256) * A18_1.i + R(32) * A19_1.i + R(32) * A20_1.i + R(-4) * A21_1.i + R(-4) * A22_1.i + R(-40) * A23_1.i;
                cz1_0 = fmadd(A4_1.r, zr, fmadd(A4_1.i, zi, cz1_0)); }
              { const R zr = R(1024) * A5_1.r + R(-40) * A6_1.r + R(-4) * A7_1.r + R(248) * A8_1.r + R(-112) * A9_1.r + R(-40) * A10_1.r + R(248) * A11_1.r + R(-4) * A12_1.r + R(32) * A13_1.r + R(284) * A14_1.r + R(248) * A15_1.r + R(320) * A16_1.r + R(-40) * A17_1.r + R(32) * A18_1.r + R(-256) * A19_1.r + R(-4) * A20_1.r + R(-40) * A21_1.r + R(32) * A22_1.r + R(-4) * A23_1.r; const R zi = R(1024) * A5_1.i + R(-40) * A6_1.i + R(-4) * A7_1.i + R(248) * A8_1.i + R(-112) * A9_1.i + R(-40) * A10_1.i + R(248) * A11_1.i + R(-4) * A12_1.i + R(32) * A13_1.i + R(284) * A14_1.i + R(248) * A15_1.i + R(320) * A16_1.i + R(-40) * A17_1.i + R(32) * A18_1.i + R(-256) * A19_1.i + R(-4) * A20_1.i + R(-40) * A21_1.i + R(32) * A22_1.i + R(-4) * A23_1.i;
                cz1_1 = fmadd(A5_1.r, zr, fmadd(A5_1.i, zi, cz1_1)); }
              { const R zr = R(1024) * A6_1.r + R(-256) * A7_1.r + R(-256) * A8_1.r + R(32) * A9_1.r + R(32) * A10_1.r + R(320) * A11_1.r + R(320) * A12_1.r + R(-40) * A13_1.r + R(32) * A14_1.r + R(-4) * A15_1.r + R(248) * A16_1.r + R(284) * A17_1.r + R(-40) * A18_1.r + R(248) * A19_1.r + R(-4) * A20_1.r + R(-40) * A21_1.r + R(-112) * A22_1.r + R(248) * A23_1.r; const R zi = R(1024) * A6_1.i + R(-256) * A7_1.i + R(-256) * A8_1.i + R(32) * A9_1.i + R(32) * A10_1.i + R(320) * A11_1.i + R(320) * A12_1.i + R(-40) * A13_1.i + R(32) * A14_1.i + R(-4) * A15_1.i + R(248) * A16_1.i + R(284) * A17_1.i + R(-40) * A18_1.i + R(248) * A19_1.i + R(-4) * A20_1.i + R(-40) * A21_1.i + R(-112) * A22_1.i + R(248) * A23_1.i;
                cz1_2 = fmadd(A6_1.r, zr, fmadd(A6_1.i, zi, cz1_2)); }
              { const R zr = R(1024) * A7_1.r + R(32) * A8_1.r + R(320) * A9_1.r + R(-256) * A10_1.r + R(32) * A11_1.r + R(-40) * A12_1.r + R(248) * A13_1.r + R(-4) * A14_1.r + R(-40) * A15_1.r + R(-112) * A16_1.r + R(248) * A17_1.r + R(320) * A18_1.r + R(-40) * A19_1.r + R(32) * A20_1.r + R(-4) * A21_1.r + R(248) * A22_1.r + R(284) * A23_1.r; const R zi = R(1024) * A7_1.i + R(32) * A8_1.i + R(320) * A9_1.i + R(-256) * A10_1.i + R(32) * A11_1.i + R(-40) * A12_1.i + R(248) * A13_1.i + R(-4) * A14_1.i + R(-40) * A15_1.i + R(-112) * A16_1.i + R(248) * A17_1.i + R(320) * A18_1.i + R(-40) * A19_1.i + R(32) * A20_1.i + R(-4) * A21_1.i + R(248) * A22_1.i + R(284) * A23_1.i;
                cz1_3 = fmadd(A7_1.r, zr, fmadd(A7_1.i, zi, cz1_3)); }
              { const R zr = R(1024) * A8_1.r + R(-256) * A9_1.r + R(320) * A10_1.r + R(32) * A11_1.r + R(32) * A12_1.r + R(-4) * A13_1.r + R(-256) * A14_1.r + R(32) * A15_1.r + R(-40) * A16_1.r + R(-4) * A17_1.r + R(248) * A18_1.r + R(-112) * A19_1.r + R(-40) * A20_1.r + R(-4) * A21_1.r + R(248) * A22_1.r + R(-40) * A23_1.r; const R zi = R(1024) * A8_1.i + R(-256) * A9_1.i + R(320) * A10_1.i + R(32) * A11_1.i + R(32) * A12_1.i + R(-4) * A13_1.i + R(-256) * A14_1.i + R(32) * A15_1.i + R(-40) * A16_1.i + R(-4) * A17_1.i + R(248) * A18_1.i + R(-112) * A19_1.i + R(-40) * A20_1.i + R(-4) * A21_1.i + R(248) * A22_1.i + R(-40) * A23_1.i;
                cz1_0 = fmadd(A8_1.r, zr, fmadd(A8_1.i, zi, cz1_0)); }
              { const R zr = R(1024) * A9_1.r + R(32) * A10_1.r + R(-256) * A11_1.r + R(-4) * A12_1.r + R(-40) * A13_1.r + R(32) * A14_1.r + R(-256) * A15_1.r + R(-4) * A16_1.r + R(32) * A17_1.r + R(284) * A18_1.r + R(248) * A19_1.r + R(-4) * A20_1.r + R(32) * A21_1.r + R(-40) * A22_1.r + R(320) * A23_1.r; const R zi = R(1024) * A9_1.i + R(32) * A10_1.i + R(-256) * A11_1.i + R(-4) * A12_1.i + R(-40) * A13_1.i + R(32) * A14_1.i + R(-256) * A15_1.i + R(-4) * A16_1.i + R(32) * A17_1.i + R(284) * A18_1.i + R(248) * A19_1.i + R(-4) * A20_1.i + R(32) * A21_1.i + R(-40) * A22_1.i + R(320) * A23_1.i;
                cz1_1 = fmadd(A9_1.r, zr, fmadd(A9_1.i, zi, cz1_1)); }
              { const R zr = R(1024) * A10_1.r + R(-256) * A11_1.r + R(248) * A12_1.r + R(-112) * A13_1.r + R(-40) * A14_1.r + R(-4) * A15_1.r + R(248) * A16_1.r + R(-40) * A17_1.r + R(32) * A18_1.r + R(-4) * A19_1.r + R(-256) * A20_1.r + R(32) * A21_1.r + R(-40) * A22_1.r + R(-4) * A23_1.r; const R zi = R(1024) * A10_1.i + R(-256) * A11_1.i + R(248) * A12_1.i + R(-112) * A13_1.i + R(-40) * A14_1.i + R(-4) * A15_1.i + R(248) * A16_1.i + R(-40) * A17_1.i + R(32) * A18_1.i + R(-4) * A19_1.i + R(-256) * A20_1.i + R(32) * A21_1.i + R(-40) * A22_1.i + R(-4) * A23_1.i;
                cz1_2 = fmadd(A10_1.r, zr, fmadd(A10_1.i, zi, cz1_2)); }
              { const R zr = R(1024) * A11_1.r + R(284) * A12_1.r + R(248) * A13_1.r + R(-4) * A14_1.r + R(32) * A15_1.r + R(-40) * A16_1.r + R(320) * A17_1.r + R(-4) * A18_1.r + R(-40) * A19_1.r + R(32) * A20_1.r + R(-256) * A21_1.r + R(-4) * A22_1.r + R(32) * A23_1.r; const R zi = R(1024) * A11_1.i + R(284) * A12_1.i + R(248) * A13_1.i + R(-4) * A14_1.i + R(32) * A15_1.i + R(-40) * A16_1.i + R(320) * A17_1.i + R(-4) * A18_1.i + R(-40) * A19_1.i + R(32) * A20_1.i + R(-256) * A21_1.i + R(-4) * A22_1.i + R(32) * A23_1.i;
                cz1_3 = fmadd(A11_1.r, zr, fmadd(A11_1.i, zi, cz1_3)); }
              { const R zr = R(1024) * A12_1.r + R(-256) * A13_1.r + R(-256) * A14_1.r + R(32) * A15_1.r + R(32) * A16_1.r + R(320) * A17_1.r + R(248) * A18_1.r + R(-40) * A19_1.r + R(-112) * A20_1.r + R(248) * A21_1.r + R(-4) * A22_1.r + R(-40) * A23_1.r; const R zi = R(1024) * A12_1.i + R(-256) * A13_1.i + R(-256) * A14_1.i + R(32) * A15_1.i + R(32) * A16_1.i + R(320) * A17_1.i + R(248) * A18_1.i + R(-40) * A19_1.i + R(-112) * A20_1.i + R(248) * A21_1.i + R(-4) * A22_1.i + R(-40) * A23_1.i;
                cz1_0 = fmadd(A12_1.r, zr, fmadd(A12_1.i, zi, cz1_0)); }
              { const R zr = R(1024) * A13_1.r + R(32) * A14_1.r + R(320) * A15_1.r + R(-256) * A16_1.r + R(32) * A17_1.r + R(-40) * A18_1.r + R(320) * A19_1.r + R(248) * A20_1.r + R(284) * A21_1.r + R(32) * A22_1.r + R(-4) * A23_1.r; const R zi = R(1024) * A13_1.i + R(32) * A14_1.i + R(320) * A15_1.i + R(-256) * A16_1.i + R(32) * A17_1.i + R(-40) * A18_1.i + R(320) * A19_1.i + R(248) * A20_1.i + R(284) * A21_1.i + R(32) * A22_1.i + R(-4) * A23_1.i;
                cz1_1 = fmadd(A13_1.r, zr, fmadd(A13_1.i, zi, cz1_1)); }
              { const R zr = R(1024) * A14_1.r + R(-256) * A15_1.r + R(320) * A16_1.r + R(32) * A17_1.r + R(-112) * A18_1.r + R(248) * A19_1.r + R(248) * A20_1.r + R(-40) * A21_1.r + R(-40) * A22_1.r + R(-4) * A23_1.r; const R zi = R(1024) * A14_1.i + R(-256) * A15_1.i + R(320) * A16_1.i + R(32) * A17_1.i + R(-112) * A18_1.i + R(248) * A19_1.i + R(248) * A20_1.i + R(-40) * A21_1.i + R(-40) * A22_1.i + R(-4) * A23_1.i;
                cz1_2 = fmadd(A14_1.r, zr, fmadd(A14_1.i, zi, cz1_2)); }
              { const R zr = R(1024) * A15_1.r + R(32) * A16_1.r + R(-256) * A17_1.r + R(248) * A18_1.r + R(284) * A19_1.r + R(-40) * A20_1.r + R(320) * A21_1.r + R(-4) * A22_1.r + R(32) * A23_1.r; const R zi = R(1024) * A15_1.i + R(32) * A16_1.i + R(-256) * A17_1.i + R(248) * A18_1.i + R(284) * A19_1.i + R(-40) * A20_1.i + R(320) * A21_1.i + R(-4) * A22_1.i + R(32) * A23_1.i;
                cz1_3 = fmadd(A15_1.r, zr, fmadd(A15_1.i, zi, cz1_3)); }
              { const R zr = R(1024) * A16_1.r + R(-256) * A17_1.r + R(-4) * A18_1.r + R(32) * A19_1.r + R(-40) * A20_1.r + R(-4) * A21_1.r + R(-256) * A22_1.r + R(32) * A23_1.r; const R zi = R(1024) * A16_1.i + R(-256) * A17_1.i + R(-4) * A18_1.i + R(32) * A19_1.i + R(-40) * A20_1.i + R(-4) * A21_1.i + R(-256) * A22_1.i + R(32) * A23_1.i;
                cz1_0 = fmadd(A16_1.r, zr, fmadd(A16_1.i, zi, cz1_0)); }
              { const R zr = R(1024) * A17_1.r + R(-40) * A18_1.r + R(-4) * A19_1.r + R(-4) * A20_1.r + R(32) * A21_1.r + R(32) * A22_1.r + R(-256) * A23_1.r; const R zi = R(1024) * A17_1.i + R(-40) * A18_1.i + R(-4) * A19_1.i + R(-4) * A20_1.i + R(32) * A21_1.i + R(32) * A22_1.i + R(-256) * A23_1.i;
                cz1_1 = fmadd(A17_1.r, zr, fmadd(A17_1.i, zi, cz1_1)); }
              { const R zr = R(1024) * A18_1.r + R(-256) * A19_1.r + R(-256) * A20_1.r + R(32) * A21_1.r + R(32) * A22_1.r + R(320) * A23_1.r; const R zi = R(1024) * A18_1.i + R(-256) * A19_1.i + R(-256) * A20_1.i + R(32) * A21_1.i + R(32) * A22_1.i + R(320) * A23_1.i;
                cz1_2 = fmadd(A18_1.r, zr, fmadd(A18_1.i, zi, cz1_2)); }
              { const R zr = R(1024) * A19_1.r + R(32) * A20_1.r + R(320) * A21_1.r + R(-256) * A22_1.r + R(32) * A23_1.r; const R zi = R(1024) * A19_1.i + R(32) * A20_1.i + R(320) * A21_1.i + R(-256) * A22_1.i + R(32) * A23_1.i;
                cz1_3 = fmadd(A19_1.r, zr, fmadd(A19_1.i, zi, cz1_3)); }
              { const R zr = R(1024) * A20_1.r + R(-256) * A21_1.r + R(320) * A22_1.r + R(32) * A23_1.r; const R zi = R(1024) * A20_1.i + R(-256) * A21_1.i + R(320) * A22_1.i + R(32) * A23_1.i;
                cz1_0 = fmadd(A20_1.r, zr, fmadd(A20_1.i, zi, cz1_0)); }
              { const R zr = R(1024) * A21_1.r + R(32) * A22_1.r + R(-256) * A23_1.r; const R zi = R(1024) * A21_1.i + R(32) * A22_1.i + R(-256) * A23_1.i;
                cz1_1 = fmadd(A21_1.r, zr, fmadd(A21_1.i, zi, cz1_1)); }
              { const R zr = R(1024) * A22_1.r + R(-256) * A23_1.r; const R zi = R(1024) * A22_1.i + R(-256) * A23_1.i;
                cz1_2 = fmadd(A22_1.r, zr, fmadd(A22_1.i, zi, cz1_2)); }
              { const R zr = R(1024) * A23_1.r; const R zi = R(1024) * A23_1.i;
                cz1_3 = fmadd(A23_1.r, zr, fmadd(A23_1.i, zi, cz1_3)); }
            }
          }
        }
      }
    }
  }
  if constexpr (CM == CM_FMA) acc = cz0_0 + cz0_1 + cz0_2 + cz0_3 + cz1_0 + cz1_1 + cz1_2 + cz1_3;
  return acc;
}

// floating-point operations of one full helicity sum (all levels, all loop trips)
constexpr long FLOPS_HEL_SUM = 404307;
}}  // namespace
