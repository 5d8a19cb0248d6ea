// Process adapters for the fused kernel: |M|^2 of one event for one
// parameter point, helicity slices combined across the 2^LB lanes of a group.
#pragma once
#include <type_traits>

#include "colour_mma.cuh"
#include "helas.cuh"
#include "kernels.cuh"
#include "qcd.cuh"
#include "qed.cuh"

namespace rw {

// Tag::KSMEM (optional, default false): keep the per-event constants in
// shared memory in the FP32 modes
template <class T, class = void>
struct tag_ksmem : std::false_type {};
template <class T>
struct tag_ksmem<T, std::void_t<decltype(T::KSMEM)>> : std::integral_constant<bool, T::KSMEM> {};

// Tag::INLINE_ME (optional, default false): the FP32 amplitude code inlined
// into the kernel's single call site (small processes: no call-site saves)
template <class T, class = void>
struct tag_inline_me : std::false_type {};
template <class T>
struct tag_inline_me<T, std::void_t<decltype(T::INLINE_ME)>> : std::integral_constant<bool, T::INLINE_ME> {};

// g g -> t tbar + n g.  Tag provides NG, NEXT, MAX_LB and hel_sum<R, LB, CM>();
// CM selects the colour sum (FMA, or tensor cores in FP16/BF16).
template <class Tag, int CM = 0>
struct QcdProc {
  static constexpr int NG = Tag::NG;
  static constexpr int NEXT = Tag::NEXT;
  static constexpr int NCOL = Tag::NCOL;
  static constexpr bool kSymmetricHelicities = true;
  // per-event constants (external wavefunctions and propagator invariants):
  // one slot per event group in shared memory, written by the group's lanes
  // and read by them at every use, instead of a copy in every lane's
  // registers (FP32, at least 4 lanes per event)
  template <class R, int LB>
  static constexpr bool ksmem() {
    return tag_ksmem<Tag>::value && sizeof(R) == 4 && LB >= 2;
  }
  static constexpr int kSlot = (int)((sizeof(QcdExt<float, NG>) + sizeof(QcdKin<float, NG>) + 15) / 16 * 16);

  // Momenta: FP64 in FP64 mode, double-float in the FP32 modes (dfloat.cuh).
  template <class R>
  using mom_t = typename std::conditional<sizeof(R) == 8, double, df>::type;
  // dynamic shared memory per thread of the amplitude code: the current store,
  // then (tensor-core colour sum) the warp's colour staging, as a per-thread share
  template <class R>
  static constexpr int store_bytes() {
    return ((Tag::JSMEM && sizeof(R) == 4) ? Tag::NJS * 32 : 0) +
           ((CM == CM_FP16 || CM == CM_BF16) ? ColourStage<(Tag::NCOL + 15) / 16 * 16>::per_thread : 0);
  }
  template <class R, int LB = 0>
  static constexpr int jstore_bytes() {
    static_assert(kSlot % 16 == 0 && kSlot % (1 << Tag::MAX_LB) == 0, "the slots split evenly over the lanes");
    return store_bytes<R>() + (ksmem<R, LB>() ? kSlot >> LB : 0);
  }

  template <class R, int LB>
  __device__ __forceinline__ static double me_body(const mom_t<R> (&p)[NEXT][4], const PointDev& pt, int lane,
                                           unsigned gmask) {
    static_assert(LB <= Tag::MAX_LB, "more lane bits than helicity levels");
    double s;
    if constexpr (ksmem<R, LB>()) {
      extern __shared__ __align__(16) unsigned char rw_dyn_bytes[];
      unsigned char* slot =
          rw_dyn_bytes + (size_t)store_bytes<R>() * blockDim.x + (size_t)(threadIdx.x >> LB) * kSlot;
      QcdExt<R, NG>& X = *reinterpret_cast<QcdExt<R, NG>*>(slot);
      QcdKin<R, NG>& Kn = *reinterpret_cast<QcdKin<R, NG>*>(slot + sizeof(QcdExt<R, NG>));
      __syncwarp(gmask);  // the group's reads of the previous evaluation are done
      // every lane of the group writes the same values (same inputs, same code)
      qcd_setup<R, NG, NEXT>(p, pt.m_t, X, Kn);
      __syncwarp(gmask);
      s = double(Tag::template hel_sum<R, LB, CM>(X, Kn, lane));
    } else {
      QcdExt<R, NG> X;
      QcdKin<R, NG> Kn;
      qcd_setup<R, NG, NEXT>(p, pt.m_t, X, Kn);
      s = double(Tag::template hel_sum<R, LB, CM>(X, Kn, lane));
    }
#pragma unroll
    for (int o = 1; o < (1 << LB); o <<= 1) s += __shfl_xor_sync(gmask, s, o);
    return s * pt.cscale;
  }  // Out of line by default: every evaluation runs the same instructions, so
  // identical inputs give bitwise identical |M|^2 (r == 1 exactly for
  // unchanged parameters).  Inlined (Tag::INLINE_ME, FP32) the kernel's one
  // call site, inside its loop over the points, keeps that property.
  template <class R>
  static constexpr bool inline_me() {
    return tag_inline_me<Tag>::value && sizeof(R) == 4;
  }
  template <class R, int LB>
  __device__ __noinline__ static double me(const mom_t<R> (&p)[NEXT][4], const PointDev& pt, int lane,
                                           unsigned gmask) {
    return me_body<R, LB>(p, pt, lane, gmask);
  }

  // The amplitudes of one event and point for a separate colour pass
  // (CM_STORE_*): the set-up as in me_body, then every J vector to sink.put();
  // false when the point's masses do not fit the event (its |M'|^2 is 0).
  template <class R, int LB, class Sink>
  __device__ __noinline__ static bool me_store(const mom_t<R> (&p)[NEXT][4], const PointDev& pt, int lane,
                                               unsigned gmask, Sink& sink) {
    static_assert(LB <= Tag::MAX_LB, "more lane bits than helicity levels");
    mom_t<R> q[NEXT][4];
    bool inside = true;
    if (pt.reshuffle) {
      inside = reshuffle<R>(p, pt.m_t, q);
    } else {
#pragma unroll
      for (int i = 0; i < NEXT; ++i)
#pragma unroll
        for (int m = 0; m < 4; ++m) q[i][m] = p[i][m];
    }
    if constexpr (ksmem<R, LB>()) {
      extern __shared__ __align__(16) unsigned char rw_dyn_bytes[];
      unsigned char* slot =
          rw_dyn_bytes + (size_t)store_bytes<R>() * blockDim.x + (size_t)(threadIdx.x >> LB) * kSlot;
      QcdExt<R, NG>& X = *reinterpret_cast<QcdExt<R, NG>*>(slot);
      QcdKin<R, NG>& Kn = *reinterpret_cast<QcdKin<R, NG>*>(slot + sizeof(QcdExt<R, NG>));
      __syncwarp(gmask);
      qcd_setup<R, NG, NEXT>(q, pt.m_t, X, Kn);
      __syncwarp(gmask);
      Tag::template hel_sum<R, LB, CM>(X, Kn, lane, &sink);
    } else {
      QcdExt<R, NG> X;
      QcdKin<R, NG> Kn;
      qcd_setup<R, NG, NEXT>(q, pt.m_t, X, Kn);
      Tag::template hel_sum<R, LB, CM>(X, Kn, lane, &sink);
    }
    return inside;
  }

  // FP64 mode refines the FP32 Newton solution with two FP64 steps, the FP32
  // modes with one double-float step.
  template <class R>
  __device__ __forceinline__ static bool reshuffle(const mom_t<R> (&p)[NEXT][4], double mt, mom_t<R> (&q)[NEXT][4]) {
    if constexpr (sizeof(R) == 8)
      return reshuffle_tops<NEXT, 2>(p, mt, q);
    else
      return reshuffle_tops<NEXT>(p, mt, q);
  }
};

// e-(p0) e+(p1) -> n photons (massless QED).  Tag provides NA, NEXT, MAX_LB
// and hel_sum<R, LB>() (generated by gen/qed_gen.py); |M|^2 = cscale * sum,
// cscale = e^(2n) / (4 n!).  Nothing moves with the parameters (no reshuffle).
template <class Tag>
struct QedProc {
  static constexpr int NA = Tag::NA;
  static constexpr int NEXT = Tag::NEXT;
  template <class R>
  using mom_t = typename std::conditional<sizeof(R) == 8, double, df>::type;
  template <class R, int LB = 0>
  static constexpr int jstore_bytes() {
    return 0;
  }
  template <class R>
  static constexpr bool inline_me() {
    return false;
  }

  template <class R, int LB>
  __device__ __noinline__ static double me(const mom_t<R> (&p)[NEXT][4], const PointDev& pt, int lane,
                                           unsigned gmask) {
    static_assert(LB <= Tag::MAX_LB, "more lane bits than helicity levels");
    QedExt<R, NA> X;
    QedKin<R, NA> Kn;
    qed_setup<R, NA, NEXT>(p, X, Kn);
    double s = double(Tag::template hel_sum<R, LB>(X, Kn, lane));
#pragma unroll
    for (int o = 1; o < (1 << LB); o <<= 1) s += __shfl_xor_sync(gmask, s, o);
    return s * pt.cscale;
  }
  template <class R>
  __device__ __forceinline__ static bool reshuffle(const mom_t<R> (&p)[NEXT][4], double, mom_t<R> (&q)[NEXT][4]) {
#pragma unroll
    for (int i = 0; i < NEXT; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) q[i][m] = p[i][m];
    return true;
  }
};

// e-(p0) e+(p1) -> mu-(p2) mu+(p3) through s-channel photon and Z (unitary
// gauge, fixed width), massless leptons:
//   M = e^2 (jo.ji)/s + [zo.zi - (k.zo)(k.zi)/MZ^2] / (s - MZ^2 + i MZ WZ)
// with ji = vbar(p1) gamma^mu u(p0), zi = vbar(p1) gamma^mu (gL PL + gR PR) u(p0)
// and jo, zo the same for ubar(p2) ... v(p3); |M|^2 averaged over the 4
// initial helicity states.
struct EeMumu {
  static constexpr int NEXT = 4;
  static constexpr int NHEL = 16;
  // FP64 momenta in every mode (a 4-particle process with no reshuffle: its
  // few FP64 invariants per event are not a bottleneck)
  template <class R>
  using mom_t = double;
  template <class R, int LB = 0>
  static constexpr int jstore_bytes() {
    return 0;
  }
  template <class R>
  static constexpr bool inline_me() {
    return false;
  }

  template <class R, int LB>
  __device__ __noinline__ static double me(const double (&p)[NEXT][4], const PointDev& pt, int lane,
                                           unsigned gmask) {
    sp<R> u0[2], vb1[2], ub2[2], v3[2];
    R pr[NEXT][4];
#pragma unroll
    for (int i = 0; i < NEXT; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) pr[i][m] = R(p[i][m]);
    u_in<R>(pr[0], R(0), u0);
    vbar_in<R>(pr[1], R(0), vb1);
    ubar_out<R>(pr[2], R(0), ub2);
    v_out<R>(pr[3], R(0), v3);
    R k[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) k[m] = R(p[0][m] + p[1][m]);
    const double sd = 2.0 * dot4(p[0], p[1]);
    const R e2s = R(pt.e * pt.e / sd);
    // 1/(s - MZ^2 + i MZ WZ)
    const double dr = sd - pt.MZ * pt.MZ, di = pt.MZ * pt.WZ, dn = dr * dr + di * di;
    const cx<R> dz = {R(dr / dn), R(-di / dn)};
    const R imz2 = R(1.0 / (pt.MZ * pt.MZ));
    const R gL = R(pt.gL), gR = R(pt.gR);
    R acc = R(0);
    constexpr int NLOC = NHEL >> LB;
#pragma unroll 1
    for (int hh = 0; hh < NLOC; ++hh) {
      const int h = (lane << (4 - LB)) | hh;  // bits: 3 -> p0, 2 -> p1, 1 -> p2, 0 -> p3
      const sp<R>& u = u0[(h >> 3) & 1];
      const sp<R>& vb = vb1[(h >> 2) & 1];
      const sp<R>& ub = ub2[(h >> 1) & 1];
      const sp<R>& v = v3[h & 1];
      const sp<R> uL = {{u.c[0], u.c[1], {R(0), R(0)}, {R(0), R(0)}}};
      const sp<R> uR = {{{R(0), R(0)}, {R(0), R(0)}, u.c[2], u.c[3]}};
      const sp<R> vL = {{v.c[0], v.c[1], {R(0), R(0)}, {R(0), R(0)}}};
      const sp<R> vR = {{{R(0), R(0)}, {R(0), R(0)}, v.c[2], v.c[3]}};
      const cv<R> jiL = fcur(vb, uL), jiR = fcur(vb, uR);
      const cv<R> joL = fcur(ub, vL), joR = fcur(ub, vR);
      cv<R> ji, jo, zi, zo;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        ji.c[m] = jiL.c[m] + jiR.c[m];
        jo.c[m] = joL.c[m] + joR.c[m];
        zi.c[m] = gL * jiL.c[m] + gR * jiR.c[m];
        zo.c[m] = gL * joL.c[m] + gR * joR.c[m];
      }
      const cx<R> zz = dot(zo, zi) - imz2 * (dotr(k, zo) * dotr(k, zi));
      const cx<R> M = e2s * dot(jo, ji) + zz * dz;
      acc += M.r * M.r + M.i * M.i;
    }
    double s = double(acc);
#pragma unroll
    for (int o = 1; o < (1 << LB); o <<= 1) s += __shfl_xor_sync(gmask, s, o);
    return 0.25 * s;
  }
  template <class R>
  __device__ __forceinline__ static bool reshuffle(const double (&p)[NEXT][4], double, double (&q)[NEXT][4]) {
#pragma unroll
    for (int i = 0; i < NEXT; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) q[i][m] = p[i][m];
    return true;
  }
};

}  // namespace rw
