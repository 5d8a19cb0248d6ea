// Multi-process kernel variants (multi.cuh): g g -> t tbar with its real
// emission g g -> t tbar g (FP64, FP32), and g g -> t tbar with g g -> t tbar g
// and g g -> t tbar g g (FP64).  Costliest process first in each list, so its
// tiles are handed out first.
#include "../../include/rwgt.h"
#include "gen_qcd_gg_tt.cuh"
#include "gen_qcd_gg_ttg.cuh"
#include "gen_qcd_gg_ttgg.cuh"
#include "multi.cuh"
#include "procs.cuh"
#include "registry.h"

namespace rw {
namespace {
#define RW_QCD_TAG(tag, ns, jsmem)                                                                       \
  struct tag {                                                                                           \
    static constexpr int NG = ns::NG;                                                                    \
    static constexpr int NEXT = ns::NEXT;                                                                \
    static constexpr int MAX_LB = ns::MAX_LB;                                                            \
    static constexpr int NJS = ns::NJS;                                                                  \
    static constexpr int NCOL = ns::K;                                                                   \
    static constexpr bool JSMEM = jsmem;                                                                 \
    template <class R, int LB, int CM>                                                                   \
    __device__ __forceinline__ static R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& K, int lane) { \
      return ns::hel_sum<R, LB, CM, JSMEM && sizeof(R) == 4>(X, K, lane);                                \
    }                                                                                                    \
  };
RW_QCD_TAG(TagTT, gg_tt, false)
RW_QCD_TAG(TagTTG, gg_ttg, false)
RW_QCD_TAG(TagTTGG, gg_ttgg, true)
#undef RW_QCD_TAG
using PTT = QcdProc<TagTT>;
using PTTG = QcdProc<TagTTG>;
using PTTGG = QcdProc<TagTTGG>;
}  // namespace

void register_multi(std::vector<MultiEntry>& t) {
  t.push_back({RW_FP64, 2, {RW_GG_TTG, RW_GG_TT}, {0, 0},
               (const void*)&k_reweight_multi<double, Lanes<PTTG, 0>, Lanes<PTT, 0>>, 0});
  t.push_back({RW_FP32, 2, {RW_GG_TTG, RW_GG_TT}, {0, 0},
               (const void*)&k_reweight_multi<float, Lanes<PTTG, 0>, Lanes<PTT, 0>>, 0});
  t.push_back({RW_FP64, 3, {RW_GG_TTGG, RW_GG_TTG, RW_GG_TT}, {1, 0, 0},
               (const void*)&k_reweight_multi<double, Lanes<PTTGG, 1>, Lanes<PTTG, 0>, Lanes<PTT, 0>>, 0});
}

}  // namespace rw
