// g g -> t tbar g g, mixed-precision modes with the colour sum as a separate
// tensor-core pass (colour_tc.cuh): the amplitude pass in the FP32 mode's
// configuration (slash and gluon vertices out of line, per-event constants in
// shared memory), J vectors stored in FP16 or BF16.  Included by one
// translation unit per 16-bit type with RW_STORE_CM set.
#define RW_FP32_OUTLINED_SLASH 1
#define RW_FP32_OUTLINED_CURRENTS 1
#include "../../include/rwgt.h"
#include "colour_tc.cuh"
#include "gen_qcd_gg_ttgg.cuh"
#include "kernels.cuh"
#include "procs.cuh"
#include "registry.h"

namespace rw {
namespace {
struct Tag {
  static constexpr int NG = gg_ttgg::NG;
  static constexpr int NEXT = gg_ttgg::NEXT;
  static constexpr int MAX_LB = gg_ttgg::MAX_LB;
  static constexpr int NJS = gg_ttgg::NJS;
  static constexpr int NCOL = gg_ttgg::K;
  static constexpr bool JSMEM = true;  // currents of 3+ gluons in shared memory (FP32)
  static constexpr bool KSMEM = true;  // per-event constants in shared memory (FP32)
  template <class R, int LB, int CM, class S = NoSink>
  __device__ __forceinline__ static R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& K, int lane,
                                              S* sink = nullptr) {
    return gg_ttgg::hel_sum<R, LB, CM, JSMEM && sizeof(R) == 4, S>(X, K, lane, sink);
  }
};
struct CTab {
  __device__ __forceinline__ static short at(int i) { return gg_ttgg::CI[i]; }
};
using PS = QcdProc<Tag, RW_STORE_CM>;
constexpr int SLOTS = 1 << (gg_ttgg::NEXT - 1);
}  // namespace

void RW_STORE_REGISTER(std::vector<KernelEntry>& t) {
  constexpr int mode = RW_STORE_CM == CM_STORE_BF16 ? RW_MIXED_BF16 : RW_MIXED_FP16;
  const void* colour = (const void*)&k_colour_tc<gg_ttgg::K, RW_STORE_CM, SLOTS, CTab>;
  t.push_back({RW_GG_TTGG, mode, 2, (const void*)&k_amp_store<PS, 2, RW_STORE_CM>, 256, 2,
               PS::jstore_bytes<float, 2>(), colour});
  t.push_back({RW_GG_TTGG, mode, 3, (const void*)&k_amp_store<PS, 3, RW_STORE_CM>, 256, 2,
               PS::jstore_bytes<float, 3>(), colour});
}

}  // namespace rw
