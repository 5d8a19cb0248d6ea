// g g -> t tbar + n g kernel variants (gg_ttgg, fp32).
// the FP32 slash and gluon vertices out of line: the 24 orderings' unrolled
// chains otherwise overflow the instruction cache and spill (helas.cuh)
#define RW_FP32_OUTLINED_SLASH 1
#define RW_FP32_OUTLINED_CURRENTS 1
#include "../../include/rwgt.h"
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
  template <class R, int LB, int CM>
  __device__ __forceinline__ static R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& K, int lane) {
    return gg_ttgg::hel_sum<R, LB, CM, JSMEM && sizeof(R) == 4>(X, K, lane);
  }
};
using P = QcdProc<Tag>;
}  // namespace

void register_gg_ttgg_fp32(std::vector<KernelEntry>& t) {
  t.push_back({RW_GG_TTGG, RW_FP32, 1, (const void*)&k_reweight<P, float, 1>, 256, 0, P::jstore_bytes<float, 1>()});
  t.push_back({RW_GG_TTGG, RW_FP32, 1, (const void*)&k_interp<P, float, 1>, 256, 1, P::jstore_bytes<float, 1>()});
  t.push_back({RW_GG_TTGG, RW_FP32, 2, (const void*)&k_reweight<P, float, 2>, 256, 0, P::jstore_bytes<float, 2>()});
  t.push_back({RW_GG_TTGG, RW_FP32, 2, (const void*)&k_interp<P, float, 2>, 256, 1, P::jstore_bytes<float, 2>()});
  t.push_back({RW_GG_TTGG, RW_FP32, 3, (const void*)&k_reweight<P, float, 3>, 256, 0, P::jstore_bytes<float, 3>()});
  t.push_back({RW_GG_TTGG, RW_FP32, 4, (const void*)&k_reweight<P, float, 4>, 256, 0, P::jstore_bytes<float, 4>()});
  t.push_back({RW_GG_TTGG, RW_FP32, 3, (const void*)&k_interp<P, float, 3>, 256, 1, P::jstore_bytes<float, 3>()});
  t.push_back({RW_GG_TTGG, RW_FP32, 4, (const void*)&k_interp<P, float, 4>, 256, 1, P::jstore_bytes<float, 4>()});
}

}  // namespace rw
