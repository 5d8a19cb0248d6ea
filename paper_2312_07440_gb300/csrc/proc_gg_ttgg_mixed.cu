// g g -> t tbar + n g kernel variants (gg_ttgg, mixed precision: FP32 amplitudes,
// FP16/BF16 tensor-core colour sum with FP32 accumulation).
// the FP32 slash out of line: the 24 orderings' unrolled chains otherwise
// overflow the instruction cache and spill (helas.cuh; the gluon vertices too
// made this kernel 11 % slower, unlike the FP32 one)
#define RW_FP32_OUTLINED_SLASH 1
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
  template <class R, int LB, int CM>
  __device__ __forceinline__ static R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& K, int lane) {
    return gg_ttgg::hel_sum<R, LB, CM, JSMEM && sizeof(R) == 4>(X, K, lane);
  }
};
using P16 = QcdProc<Tag, CM_FP16>;
using PB16 = QcdProc<Tag, CM_BF16>;
}  // namespace

// The current store (768 B) and the colour staging (168 B) per thread fit a
// 128-thread block's shared memory but not a 256-thread one's (227 KB).  (The
// per-event constants stay in registers here: in shared memory they cost the
// mixed kernel more than they save, at the same occupancy.)
constexpr int kMaxBlock = 227 * 1024 / P16::jstore_bytes<float, 2>() >= 256 ? 256 : 128;
static_assert(P16::jstore_bytes<float, 2>() == PB16::jstore_bytes<float, 2>(), "one block limit for both types");

void register_gg_ttgg_mixed(std::vector<KernelEntry>& t) {
  t.push_back({RW_GG_TTGG, RW_MIXED_FP16, 1, (const void*)&k_reweight<P16, float, 1>, kMaxBlock, 0, P16::jstore_bytes<float, 1>()});
  t.push_back({RW_GG_TTGG, RW_MIXED_BF16, 1, (const void*)&k_reweight<PB16, float, 1>, kMaxBlock, 0, PB16::jstore_bytes<float, 1>()});
  t.push_back({RW_GG_TTGG, RW_MIXED_FP16, 2, (const void*)&k_reweight<P16, float, 2>, kMaxBlock, 0, P16::jstore_bytes<float, 2>()});
  t.push_back({RW_GG_TTGG, RW_MIXED_BF16, 2, (const void*)&k_reweight<PB16, float, 2>, kMaxBlock, 0, PB16::jstore_bytes<float, 2>()});
  t.push_back({RW_GG_TTGG, RW_MIXED_FP16, 3, (const void*)&k_reweight<P16, float, 3>, kMaxBlock, 0, P16::jstore_bytes<float, 3>()});
  t.push_back({RW_GG_TTGG, RW_MIXED_FP16, 4, (const void*)&k_reweight<P16, float, 4>, kMaxBlock, 0, P16::jstore_bytes<float, 4>()});
  t.push_back({RW_GG_TTGG, RW_MIXED_BF16, 3, (const void*)&k_reweight<PB16, float, 3>, kMaxBlock, 0, PB16::jstore_bytes<float, 3>()});
  t.push_back({RW_GG_TTGG, RW_MIXED_BF16, 4, (const void*)&k_reweight<PB16, float, 4>, kMaxBlock, 0, PB16::jstore_bytes<float, 4>()});
}

}  // namespace rw
