// g g -> t tbar + n g kernel variants (gg_ttg, mixed precision: FP32 amplitudes,
// FP16/BF16 tensor-core colour sum with FP32 accumulation).
#include "../../include/rwgt.h"
#include "gen_qcd_gg_ttg.cuh"
#include "kernels.cuh"
#include "procs.cuh"
#include "registry.h"

namespace rw {
namespace {
struct Tag {
  static constexpr int NG = gg_ttg::NG;
  static constexpr int NEXT = gg_ttg::NEXT;
  static constexpr int MAX_LB = gg_ttg::MAX_LB;
  static constexpr int NJS = gg_ttg::NJS;
  static constexpr int NCOL = gg_ttg::K;
  static constexpr bool JSMEM = false;  // currents of 3+ gluons in shared memory (FP32)
  template <class R, int LB, int CM>
  __device__ __forceinline__ static R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& K, int lane) {
    return gg_ttg::hel_sum<R, LB, CM, JSMEM && sizeof(R) == 4>(X, K, lane);
  }
};
using P16 = QcdProc<Tag, CM_FP16>;
using PB16 = QcdProc<Tag, CM_BF16>;
}  // namespace

void register_gg_ttg_mixed(std::vector<KernelEntry>& t) {
  t.push_back({RW_GG_TTG, RW_MIXED_FP16, 0, (const void*)&k_reweight<P16, float, 0>, 256, 0, P16::jstore_bytes<float>()});
  t.push_back({RW_GG_TTG, RW_MIXED_BF16, 0, (const void*)&k_reweight<PB16, float, 0>, 256, 0, PB16::jstore_bytes<float>()});
  t.push_back({RW_GG_TTG, RW_MIXED_FP16, 1, (const void*)&k_reweight<P16, float, 1>, 256, 0, P16::jstore_bytes<float>()});
  t.push_back({RW_GG_TTG, RW_MIXED_BF16, 1, (const void*)&k_reweight<PB16, float, 1>, 256, 0, PB16::jstore_bytes<float>()});
  t.push_back({RW_GG_TTG, RW_MIXED_FP16, 2, (const void*)&k_reweight<P16, float, 2>, 256, 0, P16::jstore_bytes<float>()});
  t.push_back({RW_GG_TTG, RW_MIXED_BF16, 2, (const void*)&k_reweight<PB16, float, 2>, 256, 0, PB16::jstore_bytes<float>()});
}

}  // namespace rw
