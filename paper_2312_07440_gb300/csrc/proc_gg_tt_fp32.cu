// g g -> t tbar + n g kernel variants (gg_tt, fp32).
#include "../../include/rwgt.h"
#include "gen_qcd_gg_tt.cuh"
#include "kernels.cuh"
#include "procs.cuh"
#include "registry.h"

namespace rw {
namespace {
struct Tag {
  static constexpr int NG = gg_tt::NG;
  static constexpr int NEXT = gg_tt::NEXT;
  static constexpr int MAX_LB = gg_tt::MAX_LB;
  static constexpr int NJS = gg_tt::NJS;
  static constexpr int NCOL = gg_tt::K;
  static constexpr bool JSMEM = false;  // currents of 3+ gluons in shared memory (FP32)
  static constexpr bool INLINE_ME = true;  // amplitude code inlined into the kernel (FP32)
  template <class R, int LB, int CM>
  __device__ __forceinline__ static R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& K, int lane) {
    return gg_tt::hel_sum<R, LB, CM, JSMEM && sizeof(R) == 4>(X, K, lane);
  }
};
using P = QcdProc<Tag>;
}  // namespace

void register_gg_tt_fp32(std::vector<KernelEntry>& t) {
  t.push_back({RW_GG_TT, RW_FP32, 0, (const void*)&k_reweight<P, float, 0, 2>});
  t.push_back({RW_GG_TT, RW_FP32, 0, (const void*)&k_interp<P, float, 0, 2>, 256, 1});
  t.push_back({RW_GG_TT, RW_FP32, 1, (const void*)&k_reweight<P, float, 1, 2>});
  t.push_back({RW_GG_TT, RW_FP32, 1, (const void*)&k_interp<P, float, 1, 2>, 256, 1});
  t.push_back({RW_GG_TT, RW_FP32, 2, (const void*)&k_reweight<P, float, 2, 2>});
  t.push_back({RW_GG_TT, RW_FP32, 2, (const void*)&k_interp<P, float, 2, 2>, 256, 1});

}

}  // namespace rw
