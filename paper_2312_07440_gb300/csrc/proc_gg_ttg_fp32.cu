// g g -> t tbar + n g kernel variants (gg_ttg, fp32).
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
using P = QcdProc<Tag>;
}  // namespace

void register_gg_ttg_fp32(std::vector<KernelEntry>& t) {
  t.push_back({RW_GG_TTG, RW_FP32, 0, (const void*)&k_reweight<P, float, 0>});
  t.push_back({RW_GG_TTG, RW_FP32, 0, (const void*)&k_interp<P, float, 0>, 256, 1});
  t.push_back({RW_GG_TTG, RW_FP32, 1, (const void*)&k_reweight<P, float, 1>});
  t.push_back({RW_GG_TTG, RW_FP32, 1, (const void*)&k_interp<P, float, 1>, 256, 1});
  t.push_back({RW_GG_TTG, RW_FP32, 2, (const void*)&k_reweight<P, float, 2>});
  t.push_back({RW_GG_TTG, RW_FP32, 2, (const void*)&k_interp<P, float, 2>, 256, 1});
  t.push_back({RW_GG_TTG, RW_FP32, 3, (const void*)&k_reweight<P, float, 3>});
  t.push_back({RW_GG_TTG, RW_FP32, 3, (const void*)&k_interp<P, float, 3>, 256, 1});
}

}  // namespace rw
