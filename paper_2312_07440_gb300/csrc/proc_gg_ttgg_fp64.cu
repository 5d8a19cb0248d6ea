// g g -> t tbar + n g kernel variants (gg_ttgg, fp64).
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
  static constexpr bool JSMEM = false;  // currents of 3+ gluons in shared memory (FP32)
  template <class R, int LB, int CM>
  __device__ __forceinline__ static R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& K, int lane) {
    return gg_ttgg::hel_sum<R, LB, CM, JSMEM && sizeof(R) == 4>(X, K, lane);
  }
};
using P = QcdProc<Tag>;
}  // namespace

void register_gg_ttgg_fp64(std::vector<KernelEntry>& t) {
  t.push_back({RW_GG_TTGG, RW_FP64, 1, (const void*)&k_reweight<P, double, 1>});
  t.push_back({RW_GG_TTGG, RW_FP64, 1, (const void*)&k_interp<P, double, 1>, 256, 1});
  t.push_back({RW_GG_TTGG, RW_FP64, 2, (const void*)&k_reweight<P, double, 2>});
  t.push_back({RW_GG_TTGG, RW_FP64, 2, (const void*)&k_interp<P, double, 2>, 256, 1});
  t.push_back({RW_GG_TTGG, RW_FP64, 3, (const void*)&k_reweight<P, double, 3>});
  t.push_back({RW_GG_TTGG, RW_FP64, 3, (const void*)&k_interp<P, double, 3>, 256, 1});
}

void static_gg_ttgg(ProcStatic& s) {
  s = {gg_ttgg::NEXT, gg_ttgg::NHEL, gg_ttgg::K, gg_ttgg::NDIAG, gg_ttgg::CDEN, gg_ttgg::IDENT, gg_ttgg::NG,
       gg_ttgg::FLOPS_HEL_SUM, gg_ttgg::MAX_LB};
}

}  // namespace rw
