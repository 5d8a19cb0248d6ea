// e- e+ -> 5 photons kernel variants (fp64).
#include "../../include/rwgt.h"
#include "gen_qed_ee_5a.cuh"
#include "kernels.cuh"
#include "procs.cuh"
#include "registry.h"

namespace rw {
namespace {
struct Tag {
  static constexpr int NA = ee_5a::NA;
  static constexpr int NEXT = ee_5a::NEXT;
  static constexpr int MAX_LB = ee_5a::MAX_LB;
  template <class R, int LB>
  __device__ __forceinline__ static R hel_sum(const QedExt<R, NA>& X, const QedKin<R, NA>& K, int lane) {
    return ee_5a::hel_sum<R, LB>(X, K, lane);
  }
};
using P = QedProc<Tag>;
}  // namespace

void register_ee_5a_fp64(std::vector<KernelEntry>& t) {
  t.push_back({RW_EE_5A, RW_FP64, 0, (const void*)&k_reweight<P, double, 0>});
  t.push_back({RW_EE_5A, RW_FP64, 0, (const void*)&k_interp<P, double, 0>, 256, 1});
  t.push_back({RW_EE_5A, RW_FP64, 1, (const void*)&k_reweight<P, double, 1>});
  t.push_back({RW_EE_5A, RW_FP64, 1, (const void*)&k_interp<P, double, 1>, 256, 1});
  t.push_back({RW_EE_5A, RW_FP64, 2, (const void*)&k_reweight<P, double, 2>});
  t.push_back({RW_EE_5A, RW_FP64, 2, (const void*)&k_interp<P, double, 2>, 256, 1});
  t.push_back({RW_EE_5A, RW_FP64, 3, (const void*)&k_reweight<P, double, 3>});
  t.push_back({RW_EE_5A, RW_FP64, 3, (const void*)&k_interp<P, double, 3>, 256, 1});
}

void static_ee_5a(ProcStatic& s) {
  s = {ee_5a::NEXT, ee_5a::NHEL, 1, ee_5a::NDIAG, 1, ee_5a::IDENT, 0, ee_5a::FLOPS_HEL_SUM, ee_5a::MAX_LB};
}

}  // namespace rw
