// e+ e- -> mu+ mu- kernel variants.
#include "../../include/rwgt.h"
#include "kernels.cuh"
#include "procs.cuh"
#include "registry.h"

namespace rw {

// Floating-point operations of EeMumu::me's helicity sum as written, per
// helicity: 4 fermion currents (4 x 72), the vector and axial sums (16 + 48),
// the Z exchange (dot 30, two real-complex products 28, 6 + 2 + 2), the photon
// exchange (dot 30, 2), their sum (6 + 2), |M|^2 and its accumulation (4).
constexpr long long EE_MUMU_FLOPS_HEL_SUM = EeMumu::NHEL * 464LL;

void register_ee_mumu(std::vector<KernelEntry>& t, ProcStatic& s) {
  s = {4, 16, 1, 2, 1, 1, 0, EE_MUMU_FLOPS_HEL_SUM, 4};
  t.push_back({RW_EE_MUMU, RW_FP64, 0, (const void*)&k_reweight<EeMumu, double, 0>});
  t.push_back({RW_EE_MUMU, RW_FP64, 0, (const void*)&k_interp<EeMumu, double, 0>, 256, 1});
  t.push_back({RW_EE_MUMU, RW_FP64, 2, (const void*)&k_reweight<EeMumu, double, 2>});
  t.push_back({RW_EE_MUMU, RW_FP64, 2, (const void*)&k_interp<EeMumu, double, 2>, 256, 1});
  t.push_back({RW_EE_MUMU, RW_FP64, 4, (const void*)&k_reweight<EeMumu, double, 4>});
  t.push_back({RW_EE_MUMU, RW_FP64, 4, (const void*)&k_interp<EeMumu, double, 4>, 256, 1});
  t.push_back({RW_EE_MUMU, RW_FP32, 0, (const void*)&k_reweight<EeMumu, float, 0>});
  t.push_back({RW_EE_MUMU, RW_FP32, 0, (const void*)&k_interp<EeMumu, float, 0>, 256, 1});
  t.push_back({RW_EE_MUMU, RW_FP32, 2, (const void*)&k_reweight<EeMumu, float, 2>});
  t.push_back({RW_EE_MUMU, RW_FP32, 2, (const void*)&k_interp<EeMumu, float, 2>, 256, 1});
  t.push_back({RW_EE_MUMU, RW_FP32, 4, (const void*)&k_reweight<EeMumu, float, 4>});
  t.push_back({RW_EE_MUMU, RW_FP32, 4, (const void*)&k_interp<EeMumu, float, 4>, 256, 1});
}

}  // namespace rw
