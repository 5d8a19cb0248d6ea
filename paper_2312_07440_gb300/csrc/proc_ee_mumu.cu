// e+ e- -> mu+ mu- kernel variants.
#include "../../include/rwgt.h"
#include "kernels.cuh"
#include "procs.cuh"
#include "registry.h"

namespace rw {

void register_ee_mumu(std::vector<KernelEntry>& t, ProcStatic& s) {
  s = {4, 16, 1, 2, 1, 1, 0, 0, 4};
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
