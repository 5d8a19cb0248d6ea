// Internal: table of compiled kernel variants, filled by the per-process
// translation units (proc_*.cu) and looked up by the C ABI (rw_abi.cu).
#pragma once
#include <vector>

namespace rw {

struct KernelEntry {
  int process;       // RW_* process id
  int mode;          // RW_FP64 / RW_FP32
  int lane_bits;     // helicity slices per event = 2^lane_bits
  const void* func;  // __global__ k_reweight<...>(RwArgs) or k_interp<...>(InterpArgs)
  int max_block = 256;  // threads per block the variant supports
  int kind = 0;         // 0: k_reweight, 1: k_interp (interpolation surrogate), 2: k_amp_store
  int smem_per_thread = 0;  // dynamic shared memory of the amplitude code (bytes per thread)
  const void* func2 = nullptr;  // kind 2: the colour pass k_colour_tc<...>(RwArgs, int*)
};

// a k_reweight_multi instantiation: processes in its template order, each
// with its lanes per event (2^lane_bits), one precision mode for all
struct MultiEntry {
  int mode;
  int n;
  int process[4];
  int lane_bits[4];
  const void* func;
  int smem_per_thread;  // dynamic shared memory of the amplitude code (bytes per thread)
};

struct ProcStatic {
  int n_external, n_helicities, n_colour_flows, n_diagrams, colour_den, n_ident, n_gluons;
  long long flops_hel_sum;
  int max_lane_bits;  // helicity loop levels that can be mapped to lanes
};

void register_multi(std::vector<MultiEntry>& t);
void register_ee_mumu(std::vector<KernelEntry>& t, ProcStatic& s);
void register_ee_5a_fp64(std::vector<KernelEntry>& t);
void register_ee_5a_fp32(std::vector<KernelEntry>& t);
void static_ee_5a(ProcStatic& s);
#define RW_DECLARE_QCD(name)                              \
  void register_##name##_fp64(std::vector<KernelEntry>& t); \
  void register_##name##_fp32(std::vector<KernelEntry>& t); \
  void static_##name(ProcStatic& s);                          \
  void register_##name##_mixed(std::vector<KernelEntry>& t);
void register_gg_ttgg_store_fp16(std::vector<KernelEntry>& t);
void register_gg_ttgg_store_bf16(std::vector<KernelEntry>& t);
RW_DECLARE_QCD(gg_tt)
RW_DECLARE_QCD(gg_ttg)
RW_DECLARE_QCD(gg_ttgg)
#undef RW_DECLARE_QCD

}  // namespace rw
