// C ABI of librwgt.so (declared in include/rwgt.h): context, argument
// validation, parameter derivation and kernel launches.  Every step of the
// per-event path runs in the kernels of proc_*.cu; this file only prepares
// the per-point constants (O(1) per parameter point) and launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/rwgt.h"
#include "colour_tc.cuh"
#include "kernels.cuh"
#include "registry.h"

using rw::KernelEntry;
using rw::PointDev;
using rw::ProcStatic;
using rw::RwArgs;

namespace {

constexpr int GRID_CAP = 8192;
constexpr int NPROC = 5;

struct Registry {
  std::vector<KernelEntry> kernels;
  ProcStatic st[NPROC];
  Registry() {
    rw::register_ee_mumu(kernels, st[RW_EE_MUMU]);
    rw::register_gg_tt_mixed(kernels);
    rw::register_gg_ttg_mixed(kernels);
    rw::register_gg_ttgg_mixed(kernels);
    rw::register_gg_ttgg_store_fp16(kernels);
    rw::register_gg_ttgg_store_bf16(kernels);
    rw::register_gg_tt_fp64(kernels);
    rw::register_gg_tt_fp32(kernels);
    rw::static_gg_tt(st[RW_GG_TT]);
    rw::register_gg_ttg_fp64(kernels);
    rw::register_gg_ttg_fp32(kernels);
    rw::static_gg_ttg(st[RW_GG_TTG]);
    rw::register_gg_ttgg_fp64(kernels);
    rw::register_gg_ttgg_fp32(kernels);
    rw::static_gg_ttgg(st[RW_GG_TTGG]);
    rw::register_ee_5a_fp64(kernels);
    rw::register_ee_5a_fp32(kernels);
    rw::static_ee_5a(st[RW_EE_5A]);
  }
  const KernelEntry* find(int process, int mode, int lb, int kind = 0) const {
    for (const auto& k : kernels)
      if (k.process == process && k.mode == mode && k.lane_bits == lb && k.kind == kind) return &k;
    return nullptr;
  }
};

const Registry& registry() {
  static Registry r;
  return r;
}

// default lanes per event (2^bits) per process and mode, before tuning
int default_lane_bits(int process, int mode) {
  switch (process) {
    case RW_EE_MUMU: return 2;
    case RW_GG_TT: return 0;
    case RW_GG_TTG: return 0;
    case RW_GG_TTGG: return mode == RW_FP64 ? 1 : 2;
    case RW_EE_5A: return 0;
  }
  return 0;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

struct rw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int process = -1, mode = -1;
  bool have_p0 = false;
  rw_params p0{};
  std::vector<rw_params> pts;
  const double* mom = nullptr;
  const double* w = nullptr;
  int64_t E = 0;
  int64_t ld = 0;  // row stride of the momenta (the E of rw_load_events)
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int lane_bits = -1, block = 0;
  int smem_optin = 0;  // largest dynamic shared memory a block may opt in to (bytes)
  int smem_per_sm = 0;  // shared memory of one SM (bytes)
  std::string err;
  double* h_stage = nullptr;  // pinned [RW_MAX_POINTS + 2]
  std::map<std::tuple<const void*, int, size_t>, int> occ;
  bool deferred_last = false;  // the last launch ran the separate tensor-core colour pass
  // the separate colour pass's buffers: the attached workspace past its core,
  // when the caller attached it through rw_load_events (the host-buffer and
  // event-file entry points lay out their own buffers there)
  unsigned char* defer_ws = nullptr;
  size_t defer_room = 0;
  // rw_reweight_host pipeline: copy stream and events, created on first use
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> events;
};

namespace {

int fail(rw_ctx* c, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(rw_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

int cuda_fail(rw_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();  // the error is reported here: do not leave it for the caller's next CUDA call
  return fail(c, RW_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

bool finite_params(const rw_params& p) {
  const double v[8] = {p.alpha_s, p.m_t, p.w_t, p.yt_scale, p.alpha_em_inv, p.G_F, p.m_Z, p.w_Z};
  for (double x : v)
    if (!isfinite(x)) return false;
  return true;
}

int check_params(rw_ctx* c, const rw_params& p) {
  if (!finite_params(p)) return fail(c, RW_ERR_PARAM, "parameters must be finite");
  if (c->process == RW_EE_5A) {
    if (!(p.alpha_em_inv > 0)) return fail(c, RW_ERR_PARAM, "alpha_em_inv must be > 0");
  } else if (c->process == RW_EE_MUMU) {
    if (!(p.alpha_em_inv > 0 && p.G_F > 0 && p.m_Z > 0 && p.w_Z >= 0))
      return fail(c, RW_ERR_PARAM, "need alpha_em_inv > 0, G_F > 0, m_Z > 0, w_Z >= 0");
    const double a = 1.0 / p.alpha_em_inv;
    const double disc = 0.25 * pow(p.m_Z, 4) - M_PI * a * p.m_Z * p.m_Z / (sqrt(2.0) * p.G_F);
    if (!(disc >= 0)) return fail(c, RW_ERR_PARAM, "no real M_W for these (alpha, G_F, M_Z)");
  } else {
    if (!(p.alpha_s > 0)) return fail(c, RW_ERR_PARAM, "alpha_s must be > 0");
    if (!(p.m_t > 0)) return fail(c, RW_ERR_PARAM, "m_t must be > 0");
    if (p.w_t != 0.0) return fail(c, RW_ERR_PARAM, "w_t must be 0 (all top propagators are off shell)");
  }
  return RW_OK;
}

bool moves_possible(const rw_ctx* c) { return c->process >= RW_GG_TT && c->process <= RW_GG_TTGG; }

// a top-mass change moves the event onto the new mass shell (QCD processes)
bool moves_event(const rw_ctx* c, const rw_params& pt) {
  return c->process >= RW_GG_TT && c->process <= RW_GG_TTGG && pt.m_t != c->p0.m_t;
}

// per-evaluation constants (derived couplings), computed once per point
PointDev make_point(const rw_ctx* c, const rw_params& p, bool reshuffle) {
  PointDev d{};
  const ProcStatic& s = registry().st[c->process];
  d.m_t = p.m_t;
  d.reshuffle = reshuffle ? 1 : 0;
  if (c->process == RW_EE_MUMU) {
    const double alpha = 1.0 / p.alpha_em_inv, MZ = p.m_Z;
    const double MW2 = 0.5 * MZ * MZ + sqrt(0.25 * MZ * MZ * MZ * MZ - M_PI * alpha * MZ * MZ / (sqrt(2.0) * p.G_F));
    const double sw2 = 1.0 - MW2 / (MZ * MZ), sw = sqrt(sw2), cw = sqrt(1.0 - sw2);
    d.e = sqrt(4.0 * M_PI * alpha);
    // lepton: T3 = -1/2, Q = -1
    d.gL = d.e * (-0.5 + sw2) / (sw * cw);
    d.gR = d.e * sw2 / (sw * cw);
    d.MZ = MZ;
    d.WZ = p.w_Z;
    d.cscale = 1.0;
  } else if (c->process == RW_EE_5A) {
    // e^(2n) / (4 n!): couplings stripped from the amplitude, spin average, identical photons
    const double e2 = 4.0 * M_PI / p.alpha_em_inv;
    double epow = 1.0, nfact = 1.0;
    for (int i = 1; i <= s.n_ident; ++i) {
      epow *= e2;
      nfact *= i;
    }
    d.cscale = epow / (4.0 * nfact);
  } else {
    double ident_fact = 1.0;
    for (int i = 2; i <= s.n_ident; ++i) ident_fact *= i;
    const double g2 = 4.0 * M_PI * p.alpha_s;
    double gpow = 1.0;
    for (int i = 0; i < s.n_gluons; ++i) gpow *= g2;
    d.cscale = gpow / (4.0 * 64.0 * ident_fact * s.colour_den);
  }
  return d;
}

// workspace: 256-B header (ticket, bad-event counter; sigma [P+1] and the
// bad-event count from byte 64), block partials double2 [GRID_CAP][P+1], then
// the results' (sum, compensation) pairs double2 [P+1]
size_t ws_pairs_offset(int P) { return 256 + align256(8 * (size_t)(P + 2)) + (size_t)GRID_CAP * (P + 1) * 16; }
size_t ws_core_bytes(int P) { return ws_pairs_offset(P) + align256(16 * (size_t)(P + 1)); }

// Mixed modes with a compiled separate colour pass (k_amp_store + k_colour_tc)
// run it for up to DEFER_MAX_POINTS points when the attached workspace holds
// its amplitude buffers, placed after a core region sized for that many points.
bool defer_compiled(int process, int mode) {
  for (const auto& k : registry().kernels)
    if (k.process == process && k.mode == mode && k.kind == 2) return true;
  return false;
}
rw::DeferLayout defer_layout(int process, int npts, long long E) {
  const ProcStatic& st = registry().st[process];
  return rw::DeferLayout(npts, rw::align_up(E, 128), st.n_colour_flows, st.n_helicities / 2);
}
size_t defer_offset() { return ws_core_bytes(rw::DEFER_MAX_POINTS); }

int check_dev_ptr(rw_ctx* c, const void* p, const char* name) {
  if (!p) return fail(c, RW_ERR_NULL, "%s is NULL", name);
  if (reinterpret_cast<uintptr_t>(p) % 8) return fail(c, RW_ERR_ALIGN, "%s not 8-byte aligned", name);
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(c, e, name);
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(c, RW_ERR_ARG, "%s is not device memory", name);
  if (at.type == cudaMemoryTypeDevice && at.device != c->device)
    return fail(c, RW_ERR_ARG, "%s lives on device %d, context on %d", name, at.device, c->device);
  return RW_OK;
}

int ready(rw_ctx* c, bool need_events) {
  if (!c) return RW_ERR_NULL;
  if (c->process < 0) return fail(c, RW_ERR_STATE, "no process set");
  if (!c->have_p0) return fail(c, RW_ERR_STATE, "no original parameters set");
  if (need_events && !c->mom) return fail(c, RW_ERR_STATE, "no events loaded");
  return RW_OK;
}

// Raise a kernel's dynamic shared-memory limit to at least `smem` bytes.  The
// limit belongs to the function, not to a context or a launch shape, so it is
// only ever raised: lowering it for a smaller launch would make the next
// larger launch of the same kernel fail.
cudaError_t ensure_smem(const void* func, size_t smem) {
  if (smem == 0) return cudaSuccess;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// a kernel's static shared memory (its __shared__ arrays), which counts
// against the same per-block limit as the dynamic part
size_t static_smem(const void* func) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return fa.sharedSizeBytes;
}

// launch the fused kernel; `points` empty => single evaluation mode
// launch shape of the current kernel variant: the entry, threads per block,
// lanes per event, shared memory and resident blocks per SM for P points
struct Shape {
  const KernelEntry* k;
  int block, lanes, per_sm;
  size_t smem;
};

int shape(rw_ctx* c, int P, Shape& sh) {
  const int lb = c->lane_bits >= 0 ? c->lane_bits : default_lane_bits(c->process, c->mode);
  const KernelEntry* k = registry().find(c->process, c->mode, lb);
  if (!k) return fail(c, RW_ERR_MODE, "no kernel for process %d mode %d lane_bits %d", c->process, c->mode, lb);
  const int block = c->block > 0 ? c->block : 128;
  if (block > k->max_block) return fail(c, RW_ERR_ARG, "block %d above this variant's %d", block, k->max_block);
  const size_t smem = (size_t)k->smem_per_thread * block + (size_t)(block / 32) * (P + 1) * sizeof(double2);
  const size_t smem_total = smem + static_smem(k->func);
  if (c->smem_optin > 0 && smem_total > (size_t)c->smem_optin)
    return fail(c, RW_ERR_ARG,
                "block %d with %d points needs %zu bytes of shared memory, more than the %d a block may have", block, P,
                smem_total, c->smem_optin);
  // opt in to more than the default 48 KB of dynamic shared memory
  if (cudaError_t e = ensure_smem(k->func, smem); e != cudaSuccess)
    return cuda_fail(c, e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
  auto key = std::make_tuple(k->func, block, smem);
  auto it = c->occ.find(key);
  int per_sm;
  if (it == c->occ.end()) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k->func, block, smem);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) per_sm = 1;
    c->occ[key] = per_sm;
  } else {
    per_sm = it->second;
  }
  sh = {k, block, 1 << lb, per_sm, smem};
  return RW_OK;
}

// the amplitude pass, then the tensor-core colour pass (colour_tc.cuh)
int launch_deferred(rw_ctx* c, RwArgs& a, const KernelEntry* d) {
  const int block = c->block > 0 ? c->block : 128;
  const int lanes = 1 << d->lane_bits;
  if (block > d->max_block || lanes > block) return fail(c, RW_ERR_ARG, "block %d does not fit this variant", block);
  const size_t smem = (size_t)d->smem_per_thread * block;
  const size_t smem_total = smem + static_smem(d->func);
  if (c->smem_optin > 0 && smem_total > (size_t)c->smem_optin)
    return fail(c, RW_ERR_ARG, "block %d needs %zu bytes of shared memory (%d per thread), more than the %d a block may have",
                block, smem_total, d->smem_per_thread, c->smem_optin);
  for (const auto& [f, bytes] : {std::make_pair(d->func, smem), std::make_pair(d->func2, rw::CT_SMEM)})
    if (cudaError_t e = ensure_smem(f, bytes); e != cudaSuccess)
      return cuda_fail(c, e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
  // the colour pass: as many blocks per SM as its shared memory allows (the
  // default carveout may leave room for one)
  if (cudaError_t e = cudaFuncSetAttribute(d->func2, cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxShared);
      e != cudaSuccess)
    return cuda_fail(c, e, "cudaFuncSetAttribute(PreferredSharedMemoryCarveout)");
  auto occupancy = [c](const void* f, int threads, size_t bytes, int& per_sm) {
    const auto key = std::make_tuple(f, threads, bytes);
    const auto it = c->occ.find(key);
    if (it != c->occ.end()) {
      per_sm = it->second;
      return cudaSuccess;
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, bytes);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    c->occ[key] = per_sm;
    return cudaSuccess;
  };
  int per_sm = 1;
  cudaError_t e = occupancy(d->func, block, smem, per_sm);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  // colour-pass blocks per SM: by shared memory (1 KB of it reserved per
  // block) and by tensor memory (128 of 512 columns each); the occupancy
  // query does not see the carveout set above
  const int per_sm_c = std::max(
      1, std::min<int>(4, c->smem_per_sm / (int)(rw::CT_SMEM + static_smem(d->func2) + 1024)));
  const long long need = (a.E * lanes + block - 1) / block;
  const int grid = (int)std::max(1LL, std::min<long long>({(long long)GRID_CAP, (long long)per_sm * c->sm_count, need}));
  const long long tiles = (a.E + 127) / 128;
  const int grid_c =
      (int)std::max(1LL, std::min<long long>({(long long)GRID_CAP, (long long)per_sm_c * c->sm_count, tiles}));
  int* err = reinterpret_cast<int*>(reinterpret_cast<char*>(a.ticket) + 16);
  if ((e = cudaMemsetAsync(err, 0, sizeof(int), c->stream)) != cudaSuccess) return cuda_fail(c, e, "memset");
  void* args[] = {&a};
  if ((e = cudaLaunchKernel(d->func, dim3(grid), dim3(block), args, smem, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "amplitude kernel launch");
  void* args2[] = {&a, &err};
  if ((e = cudaLaunchKernel(d->func2, dim3(grid_c), dim3(rw::CT_THREADS), args2, rw::CT_SMEM, c->stream)) !=
      cudaSuccess)
    return cuda_fail(c, e, "colour kernel launch");
  c->deferred_last = true;
  return RW_OK;
}

int launch(rw_ctx* c, RwArgs& a) {
  c->deferred_last = false;
  if (a.defer) {
    const int lb = c->lane_bits >= 0 ? c->lane_bits : default_lane_bits(c->process, c->mode);
    if (const KernelEntry* d = registry().find(c->process, c->mode, lb, 2)) return launch_deferred(c, a, d);
  }
  Shape sh;
  int rc = shape(c, a.P, sh);
  if (rc) return rc;
  const KernelEntry* k = sh.k;
  const int block = sh.block, lanes = sh.lanes, per_sm = sh.per_sm;
  const size_t smem = sh.smem;
  const long long need = (a.E * lanes + block - 1) / block;
  const int grid = (int)std::max(1LL, std::min<long long>({(long long)GRID_CAP, (long long)per_sm * c->sm_count, need}));
  void* args[] = {&a};
  cudaError_t e = cudaLaunchKernel(k->func, dim3(grid), dim3(block), args, smem, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  return RW_OK;
}

void fill_ws(rw_ctx* c, RwArgs& a, int P);
void fill_core(char* b, RwArgs& a, int P);

// the separate colour pass's buffers for npts evaluations of the attached
// events, when it applies (else the fused kernel runs)
void set_defer(rw_ctx* c, RwArgs& a, int npts) {
  a.defer = nullptr;
  a.defer_ld = 0;
  if (!c->defer_ws || npts - 1 > rw::DEFER_MAX_POINTS || !defer_compiled(c->process, c->mode)) return;
  const rw::DeferLayout L = defer_layout(c->process, npts, c->E);
  if ((size_t)L.total > c->defer_room) return;
  a.defer = c->defer_ws;
  a.defer_ld = L.ld;
}

// the fused reweight of all attached events and points
void reweight_args(rw_ctx* c, RwArgs& a, double* d_wnew, double* d_ratio, double* d_me0, double* d_me_pts) {
  const int P = (int)c->pts.size();
  a.mom = c->mom;
  a.w = c->w;
  a.E = c->E;
  a.ld = c->ld;
  a.me0 = d_me0;
  a.me_pts = d_me_pts;
  a.ratio = d_ratio;
  a.wnew = d_wnew;
  a.P = P;
  a.me_only = 0;
  a.pt[0] = make_point(c, c->p0, false);
  for (int j = 0; j < P; ++j) {
    const bool moved = moves_event(c, c->pts[j]);
    a.pt[1 + j] = make_point(c, c->pts[j], moved);
  }
  fill_ws(c, a, P);
  set_defer(c, a, P + 1);
}

void fill_ws(rw_ctx* c, RwArgs& a, int P) { fill_core(c->ws, a, P); }

// the reduction slots of a launch of P points in a core region of ws_core_bytes(P)
void fill_core(char* b, RwArgs& a, int P) {
  a.ticket = reinterpret_cast<unsigned int*>(b);
  a.nbad_count = reinterpret_cast<unsigned long long*>(b + 8);
  a.sigma = reinterpret_cast<double*>(b + 64);
  a.nbad_out = reinterpret_cast<unsigned long long*>(b + 64 + 8 * (size_t)(P + 1));
  a.block_part = reinterpret_cast<double2*>(b + 256 + align256(8 * (size_t)(P + 2)));
  a.sigma_pair = reinterpret_cast<double2*>(b + ws_pairs_offset(P));
}

}  // namespace

extern "C" {

int rw_create(rw_ctx** out, int device, void* stream) {
  if (!out) return RW_ERR_NULL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return RW_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return RW_ERR_ARG;
  DeviceGuard g(device);
  if (!g.ok) return RW_ERR_CUDA;
  rw_ctx* c = new rw_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
      cudaMallocHost(&c->h_stage, sizeof(double) * (RW_MAX_POINTS + 4)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return RW_ERR_CUDA;
  }
  (void)registry();
  *out = c;
  return RW_OK;
}

int rw_destroy(rw_ctx* c) {
  if (!c) return RW_ERR_NULL;
  DeviceGuard g(c->device);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  for (cudaEvent_t ev : c->events) cudaEventDestroy(ev);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  delete c;
  return RW_OK;
}

const char* rw_last_error(const rw_ctx* c) { return c ? c->err.c_str() : "null context"; }

int rw_process_info_get(int process, rw_process_info* out) {
  if (!out) return RW_ERR_NULL;
  if (process < 0 || process >= NPROC) return RW_ERR_ARG;
  const ProcStatic& s = registry().st[process];
  out->n_external = s.n_external;
  out->n_helicities = s.n_helicities;
  out->n_colour_flows = s.n_colour_flows;
  out->n_diagrams = s.n_diagrams;
  out->colour_den = s.colour_den;
  out->flops_hel_sum = s.flops_hel_sum;
  return RW_OK;
}

int rw_set_process(rw_ctx* c, int process, int mode) {
  if (!c) return RW_ERR_NULL;
  if (process < 0 || process >= NPROC) return fail(c, RW_ERR_ARG, "unknown process %d", process);
  if (mode < RW_FP64 || mode > RW_MIXED_BF16) return fail(c, RW_ERR_MODE, "unknown mode %d", mode);
  bool any = false;
  for (const auto& k : registry().kernels) any |= k.process == process && k.mode == mode && k.kind == 0;
  if (!any) return fail(c, RW_ERR_MODE, "process %d has no kernels in mode %d", process, mode);
  c->process = process;
  c->mode = mode;
  c->have_p0 = false;
  c->pts.clear();
  c->mom = nullptr;
  c->w = nullptr;
  c->E = 0;
  return RW_OK;
}

int rw_set_params(rw_ctx* c, const rw_params* p) {
  if (!c) return RW_ERR_NULL;
  if (!p) return fail(c, RW_ERR_NULL, "params is NULL");
  if (c->process < 0) return fail(c, RW_ERR_STATE, "set the process first");
  int rc = check_params(c, *p);
  if (rc) return rc;
  c->p0 = *p;
  c->have_p0 = true;
  return RW_OK;
}

int rw_set_reweight_points(rw_ctx* c, const rw_params* pts, int P) {
  if (!c) return RW_ERR_NULL;
  if (!pts) return fail(c, RW_ERR_NULL, "points is NULL");
  if (c->process < 0) return fail(c, RW_ERR_STATE, "set the process first");
  if (P < 1 || P > RW_MAX_POINTS) return fail(c, RW_ERR_ARG, "need 1 <= P <= %d, got %d", RW_MAX_POINTS, P);
  for (int j = 0; j < P; ++j) {
    int rc = check_params(c, pts[j]);
    if (rc) return fail(c, rc, "point %d: %s", j, c->err.c_str());
  }
  if (c->mom && ws_core_bytes(P) > c->ws_bytes)
    return fail(c, RW_ERR_WORKSPACE, "attached workspace too small for %d points", P);
  c->pts.assign(pts, pts + P);
  return RW_OK;
}

int rw_set_tuning(rw_ctx* c, int lane_bits, int block) {
  if (!c) return RW_ERR_NULL;
  if (block != 0 && (block < 32 || block > 256 || block % 32))
    return fail(c, RW_ERR_ARG, "block must be a multiple of 32 in [32, 256]");
  if (lane_bits >= 0 && c->process >= 0) {
    const KernelEntry* k = registry().find(c->process, c->mode, lane_bits);
    if (!k) return fail(c, RW_ERR_MODE, "lane_bits %d not compiled for this process/mode", lane_bits);
    const KernelEntry* d = registry().find(c->process, c->mode, lane_bits, 2);  // separate colour pass
    const int max_block = d ? std::max(k->max_block, d->max_block) : k->max_block;
    if (block > max_block) return fail(c, RW_ERR_ARG, "block above this variant's %d", max_block);
    if ((1 << lane_bits) > (block ? block : 128)) return fail(c, RW_ERR_ARG, "more lanes than threads");
  }
  c->lane_bits = lane_bits;
  c->block = block;
  return RW_OK;
}

int rw_get_tuning(const rw_ctx* c, int* lane_bits, int* block) {
  if (!c || !lane_bits || !block) return RW_ERR_NULL;
  if (c->process < 0) return RW_ERR_STATE;
  *lane_bits = c->lane_bits >= 0 ? c->lane_bits : default_lane_bits(c->process, c->mode);
  *block = c->block > 0 ? c->block : 128;
  return RW_OK;
}

int rw_autotune(rw_ctx* c, int64_t max_events, const char* cache_path, double* ms_out) {
  int rc = ready(c, true);
  if (rc) return rc;
  if (c->pts.empty()) return fail(c, RW_ERR_STATE, "no reweight points set");
  if (max_events <= 0) return fail(c, RW_ERR_ARG, "max_events must be > 0");
  DeviceGuard g(c->device);
  const int P = (int)c->pts.size();
  const int64_t E = std::min<int64_t>(c->E, max_events);
  int ebits = 0;
  while ((int64_t(1) << (ebits + 1)) <= E) ++ebits;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return fail(c, RW_ERR_CUDA, "device properties");
  char key[512];
  snprintf(key, sizeof key, "%s|%d|%d|P%d|E%d", prop.name, c->process, c->mode, P, ebits);
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char line[1024];
      while (fgets(line, sizeof line, f)) {
        char k[512];
        int lb, bl;
        double ms;
        if (sscanf(line, "{\"key\": \"%511[^\"]\", \"lane_bits\": %d, \"block\": %d, \"ms\": %lf}", k, &lb, &bl, &ms) ==
                4 &&
            strcmp(k, key) == 0 && registry().find(c->process, c->mode, lb)) {
          fclose(f);
          c->lane_bits = lb;
          c->block = bl;
          if (ms_out) *ms_out = ms;
          return RW_OK;
        }
      }
      fclose(f);
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(c, RW_ERR_CUDA, "cudaEventCreate");
  const int64_t E_saved = c->E;
  const int lb_saved = c->lane_bits, bl_saved = c->block;
  c->E = E;
  double best = 1e300;
  int best_lb = -1, best_bl = 0;
  static const int blocks[] = {64, 128, 256};
  for (const auto& k : registry().kernels) {
    if (k.process != c->process || k.mode != c->mode || k.kind != 0) continue;
    // with the separate colour pass attached, its amplitude kernel's limit
    const KernelEntry* d = registry().find(c->process, c->mode, k.lane_bits, 2);
    RwArgs probe{};
    probe.P = (int)c->pts.size();
    set_defer(c, probe, probe.P + 1);
    const int max_block = (d && probe.defer) ? d->max_block : k.max_block;
    for (int bl : blocks) {
      if ((1 << k.lane_bits) > bl || bl > max_block) continue;
      c->lane_bits = k.lane_bits;
      c->block = bl;
      float t[3];
      bool ok = true;
      for (int it = -1; it < 3 && ok; ++it) {
        cudaEventRecord(e0, c->stream);
        ok = rw_reweight_async(c, nullptr, nullptr, nullptr, nullptr) == RW_OK;
        cudaEventRecord(e1, c->stream);
        if (ok && cudaEventSynchronize(e1) == cudaSuccess && it >= 0) cudaEventElapsedTime(&t[it], e0, e1);
      }
      if (!ok) continue;
      std::sort(t, t + 3);
      if (t[1] < best) {
        best = t[1];
        best_lb = k.lane_bits;
        best_bl = bl;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->E = E_saved;
  if (best_lb < 0) {
    c->lane_bits = lb_saved;
    c->block = bl_saved;
    return fail(c, RW_ERR_CUDA, "no variant ran: %s", c->err.c_str());
  }
  c->lane_bits = best_lb;
  c->block = best_bl;
  if (ms_out) *ms_out = best;
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "a")) {
      fprintf(f, "{\"key\": \"%s\", \"lane_bits\": %d, \"block\": %d, \"ms\": %.6f}\n", key, best_lb, best_bl, best);
      fclose(f);
    }
  }
  return RW_OK;
}

size_t rw_workspace_bytes(const rw_ctx* c, int64_t E) {
  if (!c) return 0;
  const int P = std::max<int>(1, (int)c->pts.size());
  if (c->process >= 0 && E > 0 && P <= rw::DEFER_MAX_POINTS && defer_compiled(c->process, c->mode))
    return defer_offset() + (size_t)defer_layout(c->process, P + 1, E).total;
  return ws_core_bytes(P);
}

static int load_events(rw_ctx* c, const double* d_mom, const double* d_w, int64_t E, void* d_ws, size_t ws_bytes,
                       bool own_layout);

int rw_load_events(rw_ctx* c, const double* d_mom, const double* d_w, int64_t E, void* d_ws, size_t ws_bytes) {
  return load_events(c, d_mom, d_w, E, d_ws, ws_bytes, false);
}

// own_layout: the caller (an entry point of this library) keeps its own
// buffers after the workspace's core, so the colour pass gets none
static int load_events(rw_ctx* c, const double* d_mom, const double* d_w, int64_t E, void* d_ws, size_t ws_bytes,
                bool own_layout) {
  if (!c) return RW_ERR_NULL;
  if (c->process < 0) return fail(c, RW_ERR_STATE, "set the process first");
  if (E <= 0) return fail(c, RW_ERR_ARG, "n_events must be > 0, got %lld", (long long)E);
  if (E > (int64_t(1) << 40)) return fail(c, RW_ERR_ARG, "n_events too large");
  DeviceGuard g(c->device);
  int rc;
  if ((rc = check_dev_ptr(c, d_mom, "momenta"))) return rc;
  if ((rc = check_dev_ptr(c, d_w, "weights"))) return rc;
  if ((rc = check_dev_ptr(c, d_ws, "workspace"))) return rc;
  if (reinterpret_cast<uintptr_t>(d_ws) % 16) return fail(c, RW_ERR_ALIGN, "workspace not 16-byte aligned");
  const size_t need = ws_core_bytes(std::max<int>(1, (int)c->pts.size()));  // the colour pass's buffers are optional
  if (ws_bytes < need) return fail(c, RW_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, need);
  cudaError_t e = cudaMemsetAsync(d_ws, 0, 256, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
  c->mom = d_mom;
  c->w = d_w;
  c->E = E;
  c->ld = E;
  c->ws = static_cast<char*>(d_ws);
  c->ws_bytes = ws_bytes;
  c->defer_ws = nullptr;
  c->defer_room = 0;
  if (!own_layout && ws_bytes > defer_offset()) {
    c->defer_ws = reinterpret_cast<unsigned char*>(d_ws) + defer_offset();
    c->defer_room = ws_bytes - defer_offset();
  }
  return RW_OK;
}

int rw_eval_me(rw_ctx* c, int point, double* d_me) {
  int rc = ready(c, true);
  if (rc) return rc;
  if (point < -1 || point >= (int)c->pts.size()) return fail(c, RW_ERR_ARG, "point %d out of range", point);
  DeviceGuard g(c->device);
  if ((rc = check_dev_ptr(c, d_me, "me_out"))) return rc;
  RwArgs a{};
  a.mom = c->mom;
  a.w = c->w;
  a.E = c->E;
  a.ld = c->ld;
  a.me0 = d_me;
  a.P = 0;
  a.me_only = 1;
  if (point < 0) {
    a.pt[0] = make_point(c, c->p0, false);
  } else {
    const bool moved = moves_event(c, c->pts[point]);
    a.pt[0] = make_point(c, c->pts[point], moved);
  }
  fill_ws(c, a, 0);
  set_defer(c, a, 1);
  return launch(c, a);
}

int rw_reweight_async(rw_ctx* c, double* d_wnew, double* d_ratio, double* d_me0, double* d_me_pts) {
  int rc = ready(c, true);
  if (rc) return rc;
  if (c->pts.empty()) return fail(c, RW_ERR_STATE, "no reweight points set");
  DeviceGuard g(c->device);
  if (d_wnew && (rc = check_dev_ptr(c, d_wnew, "wnew"))) return rc;
  if (d_ratio && (rc = check_dev_ptr(c, d_ratio, "ratio"))) return rc;
  if (d_me0 && (rc = check_dev_ptr(c, d_me0, "me0"))) return rc;
  if (d_me_pts && (rc = check_dev_ptr(c, d_me_pts, "me_pts"))) return rc;
  const int P = (int)c->pts.size();
  if (ws_core_bytes(P) > c->ws_bytes) return fail(c, RW_ERR_WORKSPACE, "workspace too small for %d points", P);
  RwArgs a{};
  reweight_args(c, a, d_wnew, d_ratio, d_me0, d_me_pts);
  return launch(c, a);
}

int rw_get_results(rw_ctx* c, double* h_sigma, double* h_sigma_orig, int64_t* h_n_bad) {
  int rc = ready(c, true);
  if (rc) return rc;
  if (c->pts.empty()) return fail(c, RW_ERR_STATE, "no reweight points set");
  DeviceGuard g(c->device);
  const int P = (int)c->pts.size();
  cudaError_t e = cudaMemcpyAsync(c->h_stage, c->ws + 64, 8 * (size_t)(P + 2), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync");
  if (c->deferred_last &&
      (e = cudaMemcpyAsync(c->h_stage + P + 2, c->ws + 16, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) !=
          cudaSuccess)
    return cuda_fail(c, e, "cudaMemcpyAsync");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  if (c->deferred_last) {
    int flag = 0;
    memcpy(&flag, c->h_stage + P + 2, sizeof(int));
    if (flag) return fail(c, RW_ERR_CUDA, "a tensor-core colour pass wait gave up (code %d): results invalid", flag);
  }
  if (h_sigma) memcpy(h_sigma, c->h_stage, 8 * (size_t)P);
  if (h_sigma_orig) *h_sigma_orig = c->h_stage[P];
  unsigned long long nb;
  memcpy(&nb, c->h_stage + P + 1, 8);
  if (h_n_bad) *h_n_bad = (int64_t)nb;
  return nb ? RW_WARN_BAD_EVENTS : RW_OK;
}

int rw_get_result_pairs(rw_ctx* c, double* h_sum, double* h_comp, int64_t* h_n_bad) {
  int rc = ready(c, true);
  if (rc) return rc;
  if (c->pts.empty()) return fail(c, RW_ERR_STATE, "no reweight points set");
  if (!h_sum || !h_comp) return fail(c, RW_ERR_NULL, "h_sum and h_comp are required");
  DeviceGuard g(c->device);
  const int P = (int)c->pts.size();
  std::vector<double2> pairs(P + 1);
  cudaError_t e = cudaMemcpyAsync(pairs.data(), c->ws + ws_pairs_offset(P), 16 * (size_t)(P + 1),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync");
  e = cudaMemcpyAsync(c->h_stage, c->ws + 64 + 8 * (size_t)(P + 1), 8, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  for (int j = 0; j <= P; ++j) {
    h_sum[j] = pairs[j].x;
    h_comp[j] = pairs[j].y;
  }
  unsigned long long nb;
  memcpy(&nb, c->h_stage, 8);
  if (h_n_bad) *h_n_bad = (int64_t)nb;
  return nb ? RW_WARN_BAD_EVENTS : RW_OK;
}

int rw_reweight(rw_ctx* c, double* d_wnew, double* d_ratio, double* h_sigma, double* h_sigma_orig,
                int64_t* h_n_bad) {
  int rc = rw_reweight_async(c, d_wnew, d_ratio, nullptr, nullptr);
  if (rc < 0) return rc;
  return rw_get_results(c, h_sigma, h_sigma_orig, h_n_bad);
}

size_t rw_workspace_bytes_host(const rw_ctx* c, int64_t E) {
  if (!c || c->process < 0 || E <= 0) return 0;
  const int N = registry().st[c->process].n_external;
  const size_t P = std::max<size_t>(1, c->pts.size());
  return ws_core_bytes((int)P) + align256(16 * (P + 1)) + align256(8 * 4 * (size_t)N * E) +
         align256(8 * (size_t)E) + align256(8 * P * E);
}

// The events are processed in chunks whose size is a multiple of the threads
// one launch keeps resident: the copy stream moves every chunk to the device
// in order, the kernel of chunk k starts on the context's stream once chunk k
// is in (while later chunks are still arriving), and W' of chunk k goes back
// on the copy stream while chunk k+1 is reweighted; the cross sections are
// carried from launch to launch in (sum, compensation) form, in chunk order
// (deterministic).
int rw_reweight_host(rw_ctx* c, const double* h_mom, const double* h_w, int64_t E, double* h_wnew, double* h_sigma,
                     double* h_sigma_orig, int64_t* h_n_bad, void* d_ws, size_t ws_bytes) {
  if (!c) return RW_ERR_NULL;
  if (!h_mom || !h_w) return fail(c, RW_ERR_NULL, "host momenta/weights are NULL");
  if (c->process < 0 || !c->have_p0 || c->pts.empty()) return fail(c, RW_ERR_STATE, "process/params/points unset");
  if (E <= 0) return fail(c, RW_ERR_ARG, "n_events must be > 0");
  if (ws_bytes < rw_workspace_bytes_host(c, E)) return fail(c, RW_ERR_WORKSPACE, "workspace too small");
  DeviceGuard g(c->device);
  const int N = registry().st[c->process].n_external;
  const int P = (int)c->pts.size();
  char* base = static_cast<char*>(d_ws);
  const size_t core = ws_core_bytes(P);
  double2* d_sacc = reinterpret_cast<double2*>(base + core);
  double* d_mom = reinterpret_cast<double*>(base + core + align256(16 * (size_t)(P + 1)));
  double* d_w = reinterpret_cast<double*>(reinterpret_cast<char*>(d_mom) + align256(8 * 4 * (size_t)N * E));
  double* d_wnew = reinterpret_cast<double*>(reinterpret_cast<char*>(d_w) + align256(8 * (size_t)E));
  int rc = load_events(c, d_mom, d_w, E, d_ws, ws_bytes, true);
  if (rc) return rc;
  Shape sh;
  if ((rc = shape(c, P, sh))) return rc;
  // events one launch keeps resident, and the chunk size: about E/8, rounded
  // up to it; the first chunk is one resident set only (its copy-in is the
  // part of the transfer nothing overlaps)
  const long long resident = std::max(1LL, (long long)sh.per_sm * c->sm_count * sh.block / sh.lanes);
  const long long chunk = std::max(resident, (((E + 7) / 8 + resident - 1) / resident) * resident);
  auto chunk_start = [&](int k) { return k == 0 ? 0LL : std::min<long long>(E, resident + (k - 1) * chunk); };
  const int K = E <= resident ? 1 : 1 + (int)((E - resident + chunk - 1) / chunk);
  cudaError_t e;
  if (K == 1) {
    e = cudaMemcpyAsync(d_mom, h_mom, 8 * 4 * (size_t)N * E, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_w, h_w, 8 * (size_t)E, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
    rc = rw_reweight_async(c, h_wnew ? d_wnew : nullptr, nullptr, nullptr, nullptr);
    if (rc < 0) return rc;
    if (h_wnew) {
      e = cudaMemcpyAsync(h_wnew, d_wnew, 8 * (size_t)P * E, cudaMemcpyDeviceToHost, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
    }
    return rw_get_results(c, h_sigma, h_sigma_orig, h_n_bad);
  }
  if (!c->copy_stream && (e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(c, e, "cudaStreamCreateWithFlags");
  while ((int)c->events.size() < 2 * K + 2) {
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(c, e, "cudaEventCreateWithFlags");
    c->events.push_back(ev);
  }
  cudaStream_t cs = c->copy_stream;
  // the copies start after the work already queued on the context's stream
  if ((e = cudaEventRecord(c->events[0], c->stream)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(cs, c->events[0], 0)) != cudaSuccess)
    return cuda_fail(c, e, "stream ordering");
  const size_t row = 8 * (size_t)E;
  // all copies in first (the copy stream is in order: a copy-out queued
  // between them would hold the next chunk's copy-in behind a kernel)
  for (int kc = 0; kc < K; ++kc) {
    const long long e0 = chunk_start(kc), n = chunk_start(kc + 1) - e0;
    e = cudaMemcpy2DAsync(d_mom + e0, row, h_mom + e0, row, 8 * (size_t)n, 4 * (size_t)N, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_w + e0, h_w + e0, 8 * (size_t)n, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(c->events[2 + 2 * kc], cs);
    if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  }
  for (int kc = 0; kc < K; ++kc) {
    const long long e0 = chunk_start(kc), n = chunk_start(kc + 1) - e0;
    cudaEvent_t ready = c->events[2 + 2 * kc], done = c->events[3 + 2 * kc];
    if ((e = cudaStreamWaitEvent(c->stream, ready, 0)) != cudaSuccess) return cuda_fail(c, e, "stream ordering");
    RwArgs a{};
    reweight_args(c, a, h_wnew ? d_wnew + e0 : nullptr, nullptr, nullptr, nullptr);
    a.mom = d_mom + e0;
    a.w = d_w + e0;
    a.E = n;
    a.ld = E;
    a.ldo = E;
    a.sigma_acc = d_sacc;
    a.accumulate = kc > 0;
    if ((rc = launch(c, a))) return rc;
    if (h_wnew) {
      e = cudaEventRecord(done, c->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, done, 0);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(h_wnew + e0, row, d_wnew + e0, row, 8 * (size_t)n, (size_t)P, cudaMemcpyDeviceToHost, cs);
      if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
    }
  }
  // the context's stream (and so rw_get_results) waits for the last copies
  if ((e = cudaEventRecord(c->events[1], cs)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(c->stream, c->events[1], 0)) != cudaSuccess)
    return cuda_fail(c, e, "stream ordering");
  return rw_get_results(c, h_sigma, h_sigma_orig, h_n_bad);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// rw_reweight_noalloc: the fused reweight with its scratch in a fixed device
// array of this file instead of a caller-provided workspace.  See rwgt.h.
// ---------------------------------------------------------------------------
namespace {

constexpr int NOALLOC_MAX_GRID = 2048;
constexpr size_t NOALLOC_HEADER = 256;  // ticket (u32 at 0), bad-event counter (u64 at 8)
static_assert(RW_NOALLOC_SCRATCH_BYTES ==
                  NOALLOC_HEADER + (size_t)NOALLOC_MAX_GRID * (RW_NOALLOC_MAX_POINTS + 1) * sizeof(double2),
              "scratch size in rwgt.h out of step");

// Shared by every call on a device; the module keeps it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RW_NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Error text without growing the context's string (no host allocation):
// every message below fits the string's smallest capacity (15 characters).
int noalloc_fail(rw_ctx* c, int code, const char* msg) {
  if (c) c->err.assign(msg, std::min(strlen(msg), c->err.capacity()));
  return code;
}

// Device address of the scratch array on the current device (set up once per
// device, with that device current).
void* noalloc_scratch(int device) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_noalloc_addr[device] = ptr;
  }
  return g_noalloc_addr[device];
}

bool noalloc_dev_ptr_ok(const void* p, int device) {
  if (!p || reinterpret_cast<uintptr_t>(p) % 8) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == device;
}

}  // namespace

extern "C" int rw_reweight_noalloc(rw_ctx* c, const double* d_mom, const double* d_w, int64_t E, double* d_wnew,
                                   double* d_ratio, double* d_sigma, unsigned long long* d_n_bad) {
  if (!c) return RW_ERR_NULL;
  if (c->process < 0 || !c->have_p0 || c->pts.empty())
    return noalloc_fail(c, RW_ERR_STATE, "state not set");
  const int P = (int)c->pts.size();
  if (P > RW_NOALLOC_MAX_POINTS) return noalloc_fail(c, RW_ERR_ARG, "too many points");
  if (E <= 0 || E > (int64_t(1) << 40)) return noalloc_fail(c, RW_ERR_ARG, "bad n_events");
  if (c->device < 0 || c->device >= NOALLOC_MAX_DEVICES) return noalloc_fail(c, RW_ERR_ARG, "bad device");
  DeviceGuard g(c->device);
  if (!g.ok) return noalloc_fail(c, RW_ERR_CUDA, "cudaSetDevice");
  if (!d_mom || !d_w || !d_sigma || !d_n_bad) return noalloc_fail(c, RW_ERR_NULL, "NULL pointer");
  if (!noalloc_dev_ptr_ok(d_mom, c->device) || !noalloc_dev_ptr_ok(d_w, c->device) ||
      !noalloc_dev_ptr_ok(d_sigma, c->device) || !noalloc_dev_ptr_ok(d_n_bad, c->device) ||
      (d_wnew && !noalloc_dev_ptr_ok(d_wnew, c->device)) || (d_ratio && !noalloc_dev_ptr_ok(d_ratio, c->device)))
    return noalloc_fail(c, RW_ERR_ARG, "bad buffer");
  char* scratch = static_cast<char*>(noalloc_scratch(c->device));
  if (!scratch) return noalloc_fail(c, RW_ERR_CUDA, "scratch lookup");

  const int lb = c->lane_bits >= 0 ? c->lane_bits : default_lane_bits(c->process, c->mode);
  const KernelEntry* k = registry().find(c->process, c->mode, lb);
  if (!k) return noalloc_fail(c, RW_ERR_MODE, "no kernel");
  const int block = c->block > 0 ? c->block : 128;
  if (block > k->max_block) return noalloc_fail(c, RW_ERR_ARG, "block too large");
  const size_t smem = (size_t)k->smem_per_thread * block + (size_t)(block / 32) * (P + 1) * sizeof(double2);
  if (c->smem_optin > 0 && smem + static_smem(k->func) > (size_t)c->smem_optin)
    return noalloc_fail(c, RW_ERR_ARG, "block too large");
  if (ensure_smem(k->func, smem) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(c, RW_ERR_CUDA, "smem attribute");
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k->func, block, smem) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(c, RW_ERR_CUDA, "occupancy query");
  }
  if (per_sm < 1) per_sm = 1;
  const long long need = (E * (1LL << lb) + block - 1) / block;
  const int grid =
      (int)std::max(1LL, std::min<long long>({(long long)NOALLOC_MAX_GRID, (long long)per_sm * c->sm_count, need}));

  RwArgs a{};
  a.mom = d_mom;
  a.w = d_w;
  a.E = E;
  a.ld = E;
  a.ratio = d_ratio;
  a.wnew = d_wnew;
  a.P = P;
  a.me_only = 0;
  a.pt[0] = make_point(c, c->p0, false);
  for (int j = 0; j < P; ++j) {
    const bool moved = moves_event(c, c->pts[j]);
    a.pt[1 + j] = make_point(c, c->pts[j], moved);
  }
  a.ticket = reinterpret_cast<unsigned int*>(scratch);
  a.nbad_count = reinterpret_cast<unsigned long long*>(scratch + 8);
  a.block_part = reinterpret_cast<double2*>(scratch + NOALLOC_HEADER);
  a.sigma = d_sigma;
  a.nbad_out = d_n_bad;
  // the ticket and the bad-event counter must start at zero
  cudaError_t e = cudaMemsetAsync(scratch, 0, NOALLOC_HEADER, c->stream);
  if (e != cudaSuccess) return noalloc_fail(c, RW_ERR_CUDA, "scratch memset");
  void* args[] = {&a};
  e = cudaLaunchKernel(k->func, dim3(grid), dim3(block), args, smem, c->stream);
  if (e != cudaSuccess) return noalloc_fail(c, RW_ERR_CUDA, "kernel launch");
  return RW_OK;
}

// ---------------------------------------------------------------------------
// Surrogate: features/labels, decision, exact fallback, sigma
// ---------------------------------------------------------------------------
namespace {

struct KappaList {
  float k[RW_MAX_POINTS];
};

// Features x[(p*E + e)][0..n_in): the event's momenta / p_scale after the
// azimuthal rotation about the beam that puts the top's p_T along +x (|M|^2 is
// invariant under it), then (kappa_p - 1)/k_scale, then (room permitting) the
// logarithms of the pairwise invariants, zero padding.  Label
// y = log r / (kappa_p - 1): the network learns the log ratio per unit shift,
// so r = 1 at kappa = 1 holds exactly (y = 0 when kappa_p = 1 or r <= 0).
__global__ void k_features(const double* __restrict__ mom, long long ld, long long E, int N, int P, KappaList kap,
                           int n_in, double inv_ps, double inv_ks, const double* __restrict__ ratio,
                           float* __restrict__ x, float* __restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)P * E) return;
  const int p = (int)(t / E);
  const long long e = t % E;
  const double tx = mom[(long long)(2 * 4 + 1) * ld + e], ty = mom[(long long)(2 * 4 + 2) * ld + e];
  const double pt = sqrt(tx * tx + ty * ty);
  const double c = pt > 0.0 ? tx / pt : 1.0, s = pt > 0.0 ? ty / pt : 0.0;
  float* xr = x + t * n_in;
  int j = 0;
  for (int i = 0; i < N && j + 4 <= n_in; ++i, j += 4) {
    const double px = mom[(long long)(i * 4 + 1) * ld + e], py = mom[(long long)(i * 4 + 2) * ld + e];
    xr[j] = (float)(mom[(long long)(i * 4) * ld + e] * inv_ps);
    xr[j + 1] = (float)((c * px + s * py) * inv_ps);
    xr[j + 2] = (float)((-s * px + c * py) * inv_ps);
    xr[j + 3] = (float)(mom[(long long)(i * 4 + 3) * ld + e] * inv_ps);
  }
  const double dk = (double)kap.k[p] - 1.0;
  if (j < n_in) xr[j++] = (float)(dk * inv_ks);
  // with room for them, the logarithms of the pairwise invariants 2 p_i.p_j / s-hat
  // (i < j; all positive for physical momenta): the propagator denominators are
  // sums of these, and |M|^2 varies over decades as one of them goes to zero,
  // which a logarithmic input spreads out for the network
  if (n_in - j >= N * (N - 1) / 2) {
    double q[8][4];
    for (int i = 0; i < N && i < 8; ++i)
      for (int m = 0; m < 4; ++m) q[i][m] = mom[(long long)(i * 4 + m) * ld + e];
    const double sh = (q[0][0] + q[1][0]) * (q[0][0] + q[1][0]) - (q[0][1] + q[1][1]) * (q[0][1] + q[1][1]) -
                      (q[0][2] + q[1][2]) * (q[0][2] + q[1][2]) - (q[0][3] + q[1][3]) * (q[0][3] + q[1][3]);
    const double ish = sh > 0.0 ? 2.0 / sh : 0.0;
    for (int a = 0; a < N && a < 8; ++a)
      for (int b2 = a + 1; b2 < N && b2 < 8; ++b2)
        xr[j++] = (float)log(fmax((q[a][0] * q[b2][0] - q[a][1] * q[b2][1] - q[a][2] * q[b2][2] -
                                   q[a][3] * q[b2][3]) * ish, 1e-30));
  }
  for (; j < n_in; ++j) xr[j] = 0.0f;
  if (ratio && y) {
    const double r = ratio[t];
    y[t] = (r > 0.0 && fabs(dk) > 1e-12) ? (float)(log(r) / dk) : 0.0f;
  }
}

// Events are recomputed exactly at the points where the network's estimate is
// over the bound: with up to MASK_POINTS points, the events are grouped by
// that set of points (one exact launch per group, with just those points);
// with more, an event over the bound at any point is recomputed at all points.
constexpr int MASK_POINTS = 6;
constexpr int N_GROUPS = 1 << MASK_POINTS;

// Accept W' = exp((kappa-1) mu) W where s + log|kappa-1| <= s_max (the
// network's predicted log error of log r), else mark (event, point) for the
// exact path in the event's bit mask; kappa = 1 gives W' = W exactly.
__global__ void k_decide(const float* __restrict__ out, const double* __restrict__ w, long long E, int P,
                         KappaList kap, float s_max, double* __restrict__ wnew, unsigned* __restrict__ mask) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)P * E) return;
  const int p = (int)(t / E);
  const long long e = t % E;
  const double dk = (double)kap.k[p] - 1.0;
  const float mu = out[2 * t], s = out[2 * t + 1];
  bool accept;
  double lr = 0.0;
  if (fabs(dk) <= 1e-12) {
    accept = true;
  } else {
    lr = dk * (double)mu;
    accept = isfinite(mu) && isfinite(s) && (double)s + log(fabs(dk)) <= (double)s_max;
  }
  wnew[t] = accept ? exp(lr) * w[e] : 0.0;
  if (!accept) atomicOr(mask + e, P <= MASK_POINTS ? 1u << p : 1u);
}

// the group of a marked event: its mask (<= MASK_POINTS points) or group 1 (all points)
__device__ __forceinline__ unsigned group_of(unsigned m, int P) { return (m && P > MASK_POINTS) ? 1u : m; }
__device__ __forceinline__ bool exact_at(unsigned m, int P, int p) {
  return P <= MASK_POINTS ? ((m >> p) & 1u) != 0 : m != 0;
}

// events per group and each marked event's rank in its group
__global__ void k_count_groups(const unsigned* __restrict__ mask, long long E, int P,
                               unsigned long long* __restrict__ count, long long* __restrict__ rank) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const unsigned g = group_of(mask[e], P);
  if (g) rank[e] = (long long)atomicAdd(count + g, 1ull);
}

struct GroupOffsets {
  long long off[N_GROUPS];
};

// the groups' event lists, one after the other (order within a group
// unspecified: each event's exact result does not depend on its place in the
// batch); fallback flags [P][E] (1 = exact)
__global__ void k_place_groups(const unsigned* __restrict__ mask, const long long* __restrict__ rank, long long E,
                               int P, GroupOffsets go, unsigned char* __restrict__ flag,
                               long long* __restrict__ list) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const unsigned m = mask[e];
  const unsigned g = group_of(m, P);
  if (g) list[go.off[g] + rank[e]] = e;
  if (flag)
    for (int p = 0; p < P; ++p) flag[(long long)p * E + e] = exact_at(m, P, p) ? 1 : 0;
}

__global__ void k_gather_events(const double* __restrict__ mom, long long ld, const double* __restrict__ w, int N,
                                 const long long* __restrict__ list, long long n, double* __restrict__ mom_g,
                                 double* __restrict__ w_g) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long e = list[i];
  for (int r = 0; r < 4 * N; ++r) mom_g[(long long)r * n + i] = mom[(long long)r * ld + e];
  w_g[i] = w[e];
}

struct RowMap {
  int row[RW_MAX_POINTS];
};

// row k of v [np][n] to row rows.row[k] of dst [P][E] at the listed events
__global__ void k_scatter(const double* __restrict__ v, const long long* __restrict__ list, long long n, int np,
                          RowMap rows, long long E, double* __restrict__ dst) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)np * n) return;
  const long long k = t / n, i = t % n;
  dst[(long long)rows.row[k] * E + list[i]] = v[t];
}

__device__ __forceinline__ void ts_acc(double& s, double& c, double x, double cx) {
  const double t = s + x, bp = t - s;
  c += cx + ((s - (t - bp)) + (x - bp));
  s = t;
}

// Compensated sums of nrows rows of n doubles (row r at rows + r*stride for
// r < nrows - 1, the last row at `last`): per-(block, row) partials on a
// fixed grid, then one warp per row, in a fixed order (deterministic).
__global__ void k_sum_partials(const double* __restrict__ rows, long long stride, int nrows,
                               const double* __restrict__ last, long long n, double2* __restrict__ part) {
  __shared__ double2 sh[256];
  const int r = blockIdx.y;
  const double* x = r < nrows - 1 ? rows + (long long)r * stride : last;
  double s = 0.0, c = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    ts_acc(s, c, x[i], 0.0);
  sh[threadIdx.x] = make_double2(s, c);
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      double2 a = sh[threadIdx.x];
      const double2 b = sh[threadIdx.x + o];
      ts_acc(a.x, a.y, b.x, b.y);
      sh[threadIdx.x] = a;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)r * gridDim.x + blockIdx.x] = sh[0];
}
__global__ void k_sum_final(const double2* __restrict__ part, int nb, double* __restrict__ out) {
  const int r = blockIdx.x, l = threadIdx.x;
  double s = 0.0, c = 0.0;
  for (int b = l; b < nb; b += 32) ts_acc(s, c, part[(long long)r * nb + b].x, part[(long long)r * nb + b].y);
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
    ts_acc(s, c, s2, c2);
  }
  if (l == 0) out[r] = s + c;
}

constexpr int SUM_BLOCKS = 256;

// sigma'_p of the P rows of W' [P][E] and sigma of W, into sig[P + 1]
cudaError_t row_sums(cudaStream_t st, const double* wnew, long long E, int P, const double* w, double2* part,
                     double* sig) {
  k_sum_partials<<<dim3(SUM_BLOCKS, P + 1), 256, 0, st>>>(wnew, E, P + 1, w, E, part);
  k_sum_final<<<P + 1, 32, 0, st>>>(part, SUM_BLOCKS, sig);
  return cudaGetLastError();
}

struct SurrogateLayout {
  size_t core, x, out, mask, counts, rank, list, mom_g, w_g, wn_g, part, sig, total;
};

SurrogateLayout surrogate_layout(const rw_ctx* c, int n_in) {
  SurrogateLayout L{};
  const size_t P = c->pts.size(), E = (size_t)c->E, N = registry().st[c->process].n_external;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o += align256(bytes);
    return at;
  };
  L.core = take(ws_core_bytes((int)P));
  L.x = take(4 * P * E * n_in);
  L.out = take(4 * P * E * 2);
  L.mask = take(4 * E);
  L.counts = take(8 * N_GROUPS);
  L.rank = take(8 * E);
  L.list = take(8 * E);
  L.mom_g = take(8 * 4 * N * E);
  L.w_g = take(8 * E);
  L.wn_g = take(8 * P * E);
  L.part = take(16 * SUM_BLOCKS * (P + 1));
  L.sig = take(8 * (P + 1));
  L.total = o;
  return L;
}

KappaList kappas(const rw_ctx* c) {
  KappaList k{};
  for (size_t j = 0; j < c->pts.size(); ++j) k.k[j] = (float)(c->pts[j].m_t / c->p0.m_t);
  return k;
}

}  // namespace

extern "C" {

int rw_surrogate_features(rw_ctx* c, int n_in, double p_scale, double k_scale, const double* d_ratio, float* d_x,
                          float* d_y) {
  int rc = ready(c, true);
  if (rc) return rc;
  if (!moves_possible(c)) return fail(c, RW_ERR_MODE, "the surrogate covers the top-mass axis of the QCD processes");
  if (c->pts.empty()) return fail(c, RW_ERR_STATE, "no points set");
  if (!d_x) return fail(c, RW_ERR_NULL, "x is NULL");
  if (n_in < 1 || !(p_scale > 0) || !(k_scale > 0)) return fail(c, RW_ERR_ARG, "bad feature parameters");
  DeviceGuard g(c->device);
  const int P = (int)c->pts.size(), N = registry().st[c->process].n_external;
  const long long tot = (long long)P * c->E;
  k_features<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(c->mom, c->ld, c->E, N, P, kappas(c), n_in,
                                                                   1.0 / p_scale, 1.0 / k_scale, d_ratio, d_x, d_y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RW_OK : cuda_fail(c, e, "features launch");
}

size_t rw_surrogate_workspace_bytes(const rw_ctx* c, int n_in) {
  if (!c || c->process < 0 || !c->mom || c->pts.empty() || n_in < 1) return 0;
  return surrogate_layout(c, n_in).total;
}

int rw_surrogate_reweight(rw_ctx* c, rw_mlp* m, double p_scale, double k_scale, double s_max, double* d_wnew,
                          unsigned char* d_fallback, double* h_sigma, int64_t* h_n_fallback, void* d_ws,
                          size_t ws_bytes) {
  int rc = ready(c, true);
  if (rc) return rc;
  if (!moves_possible(c)) return fail(c, RW_ERR_MODE, "the surrogate covers the top-mass axis of the QCD processes");
  if (!m || !d_wnew || !d_ws) return fail(c, RW_ERR_NULL, "model, W' and workspace are required");
  if (c->pts.empty()) return fail(c, RW_ERR_STATE, "no points set");
  DeviceGuard g(c->device);
  int nin = 0, hidden = 0, layers = 0;
  void* mstream = nullptr;
  if (rw_mlp_info(m, &nin, &hidden, &layers, &mstream) != RW_OK) return fail(c, RW_ERR_ARG, "bad model");
  if (mstream != static_cast<void*>(c->stream))
    return fail(c, RW_ERR_ARG, "the model must be created on the context's stream");
  const SurrogateLayout L = surrogate_layout(c, nin);
  if (ws_bytes < L.total) return fail(c, RW_ERR_WORKSPACE, "workspace %zu < %zu", ws_bytes, L.total);
  char* b = static_cast<char*>(d_ws);
  float* x = reinterpret_cast<float*>(b + L.x);
  float* out = reinterpret_cast<float*>(b + L.out);
  unsigned* mask = reinterpret_cast<unsigned*>(b + L.mask);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(b + L.counts);
  long long* rank = reinterpret_cast<long long*>(b + L.rank);
  long long* list = reinterpret_cast<long long*>(b + L.list);
  double* mom_g = reinterpret_cast<double*>(b + L.mom_g);
  double* w_g = reinterpret_cast<double*>(b + L.w_g);
  double* wn_g = reinterpret_cast<double*>(b + L.wn_g);
  double2* part = reinterpret_cast<double2*>(b + L.part);
  double* sig = reinterpret_cast<double*>(b + L.sig);
  const int P = (int)c->pts.size(), N = registry().st[c->process].n_external;
  const long long E = c->E, tot = (long long)P * E;
  // 1. features, 2. MLP
  if ((rc = rw_surrogate_features(c, nin, p_scale, k_scale, nullptr, x, nullptr))) return rc;
  cudaError_t e = cudaMemsetAsync(cnt, 0, 8 * (size_t)N_GROUPS, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(mask, 0, 4 * (size_t)E, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  if ((rc = rw_mlp_forward(m, x, tot, out))) return fail(c, rc, "mlp forward: %s", rw_mlp_last_error(m));
  // 3. decision per (event, point), then the events grouped by the points they need exactly
  const unsigned eb = (unsigned)((E + 255) / 256);
  k_decide<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(out, c->w, E, P, kappas(c), (float)s_max, d_wnew,
                                                                 mask);
  k_count_groups<<<eb, 256, 0, c->stream>>>(mask, E, P, cnt, rank);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "decide launch");
  if ((e = cudaMemcpyAsync(c->h_stage, cnt, 8 * (size_t)N_GROUPS, cudaMemcpyDeviceToHost, c->stream)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "fallback counts");
  unsigned long long gn[N_GROUPS];
  memcpy(gn, c->h_stage, sizeof gn);
  GroupOffsets go{};
  long long o = 0;
  for (int g = 1; g < N_GROUPS; ++g) {
    go.off[g] = o;
    o += (long long)gn[g];
  }
  k_place_groups<<<eb, 256, 0, c->stream>>>(mask, rank, E, P, go, d_fallback, list);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "group launch");
  if (h_n_fallback)
    for (int p = 0; p < P; ++p) h_n_fallback[p] = 0;
  // 4. per group, the exact fused kernel on its events at its points (one
  // launch; those W' are the exact path's, bit for bit)
  for (int g = 1; g < N_GROUPS; ++g) {
    const long long n = (long long)gn[g];
    if (n == 0) continue;
    const long long* lg = list + go.off[g];
    RwArgs a{};
    RowMap rows{};
    int np = 0;
    a.pt[0] = make_point(c, c->p0, false);
    for (int p = 0; p < P; ++p)
      if (P > MASK_POINTS || ((g >> p) & 1)) {
        a.pt[1 + np] = make_point(c, c->pts[p], moves_event(c, c->pts[p]));
        rows.row[np++] = p;
        if (h_n_fallback) h_n_fallback[p] += n;
      }
    k_gather_events<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->mom, c->ld, c->w, N, lg, n, mom_g, w_g);
    a.mom = mom_g;
    a.w = w_g;
    a.E = n;
    a.ld = n;
    a.wnew = wn_g;
    a.P = np;
    char* core = b + L.core;
    fill_core(core, a, np);
    a.sigma_pair = nullptr;
    if ((e = cudaMemsetAsync(core, 0, 256, c->stream)) != cudaSuccess) return cuda_fail(c, e, "memset");
    if ((rc = launch(c, a))) return rc;
    k_scatter<<<(unsigned)((np * n + 255) / 256), 256, 0, c->stream>>>(wn_g, lg, n, np, rows, E, d_wnew);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "scatter launch");
  }
  // 5. sigma'_p (and sigma of W in the last slot)
  if ((e = row_sums(c->stream, d_wnew, E, P, c->w, part, sig)) != cudaSuccess) return cuda_fail(c, e, "sum launch");
  if ((e = cudaMemcpyAsync(c->h_stage, sig, 8 * (size_t)P, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "sigma copy");
  if (h_sigma) memcpy(h_sigma, c->h_stage, 8 * (size_t)P);
  return RW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// CUDA-graph batching
// ---------------------------------------------------------------------------
struct rw_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

int rw_graph_begin(void* stream) {
  const cudaError_t e = cudaStreamBeginCapture(static_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return RW_ERR_CUDA;
  }
  return RW_OK;
}

int rw_graph_end(void* stream, rw_graph** out) {
  if (!out) return RW_ERR_NULL;
  *out = nullptr;
  rw_graph* g = new rw_graph();
  cudaError_t e = cudaStreamEndCapture(static_cast<cudaStream_t>(stream), &g->graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return RW_ERR_CUDA;
  }
  *out = g;
  return RW_OK;
}

int rw_graph_launch(rw_graph* g, void* stream) {
  if (!g) return RW_ERR_NULL;
  const cudaError_t e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return RW_ERR_CUDA;
  }
  return RW_OK;
}

int rw_graph_destroy(rw_graph* g) {
  if (!g) return RW_ERR_NULL;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return RW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// rw_split_double: the FP32 modes' FP64 -> double-float input split, run on
// an array (verification of df_from_double against the IEEE conversion).
namespace {
__global__ void k_split_double(const double* __restrict__ x, long long n, float* __restrict__ hi,
                               float* __restrict__ lo) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const rw::df v = rw::df_from_double(x[i]);
    hi[i] = v.hi;
    lo[i] = v.lo;
  }
}
}  // namespace

extern "C" int rw_split_double(const double* d_x, int64_t n, float* d_hi, float* d_lo, void* stream) {
  if (n < 0) return RW_ERR_ARG;
  if (n > 0 && (!d_x || !d_hi || !d_lo)) return RW_ERR_NULL;
  if (n == 0) return RW_OK;
  const long long blocks = std::min<long long>((n + 255) / 256, 4096);
  k_split_double<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(d_x, n, d_hi, d_lo);
  return cudaGetLastError() == cudaSuccess ? RW_OK : RW_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// rw_reweight_interp: Chebyshev interpolation of log r along one parameter
// axis (k_interp in kernels.cuh), exact fallback for the listed events.
// ---------------------------------------------------------------------------
namespace {

struct InterpLayout {
  size_t core, counts, list, mom_g, w_g, wn_g, part, sig, total;
};

InterpLayout interp_layout(const rw_ctx* c) {
  InterpLayout L{};
  const size_t P = std::max<size_t>(1, c->pts.size()), E = (size_t)c->E, N = registry().st[c->process].n_external;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o += align256(bytes);
    return at;
  };
  L.core = take(ws_core_bytes((int)P));
  L.counts = take(16);
  L.list = take(8 * E);
  L.mom_g = take(8 * 4 * N * E);
  L.w_g = take(8 * E);
  L.wn_g = take(8 * P * E);
  L.part = take(16 * SUM_BLOCKS * (P + 1));
  L.sig = take(8 * (P + 1));
  L.total = o;
  return L;
}

// the one parameter field in which every point differs from the original
// parameters (the others equal), or -1
int interp_axis(const rw_ctx* c) {
  auto field = [](const rw_params& p, int f) {
    const double v[8] = {p.alpha_s, p.m_t, p.w_t, p.yt_scale, p.alpha_em_inv, p.G_F, p.m_Z, p.w_Z};
    return v[f];
  };
  int axis = -1;
  for (const rw_params& q : c->pts)
    for (int f = 0; f < 8; ++f) {
      if (field(q, f) == field(c->p0, f)) continue;
      if (axis >= 0 && axis != f) return -1;
      axis = f;
    }
  return axis;
}

rw_params with_axis(rw_params p, int axis, double v) {
  double* f[8] = {&p.alpha_s, &p.m_t, &p.w_t, &p.yt_scale, &p.alpha_em_inv, &p.G_F, &p.m_Z, &p.w_Z};
  *f[axis] = v;
  return p;
}

__global__ void k_scatter_rows(const double* __restrict__ v, const long long* __restrict__ list, long long n, int P,
                               long long E, double* __restrict__ dst) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)P * n) return;
  const long long j = t / n, i = t % n;
  dst[j * E + list[i]] = v[j * n + i];
}

}  // namespace

extern "C" {

size_t rw_interp_workspace_bytes(const rw_ctx* c) {
  if (!c || c->process < 0 || !c->mom || c->pts.empty()) return 0;
  return interp_layout(c).total;
}

int rw_reweight_interp(rw_ctx* c, int n_nodes, double tol, double* d_wnew, unsigned char* d_fallback,
                       double* h_sigma, double* h_sigma_orig, int64_t* h_n_fallback, int64_t* h_n_bad, void* d_ws,
                       size_t ws_bytes) {
  int rc = ready(c, true);
  if (rc) return rc;
  if (c->pts.empty()) return fail(c, RW_ERR_STATE, "no points set");
  if (!d_wnew || !d_ws) return fail(c, RW_ERR_NULL, "W' and workspace are required");
  if (n_nodes < 3 || n_nodes > rw::MAX_NODES) return fail(c, RW_ERR_ARG, "n_nodes must be in [3, %d]", rw::MAX_NODES);
  if (!(tol > 0)) return fail(c, RW_ERR_ARG, "tol must be > 0");
  const InterpLayout L = interp_layout(c);
  if (ws_bytes < L.total) return fail(c, RW_ERR_WORKSPACE, "workspace %zu < %zu", ws_bytes, L.total);
  const int axis = interp_axis(c);
  if (axis < 0) return fail(c, RW_ERR_ARG, "the points must differ from the original parameters in one field only");
  const int lb = c->lane_bits >= 0 ? c->lane_bits : default_lane_bits(c->process, c->mode);
  const KernelEntry* k = registry().find(c->process, c->mode, lb, 1);
  if (!k) return fail(c, RW_ERR_MODE, "no interpolation kernel for process %d mode %d lane_bits %d", c->process,
                      c->mode, lb);
  DeviceGuard g(c->device);
  const int P = (int)c->pts.size(), N = registry().st[c->process].n_external, K = n_nodes;
  const long long E = c->E;
  auto field = [axis](const rw_params& p) {
    const double v[8] = {p.alpha_s, p.m_t, p.w_t, p.yt_scale, p.alpha_em_inv, p.G_F, p.m_Z, p.w_Z};
    return v[axis];
  };
  double lo = field(c->pts[0]), hi = lo;
  for (const rw_params& q : c->pts) {
    lo = std::min(lo, field(q));
    hi = std::max(hi, field(q));
  }
  if (!(hi > lo)) {  // one distinct value: a tiny interval around it
    lo -= 1e-6 * fabs(lo) + 1e-12;
    hi += 1e-6 * fabs(hi) + 1e-12;
  }
  rw::InterpArgs ia{};
  ia.mom = c->mom;
  ia.w = c->w;
  ia.E = E;
  ia.ld = c->ld;
  ia.wnew = d_wnew;
  ia.flag = d_fallback;
  char* b = static_cast<char*>(d_ws);
  ia.counts = reinterpret_cast<unsigned long long*>(b + L.counts);
  ia.list = reinterpret_cast<long long*>(b + L.list);
  ia.P = P;
  ia.K = K;
  ia.tol = tol;
  ia.pt0 = make_point(c, c->p0, false);
  for (int kk = 0; kk < K; ++kk) {
    const double xk = cos(M_PI * (kk + 0.5) / K);
    const rw_params q = with_axis(c->p0, axis, 0.5 * (lo + hi) + 0.5 * (hi - lo) * xk);
    ia.node[kk] = make_point(c, q, moves_event(c, q));
    for (int i = 0; i < K; ++i) ia.cheb[i][kk] = (i == 0 ? 1.0 : 2.0) / K * cos(i * M_PI * (kk + 0.5) / K);
  }
  for (int j = 0; j < P; ++j) ia.x[j] = (2.0 * field(c->pts[j]) - (lo + hi)) / (hi - lo);
  cudaError_t e = cudaMemsetAsync(ia.counts, 0, 16, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  {
    Shape sh;
    if ((rc = shape(c, 0, sh))) return rc;
    const size_t ismem = (size_t)k->smem_per_thread * sh.block;
    if ((e = ensure_smem(k->func, ismem)) != cudaSuccess)
      return cuda_fail(c, e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
    int per_sm = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k->func, sh.block, ismem)) != cudaSuccess)
      return cuda_fail(c, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    const long long need = (E * (1 << lb) + sh.block - 1) / sh.block;
    const int grid = (int)std::max(1LL, std::min<long long>({(long long)GRID_CAP,
                                                              (long long)std::max(1, per_sm) * c->sm_count, need}));
    void* args[] = {&ia};
    if ((e = cudaLaunchKernel(k->func, dim3(grid), dim3(sh.block), args, ismem, c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "interpolation kernel launch");
  }
  if ((e = cudaMemcpyAsync(c->h_stage, ia.counts, 16, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "fallback count");
  unsigned long long cnt[2];
  memcpy(cnt, c->h_stage, 16);
  const long long n = (long long)cnt[0];
  if (h_n_fallback) *h_n_fallback = n;
  if (h_n_bad) *h_n_bad = (int64_t)cnt[1];
  double* mom_g = reinterpret_cast<double*>(b + L.mom_g);
  double* w_g = reinterpret_cast<double*>(b + L.w_g);
  double* wn_g = reinterpret_cast<double*>(b + L.wn_g);
  if (n > 0) {  // the exact path for the listed events, all points in one launch
    k_gather_events<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->mom, c->ld, c->w, N, ia.list, n, mom_g,
                                                                         w_g);
    RwArgs a{};
    reweight_args(c, a, wn_g, nullptr, nullptr, nullptr);
    a.mom = mom_g;
    a.w = w_g;
    a.E = n;
    a.ld = n;
    char* core = b + L.core;
    a.ticket = reinterpret_cast<unsigned int*>(core);
    a.nbad_count = reinterpret_cast<unsigned long long*>(core + 8);
    a.sigma = reinterpret_cast<double*>(core + 64);
    a.nbad_out = reinterpret_cast<unsigned long long*>(core + 64 + 8 * (size_t)(P + 1));
    a.block_part = reinterpret_cast<double2*>(core + 256 + align256(8 * (size_t)(P + 2)));
    if ((e = cudaMemsetAsync(core, 0, 256, c->stream)) != cudaSuccess) return cuda_fail(c, e, "memset");
    if ((rc = launch(c, a))) return rc;
    k_scatter_rows<<<(unsigned)((P * n + 255) / 256), 256, 0, c->stream>>>(wn_g, ia.list, n, P, E, d_wnew);
  }
  // cross sections: deterministic compensated sums of the final W' rows and of W
  double2* part = reinterpret_cast<double2*>(b + L.part);
  double* sig = reinterpret_cast<double*>(b + L.sig);
  if ((e = row_sums(c->stream, d_wnew, E, P, c->w, part, sig)) != cudaSuccess) return cuda_fail(c, e, "sums");
  std::vector<double> hs(P + 1);
  if ((e = cudaMemcpyAsync(hs.data(), sig, 8 * (size_t)(P + 1), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "sums");
  if (h_sigma) memcpy(h_sigma, hs.data(), 8 * (size_t)P);
  if (h_sigma_orig) *h_sigma_orig = hs[P];
  return cnt[1] ? RW_WARN_BAD_EVENTS : RW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Several processes in one persistent launch (multi.cuh)
// ---------------------------------------------------------------------------
#include "multi.cuh"

namespace {

struct MultiRegistry {
  std::vector<rw::MultiEntry> kernels;
  MultiRegistry() { rw::register_multi(kernels); }
};

const MultiRegistry& multi_registry() {
  static MultiRegistry r;
  return r;
}

}  // namespace

struct rw_multi {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  struct Item {
    rw_ctx* ctx;
    double *wnew, *ratio;
  };
  std::vector<Item> items;
  std::string err;
  std::map<std::pair<const void*, size_t>, int> occ;
};

namespace {

int mfail(rw_multi* m, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int mfail(rw_multi* m, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (m) m->err = buf;
  return code;
}

constexpr size_t MULTI_WS_BYTES = 256;  // the launch's ticket

}  // namespace

extern "C" {

int rw_multi_create(rw_multi** out, int device, void* stream) {
  if (!out) return RW_ERR_NULL;
  *out = nullptr;
  rw_multi* m = new rw_multi();
  m->device = device;
  m->stream = static_cast<cudaStream_t>(stream);
  if (cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return RW_ERR_CUDA;
  }
  *out = m;
  return RW_OK;
}

int rw_multi_destroy(rw_multi* m) {
  if (!m) return RW_ERR_NULL;
  delete m;
  return RW_OK;
}

const char* rw_multi_last_error(const rw_multi* m) { return m ? m->err.c_str() : "null handle"; }

int rw_multi_add(rw_multi* m, rw_ctx* c, double* d_wnew, double* d_ratio) {
  if (!m || !c) return RW_ERR_NULL;
  if ((int)m->items.size() >= rw::MAX_MULTI) return mfail(m, RW_ERR_ARG, "at most %d processes", rw::MAX_MULTI);
  int rc = ready(c, true);
  if (rc) return mfail(m, rc, "context not ready: %s", c->err.c_str());
  if (c->pts.empty()) return mfail(m, RW_ERR_STATE, "context has no reweight points");
  if (c->device != m->device) return mfail(m, RW_ERR_ARG, "context on device %d, launch on %d", c->device, m->device);
  for (const auto& it : m->items) {
    if (it.ctx == c) return mfail(m, RW_ERR_ARG, "context added twice");
    if (it.ctx->process == c->process) return mfail(m, RW_ERR_ARG, "process %d added twice", c->process);
    if (it.ctx->mode != c->mode) return mfail(m, RW_ERR_MODE, "every process must use the same precision mode");
  }
  DeviceGuard g(c->device);
  if (d_wnew && (rc = check_dev_ptr(c, d_wnew, "wnew"))) return mfail(m, rc, "%s", c->err.c_str());
  if (d_ratio && (rc = check_dev_ptr(c, d_ratio, "ratio"))) return mfail(m, rc, "%s", c->err.c_str());
  m->items.push_back({c, d_wnew, d_ratio});
  return RW_OK;
}

size_t rw_multi_workspace_bytes(const rw_multi* m) { return m ? MULTI_WS_BYTES : 0; }

int rw_multi_reweight_async(rw_multi* m, void* d_ws, size_t ws_bytes) {
  if (!m) return RW_ERR_NULL;
  const int n = (int)m->items.size();
  if (n < 1) return mfail(m, RW_ERR_STATE, "no processes added");
  if (!d_ws) return mfail(m, RW_ERR_NULL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(d_ws) % 16) return mfail(m, RW_ERR_ALIGN, "workspace not 16-byte aligned");
  if (ws_bytes < MULTI_WS_BYTES) return mfail(m, RW_ERR_WORKSPACE, "workspace smaller than rw_multi_workspace_bytes");
  // the compiled variant whose process list holds exactly these processes
  const rw::MultiEntry* k = nullptr;
  int slot[rw::MAX_MULTI] = {};
  for (const auto& e : multi_registry().kernels) {
    if (e.mode != m->items[0].ctx->mode || e.n != n) continue;
    bool all = true;
    for (int i = 0; i < n && all; ++i) {
      slot[i] = -1;
      for (int j = 0; j < n; ++j)
        if (m->items[j].ctx->process == e.process[i]) slot[i] = j;
      all = slot[i] >= 0;
    }
    if (all) {
      k = &e;
      break;
    }
  }
  if (!k) return mfail(m, RW_ERR_MODE, "no multi-process kernel for these %d processes in this mode", n);
  DeviceGuard g(m->device);
  const int block = 128;
  size_t sums = 0;
  rw::MultiArgs a{};
  long long tiles = 0;
  int pool = 0;
  for (int i = 0; i < n; ++i) {
    rw_ctx* c = m->items[slot[i]].ctx;
    const int P = (int)c->pts.size();
    if (ws_core_bytes(P) > c->ws_bytes)
      return mfail(m, RW_ERR_WORKSPACE, "workspace of process %d too small", c->process);
    if (pool + P + 1 > rw::MULTI_POOL)
      return mfail(m, RW_ERR_ARG, "more than %d parameter points (plus one original each) in one launch",
                   rw::MULTI_POOL);
    RwArgs r{};
    reweight_args(c, r, m->items[slot[i]].wnew, m->items[slot[i]].ratio, nullptr, nullptr);
    rw::MultiItem& it = a.item[i];
    it.mom = r.mom;
    it.w = r.w;
    it.E = r.E;
    it.ld = r.ld;
    it.ldo = 0;
    it.me0 = nullptr;
    it.me_pts = nullptr;
    it.ratio = r.ratio;
    it.wnew = r.wnew;
    it.block_part = r.block_part;
    it.sigma = r.sigma;
    it.sigma_pair = r.sigma_pair;
    it.nbad_count = r.nbad_count;
    it.nbad_out = r.nbad_out;
    it.P = P;
    it.pt0 = pool;
    for (int j = 0; j <= P; ++j) a.pool[pool + j] = r.pt[j];
    pool += P + 1;
    const long long gpb = block >> k->lane_bits[i];
    tiles += (c->E + gpb - 1) / gpb;
    a.tile_end[i] = tiles;
    a.sacc_off[i] = (int)sums;
    sums += (size_t)(block / 32) * (P + 1);
  }
  a.n = n;
  a.ticket = static_cast<unsigned int*>(d_ws);
  const size_t smem = (size_t)k->smem_per_thread * block + sums * sizeof(double2);
  const auto key = std::make_pair(k->func, smem);
  int per_sm = 0;
  const auto it = m->occ.find(key);
  if (it == m->occ.end()) {
    cudaError_t e = ensure_smem(k->func, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k->func, block, smem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return mfail(m, RW_ERR_CUDA, "occupancy: %s", cudaGetErrorString(e));
    }
    per_sm = std::max(per_sm, 1);
    m->occ[key] = per_sm;
  } else {
    per_sm = it->second;
  }
  const int grid =
      (int)std::max(1LL, std::min<long long>({(long long)GRID_CAP, (long long)per_sm * m->sm_count, tiles}));
  // the ticket must start at zero (each launch leaves it at zero again)
  cudaError_t e = cudaMemsetAsync(d_ws, 0, sizeof(unsigned int), m->stream);
  if (e != cudaSuccess) return mfail(m, RW_ERR_CUDA, "workspace memset: %s", cudaGetErrorString(e));
  void* args[] = {&a};
  e = cudaLaunchKernel(k->func, dim3(grid), dim3(block), args, smem, m->stream);
  if (e != cudaSuccess) return mfail(m, RW_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return RW_OK;
}

int rw_multi_get_results(rw_multi* m, double* h_sigma, double* h_sigma_orig, int64_t* h_n_bad) {
  if (!m) return RW_ERR_NULL;
  const int n = (int)m->items.size();
  if (n < 1) return mfail(m, RW_ERR_STATE, "no processes added");
  const int P = (int)m->items[0].ctx->pts.size();
  for (const auto& it : m->items)
    if ((int)it.ctx->pts.size() != P) return mfail(m, RW_ERR_STATE, "processes have different numbers of points");
  std::vector<double> s(P + 1, 0.0), c(P + 1, 0.0), ps(P + 1), pc(P + 1);
  int64_t bad = 0;
  for (const auto& it : m->items) {
    int64_t nb = 0;
    const int rc = rw_get_result_pairs(it.ctx, ps.data(), pc.data(), &nb);
    if (rc < 0) return mfail(m, rc, "process %d: %s", it.ctx->process, it.ctx->err.c_str());
    bad += nb;
    for (int j = 0; j <= P; ++j) {  // TwoSum merge of every process's pairs, in the order they were added
      const double t = s[j] + ps[j], bp = t - s[j];
      c[j] += pc[j] + ((s[j] - (t - bp)) + (ps[j] - bp));
      s[j] = t;
    }
  }
  if (h_sigma)
    for (int j = 0; j < P; ++j) h_sigma[j] = s[j] + c[j];
  if (h_sigma_orig) *h_sigma_orig = s[P] + c[P];
  if (h_n_bad) *h_n_bad = bad;
  return bad ? RW_WARN_BAD_EVENTS : RW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Event file to event file with the host work overlapped (rw_lhe_reweight)
// ---------------------------------------------------------------------------
#include <thread>

namespace {

// device slots: two chunks of momenta [N][4][chunk], weights and W' [P][chunk]
struct LheLayout {
  size_t core, mom, w, wnew, total;
};

LheLayout lhe_layout(const rw_ctx* c, int64_t chunk) {
  const int N = registry().st[c->process].n_external;
  const size_t P = std::max<size_t>(1, c->pts.size());
  LheLayout L{};
  L.core = ws_core_bytes((int)P) + align256(16 * (P + 1));  // + the carried (sum, compensation) pairs
  L.mom = align256(8 * 4 * (size_t)N * chunk);
  L.w = align256(8 * (size_t)chunk);
  L.wnew = align256(8 * P * chunk);
  L.total = L.core + 2 * (L.mom + L.w + L.wnew);
  return L;
}

struct PinnedSlot {
  double *mom = nullptr, *w = nullptr, *wnew = nullptr;
};

}  // namespace

extern "C" {

size_t rw_lhe_workspace_bytes(const rw_ctx* c, int64_t chunk) {
  if (!c || c->process < 0 || chunk <= 0) return 0;
  return lhe_layout(c, chunk).total;
}

int rw_lhe_reweight(rw_ctx* c, rw_lhe* lhe, const char* out_path, const char* const* ids, int64_t chunk,
                    int n_threads, void* d_ws, size_t ws_bytes, double* h_sigma, double* h_sigma_orig,
                    int64_t* h_n_bad) {
  if (!c) return RW_ERR_NULL;
  if (!lhe || !out_path || !ids || !d_ws) return fail(c, RW_ERR_NULL, "event file, path, ids and workspace are required");
  if (c->process < 0 || !c->have_p0 || c->pts.empty()) return fail(c, RW_ERR_STATE, "process/params/points unset");
  const int64_t E = rw_lhe_n_events(lhe);
  if (E <= 0) return fail(c, RW_ERR_ARG, "the event file has no events");
  if (chunk <= 0) return fail(c, RW_ERR_ARG, "chunk must be > 0");
  chunk = std::min<int64_t>(chunk, E);
  if (reinterpret_cast<uintptr_t>(d_ws) % 256) return fail(c, RW_ERR_ALIGN, "workspace not 256-byte aligned");
  const LheLayout L = lhe_layout(c, chunk);
  if (ws_bytes < L.total) return fail(c, RW_ERR_WORKSPACE, "workspace smaller than rw_lhe_workspace_bytes");
  DeviceGuard g(c->device);
  const int N = registry().st[c->process].n_external;
  const int P = (int)c->pts.size();
  char* base = static_cast<char*>(d_ws);
  double2* d_sacc = reinterpret_cast<double2*>(base + ws_core_bytes(P));
  double *d_mom[2], *d_w[2], *d_wnew[2];
  for (int s = 0; s < 2; ++s) {
    char* q = base + L.core + s * (L.mom + L.w + L.wnew);
    d_mom[s] = reinterpret_cast<double*>(q);
    d_w[s] = reinterpret_cast<double*>(q + L.mom);
    d_wnew[s] = reinterpret_cast<double*>(q + L.mom + L.w);
  }
  int rc = load_events(c, d_mom[0], d_w[0], chunk, d_ws, ws_bytes, true);
  if (rc) return rc;
  // three pinned host slots: chunk k+1 is parsed into one while chunk k's
  // copies use the second and chunk k-1's weights are written from the third
  PinnedSlot hs[3];
  std::vector<cudaEvent_t> done(3, nullptr);
  auto cleanup = [&]() {
    for (auto& x : hs)
      for (double* q : {x.mom, x.w, x.wnew})
        if (q) cudaFreeHost(q);
    for (auto& ev : done)
      if (ev) cudaEventDestroy(ev);
  };
  for (int s = 0; s < 3; ++s) {
    if (cudaHostAlloc(reinterpret_cast<void**>(&hs[s].mom), 8 * 4 * (size_t)N * chunk, cudaHostAllocDefault) !=
            cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&hs[s].w), 8 * (size_t)chunk, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&hs[s].wnew), 8 * (size_t)P * chunk, cudaHostAllocDefault) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&done[s], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      cleanup();
      return fail(c, RW_ERR_CUDA, "pinned host buffers for the event-file pipeline");
    }
  }
  const int K = (int)((E + chunk - 1) / chunk);
  auto first_of = [&](int k) { return (int64_t)k * chunk; };
  auto size_of = [&](int k) { return std::min<int64_t>(chunk, E - first_of(k)); };
  int parse_rc = RW_OK;
  auto parse = [&](int k) {
    parse_rc = rw_lhe_read(lhe, c->process, first_of(k), size_of(k), hs[k % 3].mom, chunk, hs[k % 3].w, n_threads);
  };
  rc = rw_lhe_write_begin(lhe, out_path, P, ids);
  if (rc) {
    cleanup();
    return fail(c, rc, "%s", rw_lhe_last_error(lhe));
  }
  auto abort_all = [&](int code, const std::string& msg) {
    cudaStreamSynchronize(c->stream);
    rw_lhe_write_end(lhe);  // closes the partial output
    cleanup();
    return fail(c, code, "%s", msg.c_str());
  };
  parse(0);
  if (parse_rc) return abort_all(parse_rc, rw_lhe_last_error(lhe));
  const size_t row = 8 * (size_t)chunk;
  for (int k = 0; k < K; ++k) {
    const int s = k & 1, h = k % 3;
    const int64_t n = size_of(k);
    // chunk k on the GPU: copies in, the fused reweight (sums carried across
    // chunks in (sum, compensation) form), W' copied back
    cudaError_t e = cudaMemcpy2DAsync(d_mom[s], row, hs[h].mom, row, 8 * (size_t)n, 4 * (size_t)N,
                                      cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_w[s], hs[h].w, 8 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return abort_all(RW_ERR_CUDA, cudaGetErrorString(e));
    RwArgs a{};
    reweight_args(c, a, d_wnew[s], nullptr, nullptr, nullptr);
    a.mom = d_mom[s];
    a.w = d_w[s];
    a.E = n;
    a.ld = chunk;
    a.ldo = chunk;
    a.sigma_acc = d_sacc;
    a.accumulate = k > 0;
    if ((rc = launch(c, a))) return abort_all(rc, c->err);
    e = cudaMemcpy2DAsync(hs[h].wnew, row, d_wnew[s], row, 8 * (size_t)n, (size_t)P, cudaMemcpyDeviceToHost,
                          c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(done[h], c->stream);
    if (e != cudaSuccess) return abort_all(RW_ERR_CUDA, cudaGetErrorString(e));
    // meanwhile on the host: parse chunk k+1, write chunk k-1
    std::thread parser;
    if (k + 1 < K) parser = std::thread(parse, k + 1);
    int wrc = RW_OK;
    if (k > 0) {
      const int hp = (k - 1) % 3;
      if ((e = cudaEventSynchronize(done[hp])) != cudaSuccess) wrc = RW_ERR_CUDA;
      if (!wrc) wrc = rw_lhe_write_events(lhe, first_of(k - 1), size_of(k - 1), hs[hp].wnew, chunk);
    }
    if (parser.joinable()) parser.join();
    if (wrc) return abort_all(wrc, wrc == RW_ERR_CUDA ? "event synchronisation" : rw_lhe_last_error(lhe));
    if (parse_rc) return abort_all(parse_rc, rw_lhe_last_error(lhe));
  }
  cudaError_t e = cudaEventSynchronize(done[(K - 1) % 3]);
  if (e != cudaSuccess) return abort_all(RW_ERR_CUDA, cudaGetErrorString(e));
  rc = rw_lhe_write_events(lhe, first_of(K - 1), size_of(K - 1), hs[(K - 1) % 3].wnew, chunk);
  if (rc) return abort_all(rc, rw_lhe_last_error(lhe));
  rc = rw_lhe_write_end(lhe);
  cleanup();
  if (rc) return fail(c, rc, "%s", rw_lhe_last_error(lhe));
  return rw_get_results(c, h_sigma, h_sigma_orig, h_n_bad);
}

}  // extern "C"
