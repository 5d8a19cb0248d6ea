// Measured plain-ALU peaks (FP64 DFMA, FP32 FFMA) of the GPU this library
// runs on: the denominators of the amplitude kernels' rooflines, which are
// bound by the FP64 pipe (FP64 mode) or the FP32 FMA pipe (FP32 modes), not
// by memory.  The paper has no counterpart.
//
// Every thread runs NCH independent FMA chains x <- x * b + c for `iters`
// trips; the grid fills every SM at full occupancy (256-thread blocks x the
// resident-block count), so the pipes, not latency, bound the time.  The
// chains' results are folded into one value that is written only when it
// equals a value it cannot take, so the compiler keeps every FMA and the
// kernel writes nothing.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/rwgt.h"

namespace {

constexpr int NCH = 8;

__device__ double g_peak_sink_d;
__device__ float g_peak_sink_f;

template <class T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) {
  return __fma_rn(a, b, c);
}
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}

template <class T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T b, T c) {
  T x[NCH];
#pragma unroll
  for (int i = 0; i < NCH; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
#pragma unroll 4
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < NCH; ++i) x[i] = fma_t<T>(x[i], b, c);
  T s = T(0);
#pragma unroll
  for (int i = 0; i < NCH; ++i) s += x[i];
  if (s == T(-1.25e-30)) {  // never true for these inputs
    if constexpr (sizeof(T) == 8)
      g_peak_sink_d = s;
    else
      g_peak_sink_f = s;
  }
}

template <class T>
int run_peak(int device, cudaStream_t st, double* tflops, double* ms_out) {
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return RW_ERR_CUDA;
  const void* f = (const void*)&k_fma_peak<T>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 256, 0) != cudaSuccess) return RW_ERR_CUDA;
  per_sm = std::max(per_sm, 1);
  const int grid = sms * per_sm;
  // about 20-40 ms per launch at the nominal rates (FP64 is ~64x slower)
  const int iters = sizeof(T) == 8 ? 4096 : 131072;
  const T b = T(0.999999), c = T(1e-6);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return RW_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RW_ERR_CUDA;
  }
  int rc = RW_OK;
  float best = 0.0f;
  for (int rep = 0; rep < 4 && rc == RW_OK; ++rep) {  // one warm-up, best of three
    cudaEventRecord(e0, st);
    k_fma_peak<T><<<grid, 256, 0, st>>>(iters, b, c);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = RW_ERR_CUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const double flops = 2.0 * NCH * (double)iters * grid * 256.0;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return RW_OK;
}

}  // namespace

extern "C" int rw_alu_peak(int device, void* cuda_stream, int kind, double* h_tflops, double* h_ms) {
  if (!h_tflops) return RW_ERR_NULL;
  if (kind != 0 && kind != 1) return RW_ERR_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return RW_ERR_CUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return RW_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int rc = kind == 0 ? run_peak<double>(device, st, h_tflops, h_ms) : run_peak<float>(device, st, h_tflops, h_ms);
  if (prev != device) cudaSetDevice(prev);
  return rc;
}
