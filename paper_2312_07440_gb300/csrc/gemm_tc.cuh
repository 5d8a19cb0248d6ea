// Blackwell tensor-core GEMM for the surrogate MLP's hidden layers:
//   Z = A W + b,  H = bf16(SiLU(Z))   (A: BF16 activations [M][K], W: [K][N])
// optionally followed by a fused FP32 output head out = H W_out + b_out
// (N -> 2) for inference, so the last hidden layer never leaves the chip.
//
// One CTA per SM walks 128-row tiles of A (persistent).  Roles:
//   warp 0    one thread issues TMA loads (cp.async.bulk.tensor, 128-byte
//             swizzle): the whole transposed weight matrix W^T [N][K] once
//             (resident in shared memory), then the A tiles through a ring of
//             STAGES k-blocks of 64 columns;
//   warp 1    owns the tensor memory (two accumulators of N FP32 columns x
//             128 lanes); one thread issues tcgen05.mma (kind::f16, BF16 x
//             BF16 -> FP32, M = 128, N, K = 16) and commits each k-block's
//             MMAs to that A stage's "empty" barrier and each tile to its
//             accumulator's "full" barrier;
//   warps 2-17 the epilogue, four warps per lane quarter (warp w may read the
//             tensor-memory lanes 32 (w % 4) ... 32 (w % 4) + 31), each of the
//             four on a quarter of the N columns: tcgen05.ld 16 columns at a
//             time, bias, SiLU, BF16/FP32 stores or the fused head (the four
//             column quarters' partial sums meet in shared memory), then free
//             the accumulator, which the MMA thread reuses two tiles later.
// Every mbarrier wait gives up after ~2^31 clock cycles (~1 s): it sets the
// error flag, every role stops, the MMA thread drains its outstanding MMAs
// (bounded), the TMA thread waits (bounded) for its loads in flight, and the
// tensor memory is freed before the kernel returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_ptx.cuh"

namespace tcg {

constexpr int BM = 128;      // rows per tile = tensor-memory lanes
constexpr int BK = 64;       // k per TMA box and swizzle row (64 BF16 = 128 bytes)
constexpr int STAGES = 4;    // A ring depth (k-blocks)
constexpr int MAX_N = 256;   // N <= 256 (one MMA covers the whole width)
constexpr int MAX_KB = 4;    // K <= 256
constexpr int EPI_WARPS = 16;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int UMMA_K = 16;   // k of one kind::f16 MMA

// dynamic shared memory: 1024-byte alignment slack, W^T, the A ring, barriers,
// the fused head's partial sums [accumulator][column quarter][row][2]
constexpr size_t SMEM_B = (size_t)MAX_KB * MAX_N * 128;
constexpr size_t SMEM_A = (size_t)STAGES * BM * 128;
constexpr size_t SMEM_HEAD = (size_t)2 * 4 * BM * 2 * sizeof(float);
constexpr size_t SMEM_BYTES = 1024 + SMEM_B + SMEM_A + 256 + SMEM_HEAD;

struct Epi {
  const float* bias;       // [N] (forward)
  const float* Zin;        // backward data gradient: pre-activation [M][N]; H = bf16(acc SiLU'(Zin)), or null
  float* Z;                // [M][N] pre-activation (FP32), or null
  unsigned short* H;       // [M][N] SiLU(Z) as BF16, or null
  const float* w_out;      // fused output head [N][2] (FP32), or null
  const float* b_out;      // [2]
  float* out;              // [M][2]
  int* err;                // set to a nonzero code when a wait gives up
  int M, N, K;
};

// SiLU z sigma(z) = z / (1 + 2^(-z log2 e)) with the special-function unit's
// approximate base-2 exponential and reciprocal (each within a few units in
// the last place of FP32; the result is rounded to BF16).  Below z = -88 the
// exponential overflows to +inf and the result is -0.
__device__ __forceinline__ float silu_f(float z) {
  float e, r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(z * -1.4426950408889634f));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
  return z * r;
}

__device__ __forceinline__ unsigned short bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// SiLU'(z) = sigma(z) (1 + z (1 - sigma(z))), sigma from the same exp2 and reciprocal
__device__ __forceinline__ float dsilu_f(float z) {
  float e, s;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(z * -1.4426950408889634f));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(1.0f + e));
  return s * fmaf(z, 1.0f - s, 1.0f);
}

// two FP32 values rounded to BF16 in one word (lo in the low half)
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__global__ void __launch_bounds__(THREADS, 1) k_gemm_tc(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB, const Epi e) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sB = base;
  unsigned char* sA = base + SMEM_B;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + SMEM_A);
  // barrier slots: full_a[STAGES], empty_a[STAGES], full_b, acc_full[2], acc_empty[2], drain
  const uint32_t b_full_a = smem_u32(bars), b_empty_a = smem_u32(bars + STAGES), b_full_b = smem_u32(bars + 2 * STAGES);
  const uint32_t b_acc_full = smem_u32(bars + 2 * STAGES + 1), b_acc_empty = smem_u32(bars + 2 * STAGES + 3);
  const uint32_t b_drain = smem_u32(bars + 2 * STAGES + 5);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 6);
  float* head = reinterpret_cast<float*>(sA + SMEM_A + 256);  // [2][4][BM][2]
  __shared__ int abort_flag;
  __shared__ int head_count[8];  // [accumulator][lane quarter]: column quarters done

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = e.N, KB = e.K / BK;
  const int tiles = (e.M + BM - 1) / BM;
  const uint32_t tmem_cols = 2 * MAX_N;  // two accumulators of up to 256 columns

  if (threadIdx.x < 8) head_count[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(b_full_a + 8 * s, 1);
      mbar_init(b_empty_a + 8 * s, 1);
    }
    mbar_init(b_full_b, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(b_acc_full + 8 * i, 1);
      mbar_init(b_acc_empty + 8 * i, EPI_WARPS);  // one arrival per epilogue warp
    }
    mbar_init(b_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      // the transposed weights, once: KB boxes of 64 (k) x N (n)
      mbar_expect_tx(b_full_b, (uint32_t)(KB * N * 128));
      for (int kb = 0; kb < KB; ++kb) tma_load_2d(smem_u32(sB + (size_t)kb * N * 128), &tmB, kb * BK, 0, b_full_b);
      int stage = 0;
      uint32_t phase = 0;
      int issued[STAGES] = {};  // loads issued per stage (for the drain on abort)
      int uses[STAGES] = {};
      for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        for (int kb = 0; kb < KB; ++kb) {
          if (!mbar_wait(b_empty_a + 8 * stage, phase ^ 1, e.err, 1, abort)) goto tma_done;
          mbar_expect_tx(b_full_a + 8 * stage, BM * 128);
          tma_load_2d(smem_u32(sA + (size_t)stage * BM * 128), &tmA, kb * BK, t * BM, b_full_a + 8 * stage);
          ++issued[stage];
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
    tma_done:
      if (*abort) {
        // loads still in flight land in shared memory: wait for them (bounded)
        const long long t0 = clock64();
        for (int s = 0; s < STAGES; ++s) {
          uses[s] = issued[s];
          if (uses[s] == 0) continue;
          const uint32_t par = (uint32_t)((uses[s] - 1) & 1);
          while (!mbar_test(b_full_a + 8 * s, par) && clock64() - t0 < WAIT_CYCLES) {
          }
        }
        while (!mbar_test(b_full_b, 0) && clock64() - t0 < WAIT_CYCLES) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, N);
      bool ok = mbar_wait(b_full_b, 0, e.err, 2, abort);
      int stage = 0, acc = 0;
      uint32_t phase = 0, acc_phase = 0;
      for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
        if (!(ok = mbar_wait(b_acc_empty + 8 * acc, acc_phase ^ 1, e.err, 3, abort))) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * MAX_N);
        for (int kb = 0; kb < KB; ++kb) {
          if (!(ok = mbar_wait(b_full_a + 8 * stage, phase, e.err, 4, abort))) break;
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + (size_t)stage * BM * 128);
          const uint32_t b0 = smem_u32(sB + (size_t)kb * N * 128);
#pragma unroll
          for (int k = 0; k < BK / UMMA_K; ++k)
            umma_bf16(d, sw128_desc(a0 + 32 * k), sw128_desc(b0 + 32 * k), idesc, (kb | k) != 0);
          umma_commit(b_empty_a + 8 * stage);  // the stage is free once these MMAs have read it
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        umma_commit(b_acc_full + 8 * acc);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
      // every MMA issued so far has completed once this commit arrives
      umma_commit(b_drain);
      const long long t0 = clock64();
      while (!mbar_test(b_drain, 0) && clock64() - t0 < WAIT_CYCLES) {
      }
    }
  } else {
    const int q = warp & 3;             // the lane quarter this warp may read
    const int cq = (warp - 2) >> 2;     // its quarter of the columns
    const int cw = N >> 2;              // columns per quarter (a multiple of 16)
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      if (!mbar_wait(b_acc_full + 8 * acc, acc_phase, e.err, 5, abort)) break;
      tc_fence_after();
      const int r = q * 32 + lane;  // row within the tile
      const long long row = (long long)t * BM + r;
      const bool live = row < e.M;
      float h0 = 0.0f, h1 = 0.0f;
      for (int c0 = cq * cw; c0 < (cq + 1) * cw; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t)(acc * MAX_N + c0) + ((uint32_t)(q * 32) << 16), v);
        if (!live) continue;
        if (e.Zin) {
          // backward: the data gradient times SiLU' of the pre-activation, as BF16
          const float4* zp = reinterpret_cast<const float4*>(e.Zin + row * N + c0);
          uint4* hp = reinterpret_cast<uint4*>(e.H + row * N + c0);
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const float4 za = __ldg(zp + 2 * j), zb = __ldg(zp + 2 * j + 1);
            const float* x = v + 8 * j;
            hp[j] = make_uint4(bf16x2(x[0] * dsilu_f(za.x), x[1] * dsilu_f(za.y)),
                               bf16x2(x[2] * dsilu_f(za.z), x[3] * dsilu_f(za.w)),
                               bf16x2(x[4] * dsilu_f(zb.x), x[5] * dsilu_f(zb.y)),
                               bf16x2(x[6] * dsilu_f(zb.z), x[7] * dsilu_f(zb.w)));
          }
          continue;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += __ldg(e.bias + c0 + j);
        if (e.Z) {
          float4* zp = reinterpret_cast<float4*>(e.Z + row * N + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j) zp[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = silu_f(v[j]);
        if (e.H) {
          uint4* hp = reinterpret_cast<uint4*>(e.H + row * N + c0);
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] = bf16x2(v[8 * j + 2 * i], v[8 * j + 2 * i + 1]);
            hp[j] = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
        if (e.w_out) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            h0 = fmaf(v[j], __ldg(e.w_out + 2 * (c0 + j)), h0);
            h1 = fmaf(v[j], __ldg(e.w_out + 2 * (c0 + j) + 1), h1);
          }
        }
      }
      if (e.w_out) {
        // the four column quarters of these 32 rows meet in shared memory;
        // the last of the four warps to arrive adds them, in a fixed order
        // (no warp waits for another)
        float* hp = head + (size_t)((acc * 4 + cq) * BM + r) * 2;
        hp[0] = h0;
        hp[1] = h1;
        __syncwarp();
        int prior = 0;
        if (lane == 0) {
          __threadfence_block();
          prior = atomicAdd(&head_count[acc * 4 + q], 1);
        }
        prior = __shfl_sync(0xffffffffu, prior, 0);
        if (prior == 3) {
          __threadfence_block();
          if (live) {
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              s0 += head[((acc * 4 + c) * BM + r) * 2];
              s1 += head[((acc * 4 + c) * BM + r) * 2 + 1];
            }
            *reinterpret_cast<float2*>(e.out + 2 * row) = make_float2(s0 + e.b_out[0], s1 + e.b_out[1]);
          }
          __syncwarp();
          if (lane == 0) head_count[acc * 4 + q] = 0;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_acc_empty + 8 * acc);
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

}  // namespace tcg
