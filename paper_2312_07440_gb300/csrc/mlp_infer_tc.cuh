// The surrogate MLP's whole inference in one persistent kernel on the
// 5th-generation tensor cores: features x [M][n_in] (FP32) -> input layer ->
// hidden layers -> output layer out [M][2], with every activation kept in
// shared memory (nothing but x and out touches HBM).
//
//   layer 0  z = x W_0 + b_0 with x and W_0 split into BF16 pairs
//            (x = x_h + x_l, W = W_h + W_l, each part rounded to nearest):
//            one MMA over K = 3 n_in of [x_h | x_l | x_h] against
//            [W_h ; W_h ; W_l] gives x_h W_h + x_l W_h + x_h W_l, i.e. the
//            FP32 product up to the dropped x_l W_l (~2^-16 relative) and
//            FP32 accumulation;
//   layer l  z = h W_l + b_l (BF16 h and W_l, FP32 accumulation), for
//            l = 1 .. L-1, h = bf16(SiLU(z)) of the layer before;
//   output   out = SiLU(z_{L-1}) W_out + b_out in FP32 from the last
//            accumulator (the activation of the last layer is not rounded).
//
// One CTA per SM walks pairs of 128-row tiles.  The two tiles of a pair
// alternate on the tensor core layer by layer, so the epilogue of one tile
// (tensor memory -> bias, SiLU -> BF16 into its shared-memory activation
// buffer, the next layer's A operand) runs while the MMAs of the other tile
// run.  Roles:
//   warp 0     one thread streams the packed weights through a ring of
//              WSTAGES k-blocks ([256 n][64 k] BF16, 128-byte swizzle, TMA
//              from L2: every CTA reads the same 448 KB);
//   warp 1     owns 512 tensor-memory columns (one 128 x 256 FP32
//              accumulator per tile slot); one thread issues tcgen05.mma
//              (M = 128, N = 256, K = 16) and commits each weight k-block to
//              its ring slot and each layer to the slot's "full" barrier;
//   warps 2-17 the epilogue, four per lane quarter and one 64-column quarter
//              (one k-block of the next layer's A operand) each; they also
//              write the split features of each new tile into its slot, and
//              compute the output layer (the column quarters' partial sums
//              meet in the slot's free activation k-blocks; the last warp to
//              arrive adds them in a fixed order).
// Every wait is bounded (~2^31 cycles): on a timeout the error flag is set,
// every role stops, the MMA thread drains its MMAs, the TMA thread waits for
// its loads in flight, and the tensor memory is freed before the kernel
// returns.
#pragma once
#include "gemm_tc.cuh"

namespace tcg {
namespace inf {

constexpr int N = 256;                               // hidden width
constexpr int WSTAGES = 3;                           // weight ring depth
constexpr int MAX_LAYERS = 8;                        // input layer + hidden layers
constexpr int MAX_IN = 40;                           // 3 n_in <= 128: the split input fits two k-blocks
constexpr int KB_HIDDEN = N / BK;                    // k-blocks of a hidden layer
constexpr size_t KB_BYTES = (size_t)BM * 128;        // one k-block of a tile's activations (16 KB)
constexpr size_t ACT_BYTES = KB_HIDDEN * KB_BYTES;   // a tile's activations (64 KB)
constexpr size_t WBOX_BYTES = (size_t)N * 128;       // one weight k-block (32 KB)
constexpr size_t SMEM_BYTES = 1024 + 2 * ACT_BYTES + WSTAGES * WBOX_BYTES + 256;
static_assert(SMEM_BYTES <= 232448, "more shared memory than a block may have");

}  // namespace inf

struct InferArgs {
  const float* x;                       // [M][n_in] features (FP32)
  const float* bias[inf::MAX_LAYERS];   // [256] per layer (layer 0 the input layer)
  const float* w_out;                   // [256][2]
  const float* b_out;                   // [2]
  float* out;                           // [M][2]
  int* err;                             // set to a nonzero code when a wait gives up
  long long M;
  int n_in;                             // even, <= MAX_IN
  int kb0;                              // k-blocks of the split input layer: ceil(3 n_in / 64)
  int L;                                // layers before the output layer (input + hidden)
};

// byte offset of the BF16 pair at column c (even) of row r in a tile's
// activations: k-block c / 64, each row 128 bytes, its 16-byte chunks
// permuted by the 128-byte swizzle (chunk ^ row % 8) that TMA and the MMA
// descriptors use
__device__ __forceinline__ uint32_t act_off(int r, int c) {
  const int w = c & 63;
  return (uint32_t)((c >> 6) * inf::KB_BYTES + r * 128 + ((((w >> 3) ^ r) & 7) << 4) + ((w & 7) << 1));
}

// the split features of one row (this thread's share of the feature pairs)
struct FeatureShare {
  float v[2 * 5];  // up to 5 pairs: ceil(MAX_IN / 2 / 4)
};

__device__ __forceinline__ void load_features(const InferArgs& a, long long row, int cq, FeatureShare& f) {
  const int pairs = a.n_in >> 1, per = (pairs + 3) >> 2, p0 = cq * per;
  const bool live = row < a.M;
  const float* xr = a.x + (live ? row : 0) * a.n_in;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int p = p0 + i;
    const bool ok = live && i < per && p < pairs;
    f.v[2 * i] = ok ? __ldg(xr + 2 * p) : 0.0f;
    f.v[2 * i + 1] = ok ? __ldg(xr + 2 * p + 1) : 0.0f;
  }
}

// columns [0, n) x_h, [n, 2n) x_l, [2n, 3n) x_h, [3n, 64 kb0) zero
__device__ __forceinline__ void store_features(unsigned char* act, const InferArgs& a, int r, int cq,
                                               const FeatureShare& f) {
  const int n = a.n_in, pairs = n >> 1, per = (pairs + 3) >> 2, p0 = cq * per;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int p = p0 + i;
    if (i >= per || p >= pairs) break;
    const float x0 = f.v[2 * i], x1 = f.v[2 * i + 1];
    const float h0 = __bfloat162float(__float2bfloat16_rn(x0)), h1 = __bfloat162float(__float2bfloat16_rn(x1));
    const uint32_t hi = bf16x2(h0, h1), lo = bf16x2(x0 - h0, x1 - h1);
    *reinterpret_cast<uint32_t*>(act + act_off(r, 2 * p)) = hi;
    *reinterpret_cast<uint32_t*>(act + act_off(r, n + 2 * p)) = lo;
    *reinterpret_cast<uint32_t*>(act + act_off(r, 2 * n + 2 * p)) = hi;
  }
  if (cq == 3)
    for (int c = 3 * n; c < 64 * a.kb0; c += 2) *reinterpret_cast<uint32_t*>(act + act_off(r, c)) = 0u;
}

__global__ void __launch_bounds__(THREADS, 1) k_mlp_infer(const __grid_constant__ CUtensorMap tmW, const InferArgs a) {
  using namespace inf;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* act = base;                      // [2 slots][4 k-blocks][128 rows][128 B]
  unsigned char* wring = base + 2 * ACT_BYTES;    // [WSTAGES][256 rows][128 B]
  uint64_t* bars = reinterpret_cast<uint64_t*>(wring + WSTAGES * WBOX_BYTES);
  // barrier slots: wfull[WSTAGES], wempty[WSTAGES], ready[2], full[2], drain
  const uint32_t b_wfull = smem_u32(bars), b_wempty = smem_u32(bars + WSTAGES);
  const uint32_t b_ready = smem_u32(bars + 2 * WSTAGES), b_full = smem_u32(bars + 2 * WSTAGES + 2);
  const uint32_t b_drain = smem_u32(bars + 2 * WSTAGES + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * WSTAGES + 5);
  __shared__ int abort_flag;
  __shared__ int head_count[8];  // [slot][lane quarter]: column quarters done

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long tiles = (a.M + BM - 1) / BM, pairs = (tiles + 1) / 2;
  const uint32_t tmem_cols = 2 * N;

  if (threadIdx.x < 8) head_count[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < WSTAGES; ++s) {
      mbar_init(b_wfull + 8 * s, 1);
      mbar_init(b_wempty + 8 * s, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(b_ready + 8 * s, EPI_WARPS);  // one arrival per epilogue warp
      mbar_init(b_full + 8 * s, 1);
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
      int stage = 0;
      uint32_t phase = 0;
      int issued[WSTAGES] = {};
      for (long long P = blockIdx.x; P < pairs; P += gridDim.x) {
        const int ns = 2 * P + 1 < tiles ? 2 : 1;
        int kbg = 0;
        for (int l = 0; l < a.L; ++l) {
          const int KB = l == 0 ? a.kb0 : KB_HIDDEN;
          for (int s = 0; s < ns; ++s)
            for (int kb = 0; kb < KB; ++kb) {
              if (!mbar_wait(b_wempty + 8 * stage, phase ^ 1, a.err, 11, abort)) goto tma_done;
              mbar_expect_tx(b_wfull + 8 * stage, (uint32_t)WBOX_BYTES);
              tma_load_2d(smem_u32(wring + (size_t)stage * WBOX_BYTES), &tmW, 0, (kbg + kb) * N, b_wfull + 8 * stage);
              ++issued[stage];
              if (++stage == WSTAGES) {
                stage = 0;
                phase ^= 1;
              }
            }
          kbg += KB;
        }
      }
    tma_done:
      if (*abort) {
        // loads still in flight land in shared memory: wait for them (bounded)
        const long long t0 = clock64();
        for (int s = 0; s < WSTAGES; ++s) {
          if (issued[s] == 0) continue;
          const uint32_t par = (uint32_t)((issued[s] - 1) & 1);
          while (!mbar_test(b_wfull + 8 * s, par) && clock64() - t0 < WAIT_CYCLES) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, N);
      int stage = 0;
      uint32_t phase = 0, ready_ph = 0;  // bit s: the parity slot s waits for next
      bool ok = true;
      for (long long P = blockIdx.x; ok && P < pairs; P += gridDim.x) {
        const int ns = 2 * P + 1 < tiles ? 2 : 1;
        for (int l = 0; ok && l < a.L; ++l) {
          const int KB = l == 0 ? a.kb0 : KB_HIDDEN;
          for (int s = 0; ok && s < ns; ++s) {
            if (!(ok = mbar_wait(b_ready + 8 * s, (ready_ph >> s) & 1u, a.err, 12, abort))) break;
            ready_ph ^= 1u << s;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(s * N);
            const uint32_t a_base = smem_u32(act + (size_t)s * ACT_BYTES);
            for (int kb = 0; kb < KB; ++kb) {
              if (!(ok = mbar_wait(b_wfull + 8 * stage, phase, a.err, 13, abort))) break;
              tc_fence_after();
              const uint32_t a0 = a_base + (uint32_t)(kb * KB_BYTES);
              const uint32_t b0 = smem_u32(wring + (size_t)stage * WBOX_BYTES);
#pragma unroll
              for (int k = 0; k < BK / UMMA_K; ++k)
                umma_bf16(d, sw128_desc(a0 + 32 * k), sw128_desc(b0 + 32 * k), idesc, (kb | k) != 0);
              umma_commit(b_wempty + 8 * stage);  // the ring slot is free once these MMAs have read it
              if (++stage == WSTAGES) {
                stage = 0;
                phase ^= 1;
              }
            }
            if (ok) umma_commit(b_full + 8 * s);
          }
        }
      }
      // every MMA issued so far has completed once this commit arrives
      umma_commit(b_drain);
      const long long t0 = clock64();
      while (!mbar_test(b_drain, 0) && clock64() - t0 < WAIT_CYCLES) {
      }
    }
  } else {
    const int q = warp & 3;           // the lane quarter this warp may read
    const int cq = (warp - 2) >> 2;   // its 64-column quarter = one k-block of the next layer
    const int r = q * 32 + lane;      // row within the tile
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    uint32_t full_ph = 0;  // bit s: the parity slot s waits for next
    FeatureShare fs;
    // the first pair's features
    if ((long long)blockIdx.x < pairs) {
      const long long P = blockIdx.x;
      const int ns = 2 * P + 1 < tiles ? 2 : 1;
      for (int s = 0; s < ns; ++s) {
        load_features(a, (2 * P + s) * BM + r, cq, fs);
        store_features(act + (size_t)s * ACT_BYTES, a, r, cq, fs);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMAs (async proxy)
        __syncwarp();
        if (lane == 0) mbar_arrive(b_ready + 8 * s);
      }
    }
    bool ok = true;
    for (long long P = blockIdx.x; ok && P < pairs; P += gridDim.x) {
      const int ns = 2 * P + 1 < tiles ? 2 : 1;
      const long long Pn = P + gridDim.x;  // this CTA's next pair
      for (int l = 0; ok && l < a.L; ++l) {
        const bool last = l == a.L - 1;
        const float* bias = a.bias[l];
        for (int s = 0; s < ns; ++s) {
          const long long row = (2 * P + s) * BM + r;
          const bool next = Pn < pairs && 2 * Pn + s < tiles;  // a next tile for this slot
          unsigned char* as = act + (size_t)s * ACT_BYTES;
          if (last && next) load_features(a, (2 * Pn + s) * BM + r, cq, fs);  // in flight during the head
          if (!(ok = mbar_wait(b_full + 8 * s, (full_ph >> s) & 1u, a.err, 14, abort))) break;
          full_ph ^= 1u << s;
          tc_fence_after();
          const uint32_t tacc = tmem + (uint32_t)(s * N) + lane_base;
          float h0 = 0.0f, h1 = 0.0f;
          if (!last) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              // 32 columns; the bias loads are in flight with the tensor-memory loads
              const int c0 = cq * 64 + half * 32;
              uint32_t u[2][16];
              tmem_ld16_nw(tacc + (uint32_t)c0, u[0]);
              tmem_ld16_nw(tacc + (uint32_t)(c0 + 16), u[1]);
              float4 b4[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) b4[j] = __ldg(reinterpret_cast<const float4*>(bias + c0) + j);
              tmem_wait_ld();
              // the next layer's A operand: 32 columns = four 16-byte chunks
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float4 p = b4[2 * j], q = b4[2 * j + 1];
                const uint32_t* x = &u[j >> 1][(8 * j) & 15];
                const uint4 w4 = make_uint4(bf16x2(silu_f(__uint_as_float(x[0]) + p.x), silu_f(__uint_as_float(x[1]) + p.y)),
                                            bf16x2(silu_f(__uint_as_float(x[2]) + p.z), silu_f(__uint_as_float(x[3]) + p.w)),
                                            bf16x2(silu_f(__uint_as_float(x[4]) + q.x), silu_f(__uint_as_float(x[5]) + q.y)),
                                            bf16x2(silu_f(__uint_as_float(x[6]) + q.z), silu_f(__uint_as_float(x[7]) + q.w)));
                *reinterpret_cast<uint4*>(as + act_off(r, c0 + 8 * j)) = w4;
              }
            }
          } else {
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
              // 16 columns with their bias and output weights ([c][2]: two columns per float4)
              const int c0 = cq * 64 + ch * 16;
              uint32_t u[16];
              tmem_ld16_nw(tacc + (uint32_t)c0, u);
              float4 b4[4], w4[8];
#pragma unroll
              for (int j = 0; j < 4; ++j) b4[j] = __ldg(reinterpret_cast<const float4*>(bias + c0) + j);
#pragma unroll
              for (int j = 0; j < 8; ++j) w4[j] = __ldg(reinterpret_cast<const float4*>(a.w_out + 2 * c0) + j);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float bl = (j & 1) ? b4[j >> 1].z : b4[j >> 1].x, bh = (j & 1) ? b4[j >> 1].w : b4[j >> 1].y;
                const float v0 = silu_f(__uint_as_float(u[2 * j]) + bl), v1 = silu_f(__uint_as_float(u[2 * j + 1]) + bh);
                h0 = fmaf(v0, w4[j].x, h0);
                h1 = fmaf(v0, w4[j].y, h1);
                h0 = fmaf(v1, w4[j].z, h0);
                h1 = fmaf(v1, w4[j].w, h1);
              }
            }
          }
          if (last) {
            // the column quarters' partial sums in the slot's k-blocks 2-3
            // (the input features of the slot's next tile take k-blocks 0-1)
            float* hp = reinterpret_cast<float*>(as + 2 * KB_BYTES);
            hp[(cq * BM + r) * 2] = h0;
            hp[(cq * BM + r) * 2 + 1] = h1;
            __syncwarp();
            int prior = 0;
            if (lane == 0) {
              __threadfence_block();
              prior = atomicAdd(&head_count[s * 4 + q], 1);
            }
            prior = __shfl_sync(0xffffffffu, prior, 0);
            if (prior == 3) {
              __threadfence_block();
              if (row < a.M) {
                float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  s0 += hp[(c * BM + r) * 2];
                  s1 += hp[(c * BM + r) * 2 + 1];
                }
                *reinterpret_cast<float2*>(a.out + 2 * row) = make_float2(s0 + a.b_out[0], s1 + a.b_out[1]);
              }
              __syncwarp();
              if (lane == 0) head_count[s * 4 + q] = 0;
            }
            if (next) store_features(as, a, r, cq, fs);
          }
          if (!last || next) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_ready + 8 * s);
          }
        }
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
