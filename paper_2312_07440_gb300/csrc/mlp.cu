// Learned surrogate for log r = log(|M'|^2/|M|^2): a multilayer perceptron
// n_in -> [hidden, SiLU] x n_layers -> 2 (mu = predicted log r, s = predicted
// log of its error).  Hidden layers: BF16 weights and activations, FP32
// accumulation on the tensor cores; the first layer (from the unrounded FP32
// features) and the output layer run in FP32 (about 4 % of the flops); FP32
// master weights with Adam.  Every step of training and inference runs in the
// kernels of this file:
//   k_mlp_infer    (mlp_infer_tc.cuh) inference of the whole network in one
//                  tensor-core kernel, activations in shared memory, the
//                  input layer as a BF16 MMA over split operands
//   k_gemm_tc      (gemm_tc.cuh) the hidden layers' forward GEMMs on the
//                  5th-generation tensor cores (tcgen05.mma, TMA-fed, FP32
//                  accumulators in tensor memory), bias + SiLU fused, and for
//                  layer-by-layer inference the output layer fused into the last one
//   k_gemm<EPI>    C = A B with strided (optionally transposed) BF16 operands
//                  on mma.sync (the backward GEMMs; the forward when the
//                  layer shape is outside k_gemm_tc's),
//                  fused epilogues: bias + SiLU (forward), bias (output layer),
//                  x SiLU'(z) (backward data), FP32 store (weight gradients,
//                  the batch split into row slices)
//   k_colsum_part  bias gradients over row slices of the batch
//   k_sum_parts    the slices added in order (deterministic)
//   k_loss         MSE on mu + Gaussian NLL on s with the residual detached
//   k_adam         Adam on FP32 master weights, BF16 copies for the GEMMs
//   k_gather_rows  minibatch gather
// The C ABI (rw_mlp_*) is declared in include/rwgt.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/rwgt.h"
#include "gemm_tc.cuh"
#include "mlp_infer_tc.cuh"

namespace {

using bf16 = unsigned short;

__device__ __forceinline__ float bf2f(bf16 x) { return __bfloat162float(__ushort_as_bfloat16(x)); }
__device__ __forceinline__ float to_f32(bf16 x) { return bf2f(x); }
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ bf16 f2bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + __expf(-z)); }

enum Epi { EPI_FWD_SILU = 0, EPI_FWD_LINEAR = 1, EPI_BWD_DATA = 2, EPI_WGRAD = 3 };

struct GemmArgs {
  const bf16* A;  // element (m, k) at A[m * sam + k * sak]
  const bf16* B;  // element (k, n) at B[k * sbk + n * sbn]
  long long sam, sak, sbk, sbn;
  int M, N, K;
  const float* bias;  // [N] (forward epilogues)
  float* Zf;          // FWD_SILU: pre-activation out [M][N]; BWD_DATA: pre-activation in [M][N]
  bf16* H;            // FWD_SILU: activation out; BWD_DATA: dZ out  [M][N] bf16
  float* C;           // FWD_LINEAR / WGRAD: FP32 out [M][N] (WGRAD: one [M][N] slice per split)
  int kps;            // WGRAD: k (batch rows) per split; block z takes [z kps, (z + 1) kps)
};

constexpr int BM = 64, BN = 64, BK = 32, LDA = BK + 8;

// 128 threads, 2 x 2 warps, each warp 32 x 32 (2 m16 tiles x 4 n8 tiles).
template <int EPI>
__global__ void __launch_bounds__(128) k_gemm(const GemmArgs g) {
  __shared__ __align__(16) bf16 As[BM * LDA];  // [m][k]
  __shared__ __align__(16) bf16 Bs[BN * LDA];  // [n][k]
  const int tid = threadIdx.x, warp = tid >> 5, l = tid & 31;
  const int gr = l >> 2, gc = l & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = EPI == EPI_WGRAD ? blockIdx.z * g.kps : 0;
  const int ke = EPI == EPI_WGRAD ? min(g.K, kb + g.kps) : g.K;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
  for (int k0 = kb; k0 < ke; k0 += BK) {
    // cooperative tile loads (bounds -> zero); consecutive threads walk the
    // operand's contiguous dimension
    const bool a_k_fast = g.sak == 1, b_k_fast = g.sbk == 1;
#pragma unroll 4
    for (int i = tid; i < BM * BK; i += 128) {
      const int mm = a_k_fast ? i / BK : i % BM, kk = a_k_fast ? i % BK : i / BM;
      const int m = m0 + mm, k = k0 + kk;
      As[mm * LDA + kk] = (m < g.M && k < ke) ? g.A[m * g.sam + k * g.sak] : (bf16)0;
    }
#pragma unroll 4
    for (int i = tid; i < BN * BK; i += 128) {
      const int nn = b_k_fast ? i / BK : i % BN, kk = b_k_fast ? i % BK : i / BN;
      const int n = n0 + nn, k = k0 + kk;
      Bs[nn * LDA + kk] = (n < g.N && k < ke) ? g.B[k * g.sbk + n * g.sbn] : (bf16)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r0 = wm + i * 16 + gr;
        af[i][0] = *reinterpret_cast<const unsigned*>(&As[r0 * LDA + kk + 2 * gc]);
        af[i][1] = *reinterpret_cast<const unsigned*>(&As[(r0 + 8) * LDA + kk + 2 * gc]);
        af[i][2] = *reinterpret_cast<const unsigned*>(&As[r0 * LDA + kk + 8 + 2 * gc]);
        af[i][3] = *reinterpret_cast<const unsigned*>(&As[(r0 + 8) * LDA + kk + 8 + 2 * gc]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c0 = wn + j * 8 + gr;
        bfr[j][0] = *reinterpret_cast<const unsigned*>(&Bs[c0 * LDA + kk + 2 * gc]);
        bfr[j][1] = *reinterpret_cast<const unsigned*>(&Bs[c0 * LDA + kk + 8 + 2 * gc]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
  // epilogue: acc[i][j] = rows (wm+16i+gr, +8), cols (wn+8j+2gc, +1)
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + i * 16 + gr + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * gc + (q & 1);
        if (m >= g.M || n >= g.N) continue;
        const long long o = (long long)m * g.N + n;
        const float v = acc[i][j][q];
        if constexpr (EPI == EPI_FWD_SILU) {
          const float z = v + g.bias[n];
          g.Zf[o] = z;
          g.H[o] = f2bf(z * sigmoidf_(z));
        } else if constexpr (EPI == EPI_FWD_LINEAR) {
          g.C[o] = v + g.bias[n];
        } else if constexpr (EPI == EPI_BWD_DATA) {
          const float z = g.Zf[o];
          const float s = sigmoidf_(z);
          g.H[o] = f2bf(v * s * (1.0f + z * (1.0f - s)));
        } else {
          g.C[(long long)blockIdx.z * g.M * g.N + o] = v;
        }
      }
}

// First layer in FP32 (the inputs are never rounded): Z = X W + b,
// H = bf16(SiLU(Z)); one thread per (row, unit), W [nin][N] FP32.
__global__ void k_dense_in(const float* __restrict__ X, int B, int nin, const float* __restrict__ W,
                           const float* __restrict__ b, int N, float* __restrict__ Z, bf16* __restrict__ H) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * N) return;
  const int r = (int)(t / N), n = (int)(t % N);
  float z = b[n];
  for (int k = 0; k < nin; ++k) z = fmaf(X[(long long)r * nin + k], W[(long long)k * N + n], z);
  if (Z) Z[t] = z;  // pre-activation: kept for the backward pass and the unfused output layer
  H[t] = f2bf(z * sigmoidf_(z));
}

// The same first layer, register-blocked for hidden = 256 and n_in <= 64:
// a block of 256 threads computes 64 rows x 256 units; the weights [n_in][256]
// and the block's feature rows sit in shared memory, and each thread
// accumulates 8 rows x 8 consecutive units (64 FMAs per 16 shared loads),
// then writes 8-unit runs of Z (FP32, when kept) and H (BF16, 16 bytes).
constexpr int DI_ROWS = 64, DI_N = 256, DI_MAX_IN = 64;
__global__ void __launch_bounds__(256) k_dense_in_256(const float* __restrict__ X, int B, int nin,
                                                      const float* __restrict__ W, const float* __restrict__ b,
                                                      float* __restrict__ Z, bf16* __restrict__ H) {
  extern __shared__ __align__(16) float di_smem[];
  float* Ws = di_smem;                      // [nin][256]
  float* Xs = di_smem + nin * DI_N;         // [DI_ROWS][nin + 1]
  const int ldx = nin + 1;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const long long r0 = (long long)blockIdx.x * DI_ROWS;
  for (int i = tid; i < nin * DI_N / 4; i += 256)
    reinterpret_cast<float4*>(Ws)[i] = __ldg(reinterpret_cast<const float4*>(W) + i);
  for (int i = tid; i < DI_ROWS * nin; i += 256) {
    const int r = i / nin, k = i % nin;
    Xs[r * ldx + k] = r0 + r < B ? __ldg(X + (r0 + r) * nin + k) : 0.0f;
  }
  __syncthreads();
  float acc[8][8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float bj = __ldg(b + tx * 8 + j);
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][j] = bj;
  }
  for (int k = 0; k < nin; ++k) {
    const float4 w0 = reinterpret_cast<const float4*>(Ws + k * DI_N + tx * 8)[0];
    const float4 w1 = reinterpret_cast<const float4*>(Ws + k * DI_N + tx * 8)[1];
    const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float xv = Xs[(ty * 8 + i) * ldx + k];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(xv, wv[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long r = r0 + ty * 8 + i;
    if (r >= B) continue;
    const long long o = r * DI_N + tx * 8;
    if (Z) {
      reinterpret_cast<float4*>(Z + o)[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      reinterpret_cast<float4*>(Z + o)[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
    unsigned hw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float z0 = acc[i][2 * j], z1 = acc[i][2 * j + 1];
      hw[j] = (unsigned)f2bf(z0 * sigmoidf_(z0)) | ((unsigned)f2bf(z1 * sigmoidf_(z1)) << 16);
    }
    *reinterpret_cast<uint4*>(H + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  }
}

// Output layer in FP32 from the last pre-activation: out = SiLU(Z) W + b,
// W [K][2]; one warp per row.
__global__ void k_dense_out(const float* __restrict__ Z, int B, int K, const float* __restrict__ W,
                            const float* __restrict__ b, float* __restrict__ out) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), l = threadIdx.x & 31;
  if (r >= B) return;
  float a0 = 0.0f, a1 = 0.0f;
  for (int k = l; k < K; k += 32) {
    const float z = Z[(long long)r * K + k];
    const float h = z * sigmoidf_(z);
    a0 = fmaf(h, W[2 * k], a0);
    a1 = fmaf(h, W[2 * k + 1], a1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
  }
  if (l == 0) {
    out[2 * r] = a0 + b[0];
    out[2 * r + 1] = a1 + b[1];
  }
}

// Backward through the output layer: dZ[r][k] = (sum_o dOut[r][o] W[k][o]) SiLU'(Z[r][k])
__global__ void k_dense_out_bwd(const float* __restrict__ dout, const float* __restrict__ Z, int B, int K,
                                const float* __restrict__ W, bf16* __restrict__ dZ) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * K) return;
  const int r = (int)(t / K), k = (int)(t % K);
  const float z = Z[t], s = sigmoidf_(z);
  const float dh = dout[2 * r] * W[2 * k] + dout[2 * r + 1] * W[2 * k + 1];
  dZ[t] = f2bf(dh * s * (1.0f + z * (1.0f - s)));
}

// db[n] = sum_m dZ[m][n]   (one thread per column, fixed order)
// Column sums of D [M][N] (BF16 or FP32) over row slice z = blockIdx.y of
// rps rows: parts [S][N]; k_sum_parts adds the slices in order.
template <class T>
__global__ void k_colsum_part(const T* __restrict__ D, int M, int N, int rps, float* __restrict__ parts) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int r0 = blockIdx.y * rps, r1 = min(M, r0 + rps);
  float s = 0.0f;
  for (int m = r0; m < r1; ++m) s += to_f32(D[(long long)m * N + n]);
  parts[(long long)blockIdx.y * N + n] = s;
}

// out[i] = sum_{z < S} parts[z][i], slices in order (deterministic)
__global__ void k_sum_parts(const float* __restrict__ parts, int S, long long count, float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float s = 0.0f;
  for (int z = 0; z < S; ++z) s += parts[(long long)z * count + i];
  out[i] = s;
}

// Loss per sample (mean over the batch): ((y - mu)/tau)^2 + lam (r^2 e^{-2s}/2 + s),
// r = y - mu treated as a constant in the second term.  Writes dOut [B][2]
// (FP32 and BF16) and the per-sample loss.
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ y, int B, float inv_tau2, float lam,
                       float* __restrict__ dout_f, bf16* __restrict__ dout_b, float* __restrict__ loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float mu = out[2 * b], s = fminf(fmaxf(out[2 * b + 1], -16.0f), 4.0f);
  const float r = y[b] - mu;
  const float e2 = __expf(-2.0f * s);
  const float dmu = -2.0f * r * inv_tau2 / B;
  const float ds = lam * (1.0f - r * r * e2) / B;
  dout_f[2 * b] = dmu;
  dout_f[2 * b + 1] = ds;
  dout_b[2 * b] = f2bf(dmu);
  dout_b[2 * b + 1] = f2bf(ds);
  loss[b] = r * r * inv_tau2 + lam * (0.5f * r * r * e2 + s);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m1,
                       float* __restrict__ m2, bf16* __restrict__ pb, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gr[i];
  const float a = b1 * m1[i] + (1.0f - b1) * g;
  const float v = b2 * m2[i] + (1.0f - b2) * g * g;
  m1[i] = a;
  m2[i] = v;
  const float q = p[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
  p[i] = q;
  pb[i] = f2bf(q);
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = f2bf(x[i]);
}

// BF16 transpose of a K x N FP32 weight matrix: Wt[n][k] = bf16(W[k][n])
// (the tensor-core GEMM reads the weights K-major)
__global__ void k_transpose_bf16(const float* __restrict__ W, int K, int N, bf16* __restrict__ Wt) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)K * N) return;
  const int n = (int)(t / K), k = (int)(t % K);
  Wt[t] = f2bf(W[(long long)k * N + n]);
}

// The inference kernel's weights: k-block g, row n, column k of
//   g < kb0:  the split input layer [W_h ; W_h ; W_l ; 0] along k (rows of
//             W_0 [nin][256]: W_h = bf16(W), W_l = bf16(W - W_h)),
//   g >= kb0: W_l^T of hidden layer l = 1 + (g - kb0) / 4 in BF16.
struct PackArgs {
  const float* W[tcg::inf::MAX_LAYERS];
  int nin, kb0, n_kb;
};
__global__ void k_pack_infer(const PackArgs a, bf16* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)a.n_kb * 256 * 64) return;
  const int k = (int)(t & 63), n = (int)((t >> 6) & 255), g = (int)(t >> 14);
  float v = 0.0f;
  if (g < a.kb0) {
    const int c = g * 64 + k, f = c % a.nin, part = c / a.nin;
    if (part < 3) {
      const float w = a.W[0][(long long)f * 256 + n];
      const float wh = __bfloat162float(__float2bfloat16_rn(w));
      v = part == 2 ? w - wh : wh;
    }
  } else {
    const int l = 1 + (g - a.kb0) / 4, kk = ((g - a.kb0) % 4) * 64 + k;
    v = a.W[l][(long long)kk * 256 + n];
  }
  out[t] = f2bf(v);
}

// rows idx[b] of X [*][nin] (FP32) -> Xf [B][nin] (FP32) and Xb (BF16), y[idx[b]] -> yb[b]
__global__ void k_gather_rows(const float* __restrict__ X, const float* __restrict__ y, const int64_t* __restrict__ idx,
                              int B, int nin, float* __restrict__ Xf, bf16* __restrict__ Xb, float* __restrict__ yb) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * nin) return;
  const int b = (int)(t / nin), j = (int)(t % nin);
  const int64_t r = idx[b];
  const float v = X[r * nin + j];
  Xf[t] = v;
  Xb[t] = f2bf(v);
  if (j == 0 && y) yb[b] = y[r];
}

// minibatch indices: a counter-based hash (splitmix64) of (seed, step, b)
__global__ void k_batch_indices(uint64_t seed, uint64_t step, int B, int64_t n, int64_t* __restrict__ idx) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (step * 0x100000001ull + (uint64_t)b + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  idx[b] = (int64_t)(z % (uint64_t)n);
}

}  // namespace

// ---------------------------------------------------------------------------
// the model object
// ---------------------------------------------------------------------------
struct rw_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_in = 0, hidden = 0, n_layers = 0, max_batch = 0;
  int n_out = 2;
  std::vector<int> din, dout;           // per linear layer
  std::vector<long long> w_off, b_off;  // offsets in the parameter vector
  long long n_params = 0;
  float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;  // FP32 [n_params]
  bf16* pb = nullptr;                                              // BF16 copy
  long long step = 0;
  // activations for one batch
  bf16* X = nullptr;                  // [max_batch][n_in] (BF16 copy, weight gradients)
  float* Xf = nullptr;                // [max_batch][n_in] FP32 (training minibatch)
  std::vector<bf16*> H;               // per hidden layer [max_batch][hidden]
  std::vector<float*> Z;              // pre-activations
  float* out = nullptr;               // [max_batch][2]
  float* dout_f = nullptr;
  bf16* dout_b = nullptr;
  bf16 *dA = nullptr, *dB = nullptr;  // dZ ping-pong [max_batch][hidden]
  float* gparts = nullptr;            // weight-gradient slices of the split batch [<= 512 x 64 x 64]
  float* cparts = nullptr;            // bias-gradient slices [64][max(hidden, 2)]
  float* loss = nullptr;              // [max_batch]
  float* yb = nullptr;
  int64_t* idx = nullptr;
  // tensor-core forward: transposed BF16 hidden weights [l][N][K] (layer l at
  // (l - 1) hidden^2), its error flag, and the GEMM choice
  bf16* wt = nullptr;
  // whole-network inference kernel: weight k-blocks [kb][256 n][64 k] BF16 in
  // the order the MMAs take them (the split input layer's kb0, then 4 per
  // hidden layer)
  bf16* wpack = nullptr;
  int kb0 = 0;
  int* tc_err = nullptr;
  int gemm = 0;  // 0: tcgen05, inference in one kernel; 2: tcgen05 layer by layer; 1: mma.sync everywhere
  int sm_count = 0;
  std::string err;
};

namespace {

int mlp_fail(rw_mlp* m, int code, const char* msg) {
  if (m) m->err = msg;
  return code;
}

// ---- tensor-core forward (gemm_tc.cuh) ------------------------------------
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled() {
  static EncodeTiled fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiled>(f);
  }();
  return fn;
}

// a 2-D BF16 row-major matrix [rows][cols] as a TMA map with boxes of
// 64 columns (128 bytes, 128-byte swizzle) x box_rows rows
bool bf16_map(CUtensorMap* map, const bf16* ptr, long long rows, int cols, int box_rows) {
  const EncodeTiled enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(bf16)};
  const cuuint32_t box[2] = {(cuuint32_t)tcg::BK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(ptr), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// hidden layers on the tensor cores: width a multiple of 64, at most 256
bool tc_usable(const rw_mlp* m) {
  return m->gemm != 1 && m->wt && m->hidden % tcg::BK == 0 && m->hidden <= tcg::MAX_N && encode_tiled();
}

// the whole inference in one kernel: hidden 256, n_in <= 40, at most 8 layers
bool infer_usable(const rw_mlp* m) { return m->gemm == 0 && m->wpack && encode_tiled(); }

// out [n][2] = MLP(x [n][n_in]) for all n rows in one launch
int launch_mlp_infer(rw_mlp* m, const float* x, long long n, float* out) {
  const int L = m->n_layers;
  CUtensorMap tw;
  if (!bf16_map(&tw, m->wpack, (long long)(m->kb0 + 4 * (L - 1)) * 256, tcg::BK, 256))
    return mlp_fail(m, RW_ERR_CUDA, "tensor map encoding");
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tcg::k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tcg::inf::SMEM_BYTES) != cudaSuccess)
      return mlp_fail(m, RW_ERR_CUDA, "inference kernel shared memory attribute");
    attr = true;
  }
  tcg::InferArgs a{};
  a.x = x;
  for (int l = 0; l < L; ++l) a.bias[l] = m->p + m->b_off[l];
  a.w_out = m->p + m->w_off[L];
  a.b_out = m->p + m->b_off[L];
  a.out = out;
  a.err = m->tc_err;
  a.M = n;
  a.n_in = m->n_in;
  a.kb0 = m->kb0;
  a.L = L;
  const long long pairs = ((n + tcg::BM - 1) / tcg::BM + 1) / 2;
  const int grid = (int)std::max(1LL, std::min<long long>(pairs, m->sm_count));
  tcg::k_mlp_infer<<<grid, tcg::THREADS, tcg::inf::SMEM_BYTES, m->stream>>>(tw, a);
  return cudaGetLastError() == cudaSuccess ? RW_OK : mlp_fail(m, RW_ERR_CUDA, "inference kernel launch");
}

// hidden layer l (1 <= l < n_layers) of B rows: A = bf16 activations [B][hidden]
// backward (e.Zin set): dZ_{l-1} = bf16((dZ_l W_l^T) SiLU'(Z_{l-1})), whose B
// operand [k = input unit][n = output unit] is W_l's BF16 copy as stored
int launch_gemm_tc(rw_mlp* m, int l, const bf16* A, int B, tcg::Epi e) {
  const int H = m->hidden;
  CUtensorMap ta, tb;
  const bf16* Bop = e.Zin ? m->pb + m->w_off[l] : m->wt + (size_t)(l - 1) * H * H;
  if (!bf16_map(&ta, A, B, H, tcg::BM) || !bf16_map(&tb, Bop, H, H, H))
    return mlp_fail(m, RW_ERR_CUDA, "tensor map encoding");
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tcg::k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcg::SMEM_BYTES) !=
        cudaSuccess)
      return mlp_fail(m, RW_ERR_CUDA, "tensor-core GEMM shared memory attribute");
    attr = true;
  }
  e.bias = m->p + m->b_off[l];
  e.err = m->tc_err;
  e.M = B;
  e.N = H;
  e.K = H;
  const int tiles = (B + tcg::BM - 1) / tcg::BM;
  const int grid = std::max(1, std::min(tiles, m->sm_count));
  tcg::k_gemm_tc<<<grid, tcg::THREADS, tcg::SMEM_BYTES, m->stream>>>(ta, tb, e);
  return cudaGetLastError() == cudaSuccess ? RW_OK : mlp_fail(m, RW_ERR_CUDA, "tensor-core GEMM launch");
}

// transposed BF16 copies of the hidden weights (after any change of p)
int refresh_wt(rw_mlp* m) {
  const int H = m->hidden;
  if (m->wt)
    for (int l = 1; l < m->n_layers; ++l)
      k_transpose_bf16<<<(unsigned)(((long long)H * H + 255) / 256), 256, 0, m->stream>>>(
          m->p + m->w_off[l], H, H, m->wt + (size_t)(l - 1) * H * H);
  if (m->wpack) {
    PackArgs a{};
    for (int l = 0; l < m->n_layers; ++l) a.W[l] = m->p + m->w_off[l];
    a.nin = m->n_in;
    a.kb0 = m->kb0;
    a.n_kb = m->kb0 + 4 * (m->n_layers - 1);
    k_pack_infer<<<(unsigned)(((long long)a.n_kb * 256 * 64 + 255) / 256), 256, 0, m->stream>>>(a, m->wpack);
  }
  return cudaGetLastError() == cudaSuccess ? RW_OK : mlp_fail(m, RW_ERR_CUDA, "weight transpose");
}

// the tensor-core kernels' error flag (a wait that gave up); synchronises
int tc_status(rw_mlp* m) {
  if (!m->tc_err) return RW_OK;
  int h = 0;
  if (cudaMemcpyAsync(&h, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return mlp_fail(m, RW_ERR_CUDA, "status copy");
  if (h) return mlp_fail(m, RW_ERR_CUDA, "tensor-core GEMM: a pipeline wait timed out");
  return RW_OK;
}

int launch_gemm(rw_mlp* m, int epi, GemmArgs a) {
  dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM);
  switch (epi) {
    case EPI_FWD_SILU: k_gemm<EPI_FWD_SILU><<<grid, 128, 0, m->stream>>>(a); break;
    case EPI_FWD_LINEAR: k_gemm<EPI_FWD_LINEAR><<<grid, 128, 0, m->stream>>>(a); break;
    case EPI_BWD_DATA: k_gemm<EPI_BWD_DATA><<<grid, 128, 0, m->stream>>>(a); break;
    default: a.kps = a.K; k_gemm<EPI_WGRAD><<<grid, 128, 0, m->stream>>>(a); break;
  }
  return cudaGetLastError() == cudaSuccess ? RW_OK : mlp_fail(m, RW_ERR_CUDA, "gemm launch");
}

// Forward for B <= max_batch rows of FP32 features xf (device); output in
// m->out.  First and last layers in FP32, hidden layers BF16 on the tensor
// cores.  infer: only the output is needed, so the last hidden layer's
// tensor-core epilogue computes the output layer itself and writes neither
// its pre-activation nor its activation.
int forward_batch(rw_mlp* m, const float* xf, int B, bool infer = false) {
  const int L = m->n_layers;
  const bool tc = tc_usable(m);
  // inference on the tensor-core path reads no pre-activation back
  const bool keep_z = !(infer && tc && L >= 2);
  if (m->hidden == DI_N && m->n_in <= DI_MAX_IN) {
    const size_t sm = ((size_t)m->n_in * DI_N + (size_t)DI_ROWS * (m->n_in + 1)) * sizeof(float);
    static bool attr = false;
    if (!attr && sm > 48 * 1024) {
      if (cudaFuncSetAttribute(k_dense_in_256, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024) != cudaSuccess)
        return mlp_fail(m, RW_ERR_CUDA, "first-layer shared memory attribute");
      attr = true;
    }
    k_dense_in_256<<<(unsigned)((B + DI_ROWS - 1) / DI_ROWS), 256, sm, m->stream>>>(
        xf, B, m->n_in, m->p + m->w_off[0], m->p + m->b_off[0], keep_z ? m->Z[0] : nullptr, m->H[0]);
  } else {
    k_dense_in<<<(unsigned)(((long long)B * m->hidden + 255) / 256), 256, 0, m->stream>>>(
        xf, B, m->n_in, m->p + m->w_off[0], m->p + m->b_off[0], m->hidden, keep_z ? m->Z[0] : nullptr, m->H[0]);
  }
  for (int l = 1; l < L; ++l) {
    if (tc) {
      tcg::Epi e{};
      if (infer && l == L - 1) {
        e.w_out = m->p + m->w_off[L];
        e.b_out = m->p + m->b_off[L];
        e.out = m->out;
      } else {
        e.Z = keep_z ? m->Z[l] : nullptr;
        e.H = m->H[l];
      }
      const int rc = launch_gemm_tc(m, l, m->H[l - 1], B, e);
      if (rc) return rc;
      if (infer && l == L - 1) return RW_OK;
      continue;
    }
    GemmArgs a{};
    a.A = m->H[l - 1];
    a.sam = m->hidden;
    a.sak = 1;
    a.B = m->pb + m->w_off[l];
    a.sbk = m->dout[l];
    a.sbn = 1;
    a.M = B;
    a.N = m->dout[l];
    a.K = m->din[l];
    a.bias = m->p + m->b_off[l];
    a.Zf = m->Z[l];
    a.H = m->H[l];
    int rc = launch_gemm(m, EPI_FWD_SILU, a);
    if (rc) return rc;
  }
  k_dense_out<<<(B + 7) / 8, 256, 0, m->stream>>>(m->Z[L - 1], B, m->hidden, m->p + m->w_off[L], m->p + m->b_off[L],
                                                 m->out);
  return cudaGetLastError() == cudaSuccess ? RW_OK : mlp_fail(m, RW_ERR_CUDA, "forward launch");
}

// Weight gradient w.C [M][N] = sum over the batch (k) of the GemmArgs
// product, the batch split into S slices of a multiple of 32 rows so that
// about 512 blocks run; the slices go to m->gparts and are added in order.
constexpr int WGRAD_BLOCKS = 512;
int launch_wgrad(rw_mlp* m, GemmArgs w) {
  const int tiles = ((w.N + BN - 1) / BN) * ((w.M + BM - 1) / BM);
  int S = std::max(1, std::min(WGRAD_BLOCKS / tiles, (w.K + BK - 1) / BK));
  w.kps = ((w.K + S - 1) / S + BK - 1) / BK * BK;
  S = (w.K + w.kps - 1) / w.kps;
  float* dst = w.C;
  w.C = m->gparts;
  k_gemm<EPI_WGRAD><<<dim3((w.N + BN - 1) / BN, (w.M + BM - 1) / BM, S), 128, 0, m->stream>>>(w);
  const long long cnt = (long long)w.M * w.N;
  k_sum_parts<<<(unsigned)((cnt + 255) / 256), 256, 0, m->stream>>>(m->gparts, S, cnt, dst);
  return cudaGetLastError() == cudaSuccess ? RW_OK : mlp_fail(m, RW_ERR_CUDA, "weight-gradient launch");
}

// bias gradient out [N] = column sums of D [M][N], in up to 64 row slices
template <class T>
int launch_colsum(rw_mlp* m, const T* D, int M, int N, float* out) {
  const int rps = (M + 63) / 64, S = (M + rps - 1) / rps;
  k_colsum_part<T><<<dim3((N + 127) / 128, S), 128, 0, m->stream>>>(D, M, N, rps, m->cparts);
  k_sum_parts<<<(unsigned)((N + 255) / 256), 256, 0, m->stream>>>(m->cparts, S, N, out);
  return cudaGetLastError() == cudaSuccess ? RW_OK : mlp_fail(m, RW_ERR_CUDA, "bias-gradient launch");
}

// Backward: gradients of the loss (m->dout_f set, m->X holds the BF16
// inputs) into m->g.  Weight gradients on the tensor cores (BF16 operands,
// FP32 accumulation); the output layer's backward in FP32.
int backward_batch(rw_mlp* m, int B) {
  const int L = m->n_layers;
  int rc;
  // output layer: dW = H_{L-1}^T dOut, db = colsum(dOut), dZ_{L-1}
  {
    GemmArgs w{};
    w.A = m->H[L - 1];
    w.sam = 1;
    w.sak = m->hidden;
    w.B = m->dout_b;
    w.sbk = m->n_out;
    w.sbn = 1;
    w.M = m->hidden;
    w.N = m->n_out;
    w.K = B;
    w.C = m->g + m->w_off[L];
    if ((rc = launch_wgrad(m, w))) return rc;
    if ((rc = launch_colsum<float>(m, m->dout_f, B, m->n_out, m->g + m->b_off[L]))) return rc;
    k_dense_out_bwd<<<(unsigned)(((long long)B * m->hidden + 255) / 256), 256, 0, m->stream>>>(
        m->dout_f, m->Z[L - 1], B, m->hidden, m->p + m->w_off[L], m->dA);
  }
  bf16* bufs[2] = {m->dA, m->dB};
  int cur = 0;  // dZ of layer l lives in bufs[cur]
  for (int l = L - 1; l >= 0; --l) {
    const bf16* dZ = bufs[cur];
    const bf16* Hin = l == 0 ? m->X : m->H[l - 1];
    const int nin = m->din[l];
    GemmArgs w{};
    w.A = Hin;
    w.sam = 1;
    w.sak = nin;
    w.B = dZ;
    w.sbk = m->hidden;
    w.sbn = 1;
    w.M = nin;
    w.N = m->hidden;
    w.K = B;
    w.C = m->g + m->w_off[l];
    if ((rc = launch_wgrad(m, w))) return rc;
    if ((rc = launch_colsum<bf16>(m, dZ, B, m->hidden, m->g + m->b_off[l]))) return rc;
    if (l == 0) break;
    if (tc_usable(m)) {
      tcg::Epi e{};
      e.Zin = m->Z[l - 1];
      e.H = bufs[cur ^ 1];
      if ((rc = launch_gemm_tc(m, l, dZ, B, e))) return rc;
      cur ^= 1;
      continue;
    }
    GemmArgs d{};
    d.A = dZ;
    d.sam = m->hidden;
    d.sak = 1;
    d.B = m->pb + m->w_off[l];  // (k = out unit, n = in unit) -> W[n][k]
    d.sbk = 1;
    d.sbn = m->dout[l];
    d.M = B;
    d.N = nin;
    d.K = m->hidden;
    d.Zf = m->Z[l - 1];
    d.H = bufs[cur ^ 1];
    if ((rc = launch_gemm(m, EPI_BWD_DATA, d))) return rc;
    cur ^= 1;
  }
  return cudaGetLastError() == cudaSuccess ? RW_OK : mlp_fail(m, RW_ERR_CUDA, "backward launch");
}

template <class T>
bool dalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T)) == cudaSuccess;
}

}  // namespace

extern "C" {

int rw_mlp_create(rw_mlp** out, int device, void* stream, int n_in, int hidden, int n_layers, int max_batch,
                  uint64_t seed) {
  if (!out) return RW_ERR_NULL;
  *out = nullptr;
  if (n_in < 1 || n_in % 8 || hidden < 8 || hidden % 8 || n_layers < 1 || n_layers > 16 || max_batch < 1 ||
      max_batch > (1 << 24))
    return RW_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return RW_ERR_CUDA;
  rw_mlp* m = new rw_mlp();
  m->device = device;
  m->stream = static_cast<cudaStream_t>(stream);
  m->n_in = n_in;
  m->hidden = hidden;
  m->n_layers = n_layers;
  m->max_batch = max_batch;
  long long off = 0;
  for (int l = 0; l <= n_layers; ++l) {
    const int a = l == 0 ? n_in : hidden, b = l == n_layers ? m->n_out : hidden;
    m->din.push_back(a);
    m->dout.push_back(b);
    m->w_off.push_back(off);
    off += (long long)a * b;
    m->b_off.push_back(off);
    off += b;
  }
  m->n_params = off;
  // deterministic initialisation: uniform(-sqrt(6/fan_in), +) (SiLU gain ~ ReLU), zero biases,
  // output layer scaled by 0.1; splitmix64 stream from the seed
  std::vector<float> hp(off, 0.0f);
  uint64_t st = seed;
  auto rnd = [&st]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int l = 0; l <= n_layers; ++l) {
    const double lim = sqrt(6.0 / m->din[l]) * (l == n_layers ? 0.1 : 1.0);
    for (long long i = 0; i < (long long)m->din[l] * m->dout[l]; ++i)
      hp[m->w_off[l] + i] = (float)((2.0 * rnd() - 1.0) * lim);
  }
  bool ok = dalloc(&m->p, off) && dalloc(&m->g, off) && dalloc(&m->m1, off) && dalloc(&m->m2, off) &&
            dalloc(&m->pb, off) && dalloc(&m->X, (size_t)max_batch * n_in) &&
            dalloc(&m->Xf, (size_t)max_batch * n_in) &&
            dalloc(&m->out, (size_t)max_batch * 2) && dalloc(&m->dout_f, (size_t)max_batch * 2) &&
            dalloc(&m->dout_b, (size_t)max_batch * 2) && dalloc(&m->dA, (size_t)max_batch * hidden) &&
            dalloc(&m->dB, (size_t)max_batch * hidden) && dalloc(&m->loss, (size_t)max_batch) &&
            dalloc(&m->yb, (size_t)max_batch) && dalloc(&m->idx, (size_t)max_batch) &&
            dalloc(&m->gparts, (size_t)WGRAD_BLOCKS * BM * BN) &&
            dalloc(&m->cparts, (size_t)64 * std::max(hidden, m->n_out));
  for (int l = 0; ok && l < n_layers; ++l) {
    bf16* h = nullptr;
    float* z = nullptr;
    ok = dalloc(&h, (size_t)max_batch * hidden) && dalloc(&z, (size_t)max_batch * hidden);
    m->H.push_back(h);
    m->Z.push_back(z);
  }
  if (ok) ok = cudaMemcpy(m->p, hp.data(), off * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemset(m->m1, 0, off * sizeof(float)) == cudaSuccess &&
               cudaMemset(m->m2, 0, off * sizeof(float)) == cudaSuccess;
  if (ok) ok = cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, device) == cudaSuccess &&
               dalloc(&m->tc_err, 1) && cudaMemset(m->tc_err, 0, sizeof(int)) == cudaSuccess;
  if (ok && n_layers >= 2 && hidden % tcg::BK == 0 && hidden <= tcg::MAX_N)
    ok = dalloc(&m->wt, (size_t)(n_layers - 1) * hidden * hidden);
  if (ok && hidden == tcg::inf::N && n_in <= tcg::inf::MAX_IN && n_layers <= tcg::inf::MAX_LAYERS) {
    m->kb0 = (3 * n_in + tcg::BK - 1) / tcg::BK;
    ok = dalloc(&m->wpack, (size_t)(m->kb0 + 4 * (n_layers - 1)) * 256 * 64);
  }
  if (ok) {
    k_to_bf16<<<(unsigned)((off + 255) / 256), 256, 0, m->stream>>>(m->p, m->pb, off);
    ok = refresh_wt(m) == RW_OK && cudaStreamSynchronize(m->stream) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    rw_mlp_destroy(m);
    return RW_ERR_CUDA;
  }
  *out = m;
  return RW_OK;
}

int rw_mlp_destroy(rw_mlp* m) {
  if (!m) return RW_ERR_NULL;
  cudaSetDevice(m->device);
  for (void* q : {(void*)m->p, (void*)m->g, (void*)m->m1, (void*)m->m2, (void*)m->pb, (void*)m->X, (void*)m->Xf,
                  (void*)m->out,
                  (void*)m->dout_f, (void*)m->dout_b, (void*)m->dA, (void*)m->dB, (void*)m->loss, (void*)m->yb,
                  (void*)m->idx, (void*)m->wt, (void*)m->wpack, (void*)m->gparts, (void*)m->cparts, (void*)m->tc_err})
    if (q) cudaFree(q);
  for (auto* h : m->H) cudaFree(h);
  for (auto* z : m->Z) cudaFree(z);
  delete m;
  return RW_OK;
}

const char* rw_mlp_last_error(const rw_mlp* m) { return m ? m->err.c_str() : "null model"; }

int64_t rw_mlp_n_params(const rw_mlp* m) { return m ? m->n_params : -1; }

int rw_mlp_info(const rw_mlp* m, int* n_in, int* hidden, int* n_layers, void** stream) {
  if (!m) return RW_ERR_NULL;
  if (n_in) *n_in = m->n_in;
  if (hidden) *hidden = m->hidden;
  if (n_layers) *n_layers = m->n_layers;
  if (stream) *stream = static_cast<void*>(m->stream);
  return RW_OK;
}

int rw_mlp_get_state(rw_mlp* m, float* h_params, float* h_m1, float* h_m2, int64_t* h_step) {
  if (!m) return RW_ERR_NULL;
  cudaSetDevice(m->device);
  const size_t nb = m->n_params * sizeof(float);
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mlp_fail(m, RW_ERR_CUDA, "sync");
  if ((h_params && cudaMemcpy(h_params, m->p, nb, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (h_m1 && cudaMemcpy(h_m1, m->m1, nb, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (h_m2 && cudaMemcpy(h_m2, m->m2, nb, cudaMemcpyDeviceToHost) != cudaSuccess))
    return mlp_fail(m, RW_ERR_CUDA, "copy");
  if (h_step) *h_step = m->step;
  return RW_OK;
}

int rw_mlp_set_state(rw_mlp* m, const float* h_params, const float* h_m1, const float* h_m2, int64_t step) {
  if (!m || !h_params) return RW_ERR_NULL;
  cudaSetDevice(m->device);
  const size_t nb = m->n_params * sizeof(float);
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mlp_fail(m, RW_ERR_CUDA, "sync");
  bool ok = cudaMemcpy(m->p, h_params, nb, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && (h_m1 ? cudaMemcpy(m->m1, h_m1, nb, cudaMemcpyHostToDevice) : cudaMemset(m->m1, 0, nb)) == cudaSuccess;
  ok = ok && (h_m2 ? cudaMemcpy(m->m2, h_m2, nb, cudaMemcpyHostToDevice) : cudaMemset(m->m2, 0, nb)) == cudaSuccess;
  if (!ok) return mlp_fail(m, RW_ERR_CUDA, "copy");
  k_to_bf16<<<(unsigned)((m->n_params + 255) / 256), 256, 0, m->stream>>>(m->p, m->pb, m->n_params);
  m->step = step < 0 ? 0 : step;
  if (cudaGetLastError() != cudaSuccess) return mlp_fail(m, RW_ERR_CUDA, "launch");
  return refresh_wt(m);
}

// out [n][2] = MLP(x [n][n_in] FP32), processed in chunks of max_batch rows
int rw_mlp_forward(rw_mlp* m, const float* d_x, int64_t n, float* d_out) {
  if (!m) return RW_ERR_NULL;
  if (!d_x || !d_out) return mlp_fail(m, RW_ERR_NULL, "NULL buffer");
  if (n <= 0) return mlp_fail(m, RW_ERR_ARG, "n must be > 0");
  cudaSetDevice(m->device);
  if (infer_usable(m)) return launch_mlp_infer(m, d_x, n, d_out);
  for (int64_t s = 0; s < n; s += m->max_batch) {
    const int B = (int)std::min<int64_t>(m->max_batch, n - s);
    int rc = forward_batch(m, d_x + s * m->n_in, B, true);
    if (rc) return rc;
    if (cudaMemcpyAsync(d_out + 2 * s, m->out, (size_t)B * 2 * sizeof(float), cudaMemcpyDeviceToDevice,
                        m->stream) != cudaSuccess)
      return mlp_fail(m, RW_ERR_CUDA, "copy out");
  }
  return RW_OK;
}

// Loss gradient at the current parameters for the first n <= max_batch rows
// (no update): h_grad [n_params] (may be NULL), *h_loss the mean loss.
int rw_mlp_gradient(rw_mlp* m, const float* d_x, const float* d_y, int64_t n, float tau, float lam, float* h_grad,
                    float* h_loss) {
  if (!m) return RW_ERR_NULL;
  if (!d_x || !d_y) return mlp_fail(m, RW_ERR_NULL, "NULL buffer");
  if (n <= 0 || n > m->max_batch) return mlp_fail(m, RW_ERR_ARG, "n must be in [1, max_batch]");
  cudaSetDevice(m->device);
  const int B = (int)n;
  k_to_bf16<<<(unsigned)(((long long)B * m->n_in + 255) / 256), 256, 0, m->stream>>>(d_x, m->X,
                                                                                    (long long)B * m->n_in);
  int rc = forward_batch(m, d_x, B);
  if (rc) return rc;
  k_loss<<<(B + 127) / 128, 128, 0, m->stream>>>(m->out, d_y, B, 1.0f / (tau * tau), lam, m->dout_f, m->dout_b,
                                                 m->loss);
  rc = backward_batch(m, B);
  if (rc) return rc;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mlp_fail(m, RW_ERR_CUDA, "sync");
  if ((rc = tc_status(m))) return rc;
  if (h_grad && cudaMemcpy(h_grad, m->g, m->n_params * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return mlp_fail(m, RW_ERR_CUDA, "copy");
  if (h_loss) {
    std::vector<float> lb(B);
    if (cudaMemcpy(lb.data(), m->loss, B * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
      return mlp_fail(m, RW_ERR_CUDA, "copy");
    double s = 0;
    for (float v : lb) s += v;
    *h_loss = (float)(s / B);
  }
  return RW_OK;
}

// Adam training: n_steps minibatches of `batch` rows drawn (counter-based,
// with replacement) from x [n][n_in], y [n]; asynchronous on the model's
// stream.  Resumable: the draw depends on (seed, step counter).
int rw_mlp_train(rw_mlp* m, const float* d_x, const float* d_y, int64_t n, int batch, int64_t n_steps, float lr,
                 float tau, float lam, uint64_t seed) {
  if (!m) return RW_ERR_NULL;
  if (!d_x || !d_y) return mlp_fail(m, RW_ERR_NULL, "NULL buffer");
  if (n <= 0 || batch <= 0 || batch > m->max_batch || n_steps < 0) return mlp_fail(m, RW_ERR_ARG, "bad sizes");
  cudaSetDevice(m->device);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t it = 0; it < n_steps; ++it) {
    const uint64_t step = (uint64_t)m->step;
    k_batch_indices<<<(batch + 127) / 128, 128, 0, m->stream>>>(seed, step, batch, n, m->idx);
    k_gather_rows<<<(unsigned)(((long long)batch * m->n_in + 255) / 256), 256, 0, m->stream>>>(
        d_x, d_y, m->idx, batch, m->n_in, m->Xf, m->X, m->yb);
    int rc = forward_batch(m, m->Xf, batch);
    if (rc) return rc;
    k_loss<<<(batch + 127) / 128, 128, 0, m->stream>>>(m->out, m->yb, batch, 1.0f / (tau * tau), lam, m->dout_f,
                                                       m->dout_b, m->loss);
    rc = backward_batch(m, batch);
    if (rc) return rc;
    m->step += 1;
    const float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
    k_adam<<<(unsigned)((m->n_params + 255) / 256), 256, 0, m->stream>>>(m->p, m->g, m->m1, m->m2, m->pb,
                                                                         m->n_params, lr, b1, b2, eps, c1, c2);
    if ((rc = refresh_wt(m))) return rc;
  }
  return cudaGetLastError() == cudaSuccess ? RW_OK : mlp_fail(m, RW_ERR_CUDA, "train launch");
}

int rw_mlp_set_gemm(rw_mlp* m, int kind) {
  if (!m) return RW_ERR_NULL;
  if (kind < 0 || kind > 2) return mlp_fail(m, RW_ERR_ARG, "kind must be 0, 1 or 2");
  m->gemm = kind;
  return RW_OK;
}

int rw_mlp_status(rw_mlp* m) {
  if (!m) return RW_ERR_NULL;
  cudaSetDevice(m->device);
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mlp_fail(m, RW_ERR_CUDA, "sync");
  return tc_status(m);
}

int rw_mlp_hidden_layer(rw_mlp* m, int layer, const void* d_h_in, int64_t n, float* d_z, void* d_h_out) {
  if (!m) return RW_ERR_NULL;
  if (!d_h_in || !d_z || !d_h_out) return mlp_fail(m, RW_ERR_NULL, "NULL buffer");
  if (layer < 1 || layer >= m->n_layers) return mlp_fail(m, RW_ERR_ARG, "layer must be a hidden layer (1..n_layers-1)");
  if (n <= 0 || n > (int64_t(1) << 30)) return mlp_fail(m, RW_ERR_ARG, "bad n");
  if (reinterpret_cast<uintptr_t>(d_h_in) % 16 || reinterpret_cast<uintptr_t>(d_z) % 16 ||
      reinterpret_cast<uintptr_t>(d_h_out) % 16)
    return mlp_fail(m, RW_ERR_ALIGN, "buffers must be 16-byte aligned");
  cudaSetDevice(m->device);
  const bf16* A = static_cast<const bf16*>(d_h_in);
  bf16* Hout = static_cast<bf16*>(d_h_out);
  if (tc_usable(m)) {
    tcg::Epi e{};
    e.Z = d_z;
    e.H = Hout;
    return launch_gemm_tc(m, layer, A, (int)n, e);
  }
  for (int64_t s = 0; s < n; s += 65535LL * BM) {  // the mma.sync grid's row limit
    GemmArgs a{};
    a.A = A + s * m->hidden;
    a.sam = m->hidden;
    a.sak = 1;
    a.B = m->pb + m->w_off[layer];
    a.sbk = m->dout[layer];
    a.sbn = 1;
    a.M = (int)std::min<int64_t>(n - s, 65535LL * BM);
    a.N = m->dout[layer];
    a.K = m->din[layer];
    a.bias = m->p + m->b_off[layer];
    a.Zf = d_z + s * m->hidden;
    a.H = Hout + s * m->hidden;
    const int rc = launch_gemm(m, EPI_FWD_SILU, a);
    if (rc) return rc;
  }
  return RW_OK;
}

}  // extern "C"
