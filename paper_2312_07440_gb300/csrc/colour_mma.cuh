// Colour sum J^dagger C J on the tensor cores (mixed-precision modes).
//
// Each of the 32 lanes of a warp holds the K colour-ordered amplitudes J of
// one (event, helicity).  The warp stages them as 64 real rows (Re J, Im J per
// lane) of FP16 or BF16 in shared memory, scaled per lane by an exact power
// of two so that max |J_k| lies in [0.5, 1) (FP16 range), multiplies the
// 64 x KP block by the integer colour matrix C_int (K x K, every entry exact
// in FP16 and BF16) with mma.sync m16n8k16 and FP32 accumulation, and forms
// each row's dot product J16 . (C J16) from the A and D fragments the thread
// already holds.  Since C is real and symmetric,
//   J^dagger C J = (Re J)^T C (Re J) + (Im J)^T C (Im J),
// the lane's result is the sum of its two rows, unscaled by 2^(2e).
// Error: the rounding of J to 11 (FP16) or 8 (BF16) significant bits, i.e. a
// relative error of order 1e-3 (FP16) or 1e-2 (BF16) on each helicity's
// colour sum; FP32 accumulation adds nothing visible.
//
// Warp-synchronous: all 32 lanes must call it together.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "helas.cuh"

namespace rw {

enum ColourMode { CM_FMA = 0, CM_FP16 = 1, CM_BF16 = 2 };

template <int CM>
__device__ __forceinline__ unsigned short to_16(float x) {
  if constexpr (CM == CM_FP16) {
    return __half_as_ushort(__float2half_rn(x));
  } else {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
  }
}
template <int CM>
__device__ __forceinline__ float from_16(unsigned short x) {
  if constexpr (CM == CM_FP16) {
    return __half2float(__ushort_as_half(x));
  } else {
    return __bfloat162float(__ushort_as_bfloat16(x));
  }
}

template <int CM>
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  if constexpr (CM == CM_FP16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
}

// Shared staging for one warp: 64 rows x LDS 16-bit words, then 64 row sums.
template <int KP>
struct ColourStage {
  static constexpr int LDS = KP + 8;  // row stride (words): +16 B breaks bank conflicts
  unsigned short j[64 * LDS];
  float row[64];
};

// The tensor-core colour sum of one process.  CI: the integer colour matrix
// (K x K, row-major, device memory).  Construct once per amplitude call (B
// fragments kept in registers); sum() is warp-synchronous.
template <int K, int CM>
struct ColourMma {
  static constexpr int KP = (K + 15) / 16 * 16;  // k extent (multiple of 16)
  static constexpr int NP = (K + 7) / 8 * 8;     // n extent (multiple of 8)
  static constexpr int KT = KP / 16, NT = NP / 8;
  using Stage = ColourStage<KP>;
  static constexpr int LDS = Stage::LDS;
  unsigned bf[KT][NT][2];
  int l, g, c;

  // B fragments of C_int (col-major K x N): b0,b1 = rows 2c, 2c+1 of column g;
  // b2,b3 = rows 2c+8, 2c+9 (zero outside K x K).
  __device__ __forceinline__ explicit ColourMma(const short* __restrict__ CI) {
    l = threadIdx.x & 31;
    g = l >> 2;
    c = l & 3;
    if (!CI) return;  // FMA colour sum: nothing to stage
#pragma unroll
    for (int kt = 0; kt < KT; ++kt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int n = nt * 8 + g;
          const int k0 = kt * 16 + h * 8 + 2 * c;
          const float v0 = (k0 < K && n < K) ? float(CI[k0 * K + n]) : 0.0f;
          const float v1 = (k0 + 1 < K && n < K) ? float(CI[(k0 + 1) * K + n]) : 0.0f;
          bf[kt][nt][h] = (unsigned)to_16<CM>(v0) | ((unsigned)to_16<CM>(v1) << 16);
        }
  }

  // this lane's sum_{i,j} C_int_ij Re(J_i^* J_j)
  __device__ __forceinline__ float sum(const cx<float> (&J)[K]) const {
    __shared__ __align__(16) Stage stage_all[4];  // blocks of at most 128 threads
    Stage& st = stage_all[threadIdx.x >> 5];
    // per-lane power-of-two scale: max |J| -> [0.5, 1)
    float mx = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) mx = fmaxf(mx, fmaxf(fabsf(J[k].r), fabsf(J[k].i)));
    int e = 0;
    if (mx > 0.0f && isfinite(mx)) frexpf(mx, &e);
    const float sc = ldexpf(1.0f, -e);
#pragma unroll
    for (int k = 0; k < KP; k += 2) {
      const unsigned re = (unsigned)(k < K ? to_16<CM>(J[k].r * sc) : 0) |
                          ((unsigned)(k + 1 < K ? to_16<CM>(J[k + 1].r * sc) : 0) << 16);
      const unsigned im = (unsigned)(k < K ? to_16<CM>(J[k].i * sc) : 0) |
                          ((unsigned)(k + 1 < K ? to_16<CM>(J[k + 1].i * sc) : 0) << 16);
      *reinterpret_cast<unsigned*>(&st.j[(2 * l) * LDS + k]) = re;
      *reinterpret_cast<unsigned*>(&st.j[(2 * l + 1) * LDS + k]) = im;
    }
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      const int r0 = mt * 16 + g, r1 = r0 + 8;
      unsigned af[KT][4];
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
        const int k0 = kt * 16 + 2 * c;
        af[kt][0] = *reinterpret_cast<const unsigned*>(&st.j[r0 * LDS + k0]);
        af[kt][1] = *reinterpret_cast<const unsigned*>(&st.j[r1 * LDS + k0]);
        af[kt][2] = *reinterpret_cast<const unsigned*>(&st.j[r0 * LDS + k0 + 8]);
        af[kt][3] = *reinterpret_cast<const unsigned*>(&st.j[r1 * LDS + k0 + 8]);
      }
      float p0 = 0.0f, p1 = 0.0f;  // row partial dots (rows r0, r1)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) mma16816<CM>(d, af[kt], bf[kt][nt]);
        // D(r, 8nt + 2c + q) pairs with J16(r, 8nt + 2c + q): A fragment of k-tile nt/2
        const unsigned ar0 = af[nt / 2][(nt & 1) ? 2 : 0];
        const unsigned ar1 = af[nt / 2][(nt & 1) ? 3 : 1];
        p0 += from_16<CM>(ar0 & 0xffffu) * d[0] + from_16<CM>(ar0 >> 16) * d[1];
        p1 += from_16<CM>(ar1 & 0xffffu) * d[2] + from_16<CM>(ar1 >> 16) * d[3];
      }
      p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
      p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
      p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
      p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
      if (c == 0) {
        st.row[r0] = p0;
        st.row[r1] = p1;
      }
    }
    __syncwarp();
    const float v = st.row[2 * l] + st.row[2 * l + 1];
    __syncwarp();  // the stage is reused by the next call
    return ldexpf(v, 2 * e);
  }
};

}  // namespace rw
