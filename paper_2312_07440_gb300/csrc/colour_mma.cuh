// Colour sum J^dagger C J on the tensor cores (mixed-precision modes).
//
// Each of the 32 lanes of a warp holds the K colour-ordered amplitudes J of
// one (event, helicity).  The warp stages them as 64 real rows (Re J, Im J per
// lane) of FP16 or BF16 in shared memory (16-byte stores), scaled per lane by
// an exact power of two so that max |J_k| lies in [0.5, 1) (FP16 range),
// reads them back as A fragments with ldmatrix, multiplies the 64 x KP block
// by the integer colour matrix C_int (K x K, every entry exact in FP16 and
// BF16) with mma.sync m16n8k16 and FP32 accumulation, and forms each row's
// dot product J16 . (C J16) of the rounded, scaled amplitudes J16 from the A
// and D fragments the thread already holds.  Since C is real and symmetric,
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

// CM_STORE_FP16 / CM_STORE_BF16: the amplitude code writes each J vector
// (rounded to FP16 / BF16) to global memory for a separate tensor-core colour
// pass instead of summing colours itself (colour_tc.cuh).
enum ColourMode { CM_FMA = 0, CM_FP16 = 1, CM_BF16 = 2, CM_STORE_FP16 = 3, CM_STORE_BF16 = 4 };

// the sink of the fused kernels: nothing is stored
struct NoSink {
  template <int K>
  __device__ __forceinline__ void put(const cx<float> (&)[K]) {}
};

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
// LDS = KP + 8 keeps every row 16-byte aligned and makes the eight rows an
// ldmatrix reads at a time fall into distinct bank groups.  The stages of a
// block's warps sit in its dynamic shared memory right after the amplitude
// code's current store (the kernel accounts per_thread bytes per thread).
template <int KP>
struct ColourStage {
  static constexpr int LDS = KP + 8;
  unsigned short j[64 * LDS];
  float row[64];
  static constexpr int bytes = 64 * LDS * 2 + 64 * 4;
  static_assert(bytes % 32 == 0, "a whole number of bytes per thread of the warp");
  static constexpr int per_thread = bytes / 32;
};

__device__ __forceinline__ void ldmatrix_x4(unsigned (&r)[4], const void* row_addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"((unsigned)__cvta_generic_to_shared(row_addr)));
}

// The tensor-core colour sum of one process.  CI: the integer colour matrix
// (K x K, row-major, device memory); js: the amplitude code's shared bytes
// per thread that precede the stages.  Construct once per amplitude call (B
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
  Stage* st;

  // B fragments of C_int (col-major K x N): b0,b1 = rows 2c, 2c+1 of column g;
  // b2,b3 = rows 2c+8, 2c+9 (zero outside K x K).
  __device__ __forceinline__ ColourMma(const short* __restrict__ CI, int js) {
    l = threadIdx.x & 31;
    g = l >> 2;
    c = l & 3;
    st = nullptr;
    if (!CI) return;  // FMA colour sum: nothing to stage
    extern __shared__ __align__(16) unsigned char rw_dyn_bytes[];
    st = reinterpret_cast<Stage*>(rw_dyn_bytes + (size_t)js * blockDim.x) + (threadIdx.x >> 5);
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

  // this lane's sum_{i,j} C_int_ij Re(J16_i^* J16_j) with J16 the scaled,
  // rounded amplitudes, unscaled again
  __device__ __forceinline__ float sum(const cx<float> (&J)[K]) const {
    Stage& S = *st;
    // per-lane power-of-two scale: max |J| -> [0.5, 1)
    float mx = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) mx = fmaxf(mx, fmaxf(fabsf(J[k].r), fabsf(J[k].i)));
    int e = 0;
    if (mx > 0.0f && isfinite(mx)) frexpf(mx, &e);
    const float sc = ldexpf(1.0f, -e);
    // rows 2l (Re J) and 2l+1 (Im J), 16 bytes at a time
    unsigned re[KP / 2], im[KP / 2];
#pragma unroll
    for (int k = 0; k < KP; k += 2) {
      re[k / 2] = (unsigned)(k < K ? to_16<CM>(J[k].r * sc) : 0) |
                  ((unsigned)(k + 1 < K ? to_16<CM>(J[k + 1].r * sc) : 0) << 16);
      im[k / 2] = (unsigned)(k < K ? to_16<CM>(J[k].i * sc) : 0) |
                  ((unsigned)(k + 1 < K ? to_16<CM>(J[k + 1].i * sc) : 0) << 16);
    }
    uint4* rr = reinterpret_cast<uint4*>(&S.j[(2 * l) * LDS]);
    uint4* ri = reinterpret_cast<uint4*>(&S.j[(2 * l + 1) * LDS]);
#pragma unroll
    for (int q = 0; q < KP / 8; ++q) {
      rr[q] = make_uint4(re[4 * q], re[4 * q + 1], re[4 * q + 2], re[4 * q + 3]);
      ri[q] = make_uint4(im[4 * q], im[4 * q + 1], im[4 * q + 2], im[4 * q + 3]);
    }
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      const int r0 = mt * 16 + g, r1 = r0 + 8;
      // A fragments: lanes 0-15 address rows mt*16 + (0..15) at k0, lanes
      // 16-31 the same rows at k0 + 8 -> (a0, a1, a2, a3) of m16n8k16
      unsigned af[KT][4];
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) ldmatrix_x4(af[kt], &S.j[(mt * 16 + (l & 15)) * LDS + kt * 16 + (l >> 4) * 8]);
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
        S.row[r0] = p0;
        S.row[r1] = p1;
      }
    }
    __syncwarp();
    const float v = S.row[2 * l] + S.row[2 * l + 1];
    __syncwarp();  // the stage is reused by the next call
    return ldexpf(v, 2 * e);
  }
};

}  // namespace rw
