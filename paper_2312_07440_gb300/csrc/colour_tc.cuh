// Colour sum J^dagger C J as a separate pass on the 5th-generation tensor
// cores (mixed-precision modes of g g -> t tbar g g; the colour sum is a5 of
// the hot path: |M_h|^2 = (Re J)^T C (Re J) + (Im J)^T C (Im J), C = C_int/den
// real and symmetric).
//
// k_amp_store runs the helicity amplitudes exactly as the FP32 mode does (same
// set-up, same current recursion, same launch shapes), but instead of summing
// colours it writes every colour-ordered amplitude vector J (the K complex
// amplitudes of one event, parameter point and helicity) to global memory as
// two real rows, Re J and Im J, of K FP16 or BF16 values scaled by 2^-e so
// that max_k |J_k| lies in [0.5, 1), with e stored beside them.  The rows of
// one plane -- a (point, helicity slot, Re/Im) triple -- are consecutive over
// the events, so a warp's stores are contiguous and the colour pass reads
// whole 128-event tiles of a plane.
//
// k_colour_tc walks those tiles, one helicity slot of 128 events at a time:
// the Re and Im rows of an event share one 128-byte row of the staged tile
// ([Re J | 0 | Im J | 0], K = 64), multiplied on the tensor cores by the
// block-diagonal [[C_int, 0], [0, C_int]] (tcgen05.mma kind::f16, M = 128,
// N = 64, four K = 16 steps, FP32 accumulator in tensor memory, the tile in
// the 128-byte-swizzled K-major layout; the next slot's rows are already on
// their way into registers), and each of the 128 threads, owning one event,
// forms Re J16 . (C_int Re J16) + Im J16 . (C_int Im J16) from its
// accumulator row and its staged row, scales by 2^(2e) and sums the slots of
// a point:
//   |M_p|^2 = cscale_p x 2 x sum over the point's planes
// (the 2 for the helicity flip, as in the fused kernel).  The ratio, W' and
// the compensated cross sections then follow exactly as in k_reweight
// (kernels.cuh), for up to DEFER_MAX_POINTS points.
//
// Error: J is rounded to 11 (FP16) or 8 (BF16) significant bits, as in the
// in-kernel tensor-core colour sum (colour_mma.cuh); the products are exact
// in FP32 and accumulate in FP32.
//
// Every mbarrier wait gives up after ~2^31 clock cycles: the error flag is
// set, all threads leave the tile loop together, MMAs still in flight are
// waited for (bounded) and the tensor memory is freed before the kernel
// returns; the cross sections of such a launch are not valid.
#pragma once
#include "colour_mma.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace rw {

constexpr int DEFER_MAX_POINTS = 3;  // modified points per launch of the deferred colour pass
constexpr int CT_THREADS = 128;      // one event (tensor-memory lane) per thread
constexpr int CT_TILE_BYTES = 128 * 128;  // one A tile: 128 rows x 128 bytes (swizzle rows)
// A tiles (two in flight), the B tile (64 rows x 128 bytes), barriers; the
// request is rounded up so that four blocks share an SM (with the largest
// shared-memory carveout), whose 512 tensor-memory columns hold their 128 each
constexpr size_t CT_SMEM_USED = 1024 + 2 * CT_TILE_BYTES + 64 * 128 + 64;
constexpr size_t CT_SMEM = 48 * 1024;
static_assert(CT_SMEM >= CT_SMEM_USED, "shared memory of the colour pass");

__host__ __device__ constexpr long long align_up(long long x, long long a) { return (x + a - 1) / a * a; }

// the amplitude buffers of a launch with npts evaluations (original + points)
// of events padded to ld rows, K colour flows, SLOTS J vectors per event and
// evaluation: rows [npts][SLOTS][2][ld][K] (16-bit), exponents
// [npts][SLOTS][ld] (int16), "masses fit" flags [npts][ld]
struct DeferLayout {
  long long ld;
  long long j16_off, ex_off, ins_off, total;
  __host__ __device__ DeferLayout(int npts, long long ld_, int K, int slots) : ld(ld_) {
    j16_off = 0;
    ex_off = align_up((long long)npts * slots * 2 * ld * K * 2, 256);
    ins_off = ex_off + align_up((long long)npts * slots * ld * 2, 256);
    total = ins_off + align_up((long long)npts * ld, 256);
  }
};

// where the amplitude code's J vectors go (CM_STORE_*): slot q of this
// (event, point) in the planes 2q (Re) and 2q + 1 (Im), exponent at [q][ev];
// ev < 0 (a padding lane of the last grid-stride trip) stores nothing
template <int K, int CM>
struct ColourSink {
  static_assert(K % 8 == 0, "rows of whole 16-byte chunks");
  static constexpr int CM16 = CM == CM_STORE_BF16 ? CM_BF16 : CM_FP16;
  uint4* j16;
  short* ex;
  long long ld, ev;
  int q;
  __device__ __forceinline__ void put(const cx<float> (&J)[K]) {
    if (ev >= 0) {
      float mx = 0.0f;
#pragma unroll
      for (int k = 0; k < K; ++k) mx = fmaxf(mx, fmaxf(fabsf(J[k].r), fabsf(J[k].i)));
      int e = 0;
      if (mx > 0.0f && isfinite(mx)) frexpf(mx, &e);
      e = max(e, -120);  // keeps 2^-e finite in FP32
      const float sc = ldexpf(1.0f, -e);
      uint4* rr = j16 + ((long long)(2 * q) * ld + ev) * (K / 8);
      uint4* ri = rr + ld * (K / 8);
#pragma unroll
      for (int c = 0; c < K / 8; ++c) {
        unsigned wr[4], wi[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int k = 8 * c + 2 * h;
          wr[h] = (unsigned)to_16<CM16>(J[k].r * sc) | ((unsigned)to_16<CM16>(J[k + 1].r * sc) << 16);
          wi[h] = (unsigned)to_16<CM16>(J[k].i * sc) | ((unsigned)to_16<CM16>(J[k + 1].i * sc) << 16);
        }
        rr[c] = make_uint4(wr[0], wr[1], wr[2], wr[3]);
        ri[c] = make_uint4(wi[0], wi[1], wi[2], wi[3]);
      }
      ex[(long long)q * ld + ev] = (short)e;
    }
    ++q;
  }
};

// The amplitude pass: grid-stride over events like k_reweight, every
// evaluation (original, then each point) through Proc::me_store.
template <class Proc, int LB, int CM>
__global__ void __launch_bounds__(256, 1) k_amp_store(const __grid_constant__ RwArgs a) {
  constexpr int NEXT = Proc::NEXT;
  constexpr int LANES = 1 << LB;
  constexpr int K = Proc::NCOL;
  constexpr int SLOTS = 1 << (NEXT - 1);  // helicities with the first gluon at +1
  const int tid = threadIdx.x;
  const int wl = tid & 31;
  const int lane = tid & (LANES - 1);
  const unsigned gmask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << (wl & ~(LANES - 1)));
  const long long gpb = blockDim.x / LANES;
  const long long ngroups = (long long)gridDim.x * gpb;
  const long long g0 = (long long)blockIdx.x * gpb + tid / LANES;
  const long long E = a.E;
  const int npts = a.me_only ? 1 : a.P + 1;
  const DeferLayout L(npts, a.defer_ld, K, SLOTS);
  uint4* j16 = reinterpret_cast<uint4*>(a.defer + L.j16_off);
  short* ex = reinterpret_cast<short*>(a.defer + L.ex_off);
  unsigned char* ins = a.defer + L.ins_off;
  for (long long base = 0; base < E; base += ngroups) {
    const long long ev = base + g0;
    const bool valid = ev < E;
    const long long evc = valid ? ev : E - 1;
    typename Proc::template mom_t<float> p[NEXT][4];
#pragma unroll
    for (int i = 0; i < NEXT; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) load_mom(p[i][m], __ldg(a.mom + ((long long)(i * 4 + m)) * a.ld + evc));
#pragma unroll 1
    for (int j = 0; j < npts; ++j) {
      ColourSink<K, CM> sk{j16, ex, L.ld, valid ? ev : -1, j * SLOTS + lane * (SLOTS >> LB)};
      const bool inside = Proc::template me_store<float, LB>(p, a.pt[j], lane, gmask, sk);
      if (valid && lane == 0) ins[(long long)j * L.ld + ev] = inside ? 1 : 0;
    }
  }
}

// the colour matrix of a process: CTab::at(i) = C_int[i / K][i % K]
template <int K, int CM, int SLOTS, class CTab>
__global__ void __launch_bounds__(CT_THREADS) k_colour_tc(const __grid_constant__ RwArgs a, int* err) {
  static_assert(K <= 32 && K % 8 == 0, "Re and Im halves of one 128-byte row");
  constexpr int CM16 = CM == CM_STORE_BF16 ? CM_BF16 : CM_FP16;
  constexpr int KC = K / 8;  // 16-byte chunks of one J row
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sbase =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = sbase;                      // [2][128 rows][128 B]
  unsigned char* sB = sbase + 2 * CT_TILE_BYTES;  // [64 rows][128 B]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 64 * 128);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  __shared__ double2 sacc[CT_THREADS / 32][DEFER_MAX_POINTS + 1];
  __shared__ double2 red[32];
  __shared__ int is_last;
  __shared__ int abort_flag;
  const int t = threadIdx.x, warp = t >> 5, wl = t & 31;
  const int P = a.me_only ? 0 : a.P;
  const int npts = P + 1;
  const int nsl = npts * SLOTS;  // items (helicity slots) per event tile
  const long long E = a.E;
  const long long ldo = a.ldo ? a.ldo : a.E;
  const DeferLayout L(npts, a.defer_ld, K, SLOTS);
  const long long ld = L.ld;
  const uint4* j16 = reinterpret_cast<const uint4*>(a.defer + L.j16_off);
  const short* ex = reinterpret_cast<const short*>(a.defer + L.ex_off);
  const unsigned char* ins = a.defer + L.ins_off;

  // B operand, K-major: row n < 32 holds C_int[n][k] at k < K, row 32 + n
  // holds C_int[n][k - 32] at 32 <= k < 32 + K (C_int is symmetric), zero
  // elsewhere; 16-byte chunk c of row n at position c ^ (n % 8)
  for (int i = t; i < 64 * 64; i += CT_THREADS) {
    const int n = i >> 6, k = i & 63;
    const int nn = n & 31, kk = k - (n & 32);
    const float v = (nn < K && kk >= 0 && kk < K) ? (float)CTab::at(nn * K + kk) : 0.0f;
    *reinterpret_cast<unsigned short*>(sB + n * 128 + (((k >> 3) ^ (n & 7)) << 4) + (k & 7) * 2) = to_16<CM16>(v);
  }
  const uint32_t bar0 = tcg::smem_u32(bars);
  if (t == 0) {
    abort_flag = 0;
    tcg::mbar_init(bar0, 1);
    tcg::mbar_init(bar0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // sB visible to the tensor cores
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tcg::smem_u32(tmem_slot)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tcg::tc_fence_before();
  __syncthreads();
  tcg::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t fmt = CM16 == CM_BF16 ? 1u : 0u;
  constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
  volatile int* abort = &abort_flag;

  const long long tiles = (E + 127) / 128;
  const long long mine = tiles > blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long total = mine * nsl;
  double rs[DEFER_MAX_POINTS + 1], rc[DEFER_MAX_POINTS + 1];
#pragma unroll
  for (int q = 0; q <= DEFER_MAX_POINTS; ++q) rs[q] = rc[q] = 0.0;
  unsigned long long nbad = 0;
  float acc = 0.0f;
  double me0 = 0.0, w = 0.0;
  bool ok0 = false;
  uint32_t par[2] = {0u, 0u};
  int issued[2] = {0, 0}, seen[2] = {0, 0};
  // item it: event tile blockIdx.x + (it / nsl) gridDim.x, slot it % nsl; its
  // rows (Re then Im chunks) and exponent are loaded one item ahead
  uint4 nre[KC], nim[KC];
  int ne = 0, ce = 0, pe = 0;
  auto load_item = [&](long long it) {
    const long long ev = (blockIdx.x + (it / nsl) * gridDim.x) * 128 + t;  // < ld: planes padded to whole tiles
    const int q = (int)(it % nsl);
    const uint4* re = j16 + ((long long)(2 * q) * ld + ev) * KC;
    const uint4* im = re + ld * KC;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      nre[c] = __ldcs(re + c);
      nim[c] = __ldcs(im + c);
    }
    ne = __ldcs(ex + (long long)q * ld + ev);
  };
  if (total > 0) load_item(0);
  for (long long it = 0; it <= total; ++it) {
    if (it < total) {
      unsigned char* row = sA + (it & 1) * CT_TILE_BYTES + t * 128;
      const int sw = t & 7;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        *reinterpret_cast<uint4*>(row + ((c ^ sw) << 4)) = c < KC ? nre[c] : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(row + (((4 + c) ^ sw) << 4)) = c < KC ? nim[c] : make_uint4(0u, 0u, 0u, 0u);
      }
      ce = ne;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the row visible to the tensor cores
      if (it + 1 < total) load_item(it + 1);
    }
    tcg::tc_fence_before();
    __syncthreads();
    tcg::tc_fence_after();
    if (*abort) break;  // set before the barrier by a wait that gave up: every thread leaves
    if (it < total && t == 0) {
      const int b = (int)(it & 1);
      const uint32_t a0 = tcg::smem_u32(sA + b * CT_TILE_BYTES), b0 = tcg::smem_u32(sB);
      const uint32_t d = tmem + 64u * b;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        tcg::umma_bf16(d, tcg::sw128_desc(a0 + 32 * k), tcg::sw128_desc(b0 + 32 * k), idesc, k ? 1u : 0u);
      tcg::umma_commit(bar0 + 8 * b);
      ++issued[b];
    }
    if (it >= 1) {
      const int b = (int)((it - 1) & 1);
      // on a timeout the loop ends at the next barrier (this item's sums are void)
      if (tcg::mbar_wait(bar0 + 8 * b, par[b], err, 1, abort)) {
        par[b] ^= 1u;
        ++seen[b];
      }
      tcg::tc_fence_after();
      // the accumulator row (C Re J16 in columns 0..31, C Im J16 in 32..63)
      // and this thread's staged row of the previous item
      const uint32_t taddr = tmem + 64u * b + ((uint32_t)(warp * 32) << 16);
      const unsigned char* row = sA + b * CT_TILE_BYTES + t * 128;
      const int sw = t & 7;
      uint32_t dr[4][16];
#pragma unroll
      for (int q = 0; q < 4; ++q) tcg::tmem_ld16_nw(taddr + 16 * q, dr[q]);
      tcg::tmem_wait_ld();
      float dot = 0.0f;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float d[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) d[i] = __uint_as_float(dr[2 * half + i / 16][i % 16]);
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          const uint4 v = *reinterpret_cast<const uint4*>(row + (((4 * half + c) ^ sw) << 4));
          const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            dot = fmaf(from_16<CM16>((unsigned short)(u[h] & 0xffffu)), d[8 * c + 2 * h], dot);
            dot = fmaf(from_16<CM16>((unsigned short)(u[h] >> 16)), d[8 * c + 2 * h + 1], dot);
          }
        }
      }
      acc += ldexpf(dot, 2 * pe);
      const int sp = (int)((it - 1) % nsl);
      if (sp % SLOTS == SLOTS - 1) {  // the last slot of evaluation jp of this tile
        const int jp = sp / SLOTS;
        const long long ev = (blockIdx.x + ((it - 1) / nsl) * gridDim.x) * 128 + t;
        const bool valid = ev < E;
        const double me = (valid && ins[(long long)jp * ld + ev]) ? 2.0 * (double)acc * a.pt[jp].cscale : 0.0;
        acc = 0.0f;
        if (jp == 0) {
          me0 = me;
          if (valid) {
            if (a.me_only) {
              a.me0[ev] = me;
            } else {
              ok0 = isfinite(me0) && me0 != 0.0;
              if (!ok0) ++nbad;
              if (a.me0) a.me0[ev] = me0;
              w = __ldg(a.w + ev);
#pragma unroll
              for (int q = 0; q <= DEFER_MAX_POINTS; ++q)
                if (q == P) two_sum_acc(rs[q], rc[q], w, 0.0);
            }
          }
        } else if (valid) {
          const double r = ok0 ? me / me0 : 0.0;
          const double wn = ok0 ? r * w : 0.0;
          const long long o = (long long)(jp - 1) * ldo + ev;
          if (a.me_pts) a.me_pts[o] = me;
          if (a.ratio) a.ratio[o] = r;
          if (a.wnew) a.wnew[o] = wn;
#pragma unroll
          for (int q = 0; q < DEFER_MAX_POINTS; ++q)
            if (q == jp - 1) two_sum_acc(rs[q], rc[q], wn, 0.0);
        }
      }
      tcg::tc_fence_before();
    }
    pe = ce;
  }
  // MMAs whose completion was not seen (a wait gave up): wait for them, bounded
  if (t == 0) {
    const long long t0 = clock64();
    for (int b = 0; b < 2; ++b)
      while (seen[b] < issued[b] && clock64() - t0 < tcg::WAIT_CYCLES) {
        if (tcg::mbar_test(bar0 + 8 * b, par[b])) {
          par[b] ^= 1u;
          ++seen[b];
        }
      }
  }
  tcg::tc_fence_before();
  __syncthreads();
  tcg::tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
  if (a.me_only) return;
  // block partial sums, then the last block to finish reduces them in a fixed order
  const int stride = P + 1;
#pragma unroll
  for (int q = 0; q <= DEFER_MAX_POINTS; ++q) {
    if (q > P) break;
    double s = rs[q], c = rc[q];
    warp_sum2(s, c);
    if (wl == 0) sacc[warp][q] = make_double2(s, c);
  }
  __syncthreads();
  for (int j = t; j < stride; j += CT_THREADS) {
    double s = 0.0, c = 0.0;
    for (int wi = 0; wi < CT_THREADS / 32; ++wi) two_sum_acc(s, c, sacc[wi][j].x, sacc[wi][j].y);
    a.block_part[(long long)blockIdx.x * stride + j] = make_double2(s, c);
  }
  if (nbad) atomicAdd(a.nbad_count, nbad);
  __threadfence();
  __syncthreads();
  if (t == 0) is_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int j = 0; j < stride; ++j) {
    double s = 0.0, c = 0.0;
    for (int b = t; b < (int)gridDim.x; b += CT_THREADS) {
      const double2 v = __ldcg(a.block_part + (long long)b * stride + j);
      two_sum_acc(s, c, v.x, v.y);
    }
    block_sum2(s, c, red);
    if (t == 0) {
      if (a.sigma_acc) {
        double2 u = a.accumulate ? a.sigma_acc[j] : make_double2(0.0, 0.0);
        two_sum_acc(u.x, u.y, s, c);
        a.sigma_acc[j] = u;
        a.sigma[j] = u.x + u.y;
        if (a.sigma_pair) a.sigma_pair[j] = u;
      } else {
        a.sigma[j] = s + c;
        if (a.sigma_pair) a.sigma_pair[j] = make_double2(s, c);
      }
    }
  }
  if (t == 0) {
    const unsigned long long nb = atomicExch(a.nbad_count, 0ull);
    *a.nbad_out = a.accumulate ? *a.nbad_out + nb : nb;
    *a.ticket = 0u;
  }
}

}  // namespace rw
