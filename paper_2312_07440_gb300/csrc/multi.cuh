// Several processes in one persistent launch.
//
// The reweighting of Sec. 3.2 applies event by event whatever the process,
// and an NLO sample's real-emission events are tree-level events of one more
// parton (Sec. 4: the real emission reuses the LO machinery), so the events
// of several processes -- e.g. g g -> t tbar and its real emission
// g g -> t tbar g -- can share one launch.  Work items are tiles of one
// process's events (a block's event groups); the tiles of all processes form
// one index range, which the blocks walk grid-stride, so one grid sized to
// the GPU serves every process and the short tiles of a cheap process fill
// the gaps a costly one leaves at the end.  Each process keeps its own
// arguments (points, outputs, workspace: as in k_reweight) and its own cross
// sections sigma'_p and sigma; the last block to finish reduces every
// process's block partials in a fixed order, so results are deterministic
// for a given launch shape.  No block waits on another.
#pragma once
#include "kernels.cuh"

namespace rw {

constexpr int MAX_MULTI = 4;

// a process adapter and the lanes per event (2^LB) it runs with
template <class P, int L>
struct Lanes {
  using Proc = P;
  static constexpr int LB = L;
};

// one process's share of a launch: k_reweight's arguments without the
// point constants, which sit in the launch's common pool from pt0 on
struct MultiItem {
  const double* mom;  // [N][4][ld]
  const double* w;    // [E]
  long long E, ld, ldo;
  double *me0, *me_pts, *ratio, *wnew;  // outputs, each may be null
  double2* block_part;                  // [gridDim.x][P+1]
  double* sigma;                        // [P+1]
  double2* sigma_pair;                  // [P+1]
  unsigned long long* nbad_count;       // zero between launches
  unsigned long long* nbad_out;
  int P, pt0;                           // pool[pt0] original point, pool[pt0 + 1 + j] point j
};

constexpr int MULTI_POOL = 420;  // point constants of all processes (the arguments stay below 32 KB)

struct MultiArgs {
  MultiItem item[MAX_MULTI];      // in the kernel's template order
  long long tile_end[MAX_MULTI];  // item i owns tiles [tile_end[i-1], tile_end[i])
  int sacc_off[MAX_MULTI];        // offset (double2) of item i's warp sums [nwarps][P_i+1]
  int n;
  unsigned int* ticket;           // zero between launches
  PointDev pool[MULTI_POOL];
};
static_assert(sizeof(MultiArgs) <= 32764, "kernel arguments are limited to 32,764 bytes");

// one tile of one process: every event of the block's groups, all points
template <class Proc, class R, int LB>
__device__ __forceinline__ void multi_tile(const MultiItem& a, const PointDev* pts, long long tile, double2* sacc,
                                           unsigned long long* sbad) {
  constexpr int NEXT = Proc::NEXT;
  constexpr int LANES = 1 << LB;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, wl = tid & 31;
  const int lane = tid & (LANES - 1);
  const unsigned gmask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << (wl & ~(LANES - 1)));
  const int P = a.P;
  const int stride = P + 1;
  const long long E = a.E;
  const long long ldo = a.ldo ? a.ldo : E;
  const long long ev = tile * (long long)(blockDim.x / LANES) + tid / LANES;
  const bool valid = ev < E;
  const long long evc = valid ? ev : E - 1;
  typename Proc::template mom_t<R> p[NEXT][4];
#pragma unroll
  for (int i = 0; i < NEXT; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) load_mom(p[i][m], __ldg(a.mom + ((long long)(i * 4 + m)) * a.ld + evc));
  const bool leader = valid && lane == 0;
  const double w = __ldg(a.w + evc);
  double me0 = 0.0;
  bool ok = false;
#pragma unroll 1
  for (int j = 0; j <= P; ++j) {
    const double me = eval_point<Proc, R, LB>(p, pts[a.pt0 + j], lane, gmask);
    if (j == 0) {
      me0 = me;
      ok = isfinite(me0) && me0 != 0.0;
      if (leader && !ok) atomicAdd(sbad, 1ull);
      if (leader && a.me0) a.me0[ev] = me0;
      warp_accumulate(sacc, warp, stride, P, leader ? w : 0.0);
      continue;
    }
    const double r = ok ? me / me0 : 0.0;
    const double wn = ok ? r * w : 0.0;
    if (leader) {
      const long long o = (long long)(j - 1) * ldo + ev;
      if (a.me_pts) a.me_pts[o] = me;
      if (a.ratio) a.ratio[o] = r;
      if (a.wnew) a.wnew[o] = wn;
    }
    warp_accumulate(sacc, warp, stride, j - 1, leader ? wn : 0.0);
  }
}

template <class R, class First, class... Rest>
__device__ __forceinline__ void multi_dispatch(int i, const MultiItem* items, const PointDev* pts, long long tile,
                                               double2* smem_sums, const int* off, unsigned long long* sbad) {
  if (i == 0) {
    multi_tile<typename First::Proc, R, First::LB>(items[0], pts, tile, smem_sums + off[0], sbad);
  } else {
    if constexpr (sizeof...(Rest) > 0)
      multi_dispatch<R, Rest...>(i - 1, items + 1, pts, tile, smem_sums, off + 1, sbad + 1);
  }
}

template <class First, class... Rest>
__host__ __device__ constexpr int max_jstore_bytes() {
  constexpr int a = First::Proc::template jstore_bytes<float, First::LB>();
  if constexpr (sizeof...(Rest) > 0) {
    constexpr int b = max_jstore_bytes<Rest...>();
    return a > b ? a : b;
  } else {
    return a;
  }
}

// R: the working precision of every item; Items: Lanes<Proc, LB>..., the
// process order the host fills MultiArgs in.
template <class R, class... Items>
__global__ void __launch_bounds__(256, 1) k_reweight_multi(const __grid_constant__ MultiArgs m) {
  constexpr int NI = sizeof...(Items);
  static_assert(NI >= 1 && NI <= MAX_MULTI, "1..MAX_MULTI processes");
  // dynamic shared memory: the largest amplitude current store (FP32), then
  // every item's warp sums
  extern __shared__ __align__(16) unsigned char rw_dyn_bytes[];
  constexpr int JS = sizeof(R) == 4 ? max_jstore_bytes<Items...>() : 0;
  double2* sums = reinterpret_cast<double2*>(rw_dyn_bytes + (size_t)JS * blockDim.x);
  __shared__ unsigned long long sbad[MAX_MULTI];
  __shared__ double2 red[32];
  __shared__ int is_last;
  const int tid = threadIdx.x;
  const int nw = blockDim.x >> 5;
  for (int i = tid; i < m.sacc_off[NI - 1] + nw * (m.item[NI - 1].P + 1); i += blockDim.x)
    sums[i] = make_double2(0.0, 0.0);
  if (tid < MAX_MULTI) sbad[tid] = 0ull;
  __syncthreads();
  const long long total = m.tile_end[NI - 1];
  int item = 0;
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    while (t >= m.tile_end[item]) ++item;  // tiles ascend, so the item index only grows
    const long long first = item ? m.tile_end[item - 1] : 0;
    multi_dispatch<R, Items...>(item, m.item, m.pool, t - first, sums, m.sacc_off, sbad);
  }
  __syncthreads();
  // block partials of every item, then the one ticket of the launch
  for (int i = 0; i < NI; ++i) {
    const MultiItem& a = m.item[i];
    const int stride = a.P + 1;
    const double2* sacc = sums + m.sacc_off[i];
    for (int j = tid; j < stride; j += blockDim.x) {
      double s = 0.0, c = 0.0;
      for (int wi = 0; wi < nw; ++wi) two_sum_acc(s, c, sacc[wi * stride + j].x, sacc[wi * stride + j].y);
      a.block_part[(long long)blockIdx.x * stride + j] = make_double2(s, c);
    }
    if (tid == 0 && sbad[i]) atomicAdd(a.nbad_count, sbad[i]);
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = atomicAdd(m.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int i = 0; i < NI; ++i) {
    const MultiItem& a = m.item[i];
    const int stride = a.P + 1;
    for (int j = 0; j < stride; ++j) {
      double s = 0.0, c = 0.0;
      for (int b = tid; b < (int)gridDim.x; b += blockDim.x) {
        const double2 v = __ldcg(a.block_part + (long long)b * stride + j);
        two_sum_acc(s, c, v.x, v.y);
      }
      block_sum2(s, c, red);
      if (tid == 0) {
        a.sigma[j] = s + c;
        if (a.sigma_pair) a.sigma_pair[j] = make_double2(s, c);
      }
    }
    if (tid == 0) *a.nbad_out = atomicExch(a.nbad_count, 0ull);
  }
  if (tid == 0) *m.ticket = 0u;
}

}  // namespace rw
