// The fused reweighting kernel (Sec. 3.2, steps 3-7, Eqs. 2-3 of
// arXiv:2312.07440), one launch for a whole event batch and every parameter
// point:
//   per event: load the FP64 momenta (structure of arrays, coalesced), |M|^2
//   under the original parameters, then for each point p: (mass-shell
//   reshuffle if the top mass changed) |M'_p|^2, r_p = |M'_p|^2/|M|^2 in FP64,
//   W'_p = r_p W; the cross sections sigma'_p = sum W'_p and sigma = sum W are
//   accumulated as compensated (TwoSum) pairs per warp and block and reduced
//   in a fixed order by the last block to finish, so the result is
//   deterministic for a given launch shape.
// Events violating |M|^2 != 0 (zero or non-finite) get r = W' = 0, are left
// out of sigma' and are counted.
//
// Threads: a group of 2^LB lanes shares one event; each lane sums its slice
// of the helicities and the slices are combined by xor shuffles inside the
// group.  The grid is at most (resident blocks x SMs) and strides over the
// events.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"
#include "helas.cuh"

namespace rw {

constexpr int MAX_POINTS = 256;

struct PointDev {
  double cscale;  // QCD: (4 pi alpha_s)^n / (spin/colour average x n_ident! x colour denominator)
  double m_t;     // top mass of this evaluation
  double e, gL, gR, MZ, WZ;  // electroweak couplings (e+e- -> mu+mu-)
  int reshuffle;  // 1: move the event onto the m_t mass shell first
  int pad;
};

struct RwArgs {
  const double* mom;  // [N][4][ld]
  const double* w;    // [E]
  long long E;
  long long ld;       // row stride of mom (>= E)
  double* me0;     // [E] or null
  double* me_pts;  // [P][E] or null
  double* ratio;   // [P][E] or null
  double* wnew;    // [P][E] or null
  double2* block_part;            // [gridDim.x][P+1] scratch
  double* sigma;                  // [P+1]: sigma'_0..P-1, sigma (original)
  unsigned int* ticket;           // zero between launches
  unsigned long long* nbad_count; // zero between launches
  unsigned long long* nbad_out;
  double2* sigma_acc;  // [P+1] (sum, compensation) carried across launches, or null
  double2* sigma_pair; // [P+1] each result's (sum, compensation) pair, or null
  long long ldo;       // row stride of the [P][.] outputs (0: E)
  int accumulate;      // 1: add this launch's sums and bad events to the previous launch's
  int P;
  int me_only;  // evaluate pt[0] only and write me0 (no reductions)
  unsigned char* defer;  // mixed modes with a separate colour pass: its amplitude buffers, or null
  long long defer_ld;    // rows per amplitude plane (events rounded up to 128)
  PointDev pt[MAX_POINTS + 1];  // [0] original, [1..P] modified points
};

// ---- compensated (TwoSum) accumulation -------------------------------------
__device__ __forceinline__ void two_sum_acc(double& s, double& c, double x, double cx) {
  const double t = s + x;
  const double bp = t - s;
  const double e = (s - (t - bp)) + (x - bp);
  s = t;
  c += cx + e;
}

__device__ __forceinline__ void warp_sum2(double& s, double& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const double c2 = __shfl_xor_sync(0xffffffffu, c, o);
    two_sum_acc(s, c, s2, c2);
  }
}

// lane 0 of the warp adds the warp total of x into slot (warp, j)
__device__ __forceinline__ void warp_accumulate(double2* sacc, int warp, int stride, int j, double x) {
  __syncwarp();
  double s = x, c = 0.0;
  warp_sum2(s, c);
  if ((threadIdx.x & 31) == 0) {
    double2 v = sacc[warp * stride + j];
    two_sum_acc(v.x, v.y, s, c);
    sacc[warp * stride + j] = v;
  }
}

// deterministic block reduction of (s, c); result valid in thread 0
__device__ __forceinline__ void block_sum2(double& s, double& c, double2* scratch) {
  warp_sum2(s, c);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) scratch[warp] = make_double2(s, c);
  __syncthreads();
  if (threadIdx.x == 0) {
    double ss = 0.0, cc = 0.0;
    for (int i = 0; i < nw; ++i) two_sum_acc(ss, cc, scratch[i].x, scratch[i].y);
    s = ss;
    c = cc;
  }
  __syncthreads();
}

// |M|^2 for one parameter point; a point with a new top mass first moves the
// event onto its mass shell (|M'|^2 = 0 when the new masses do not fit).
// FP64 input momenta to the process's momentum type: FP64 as is, or the
// double-float split done with integer operations (no FP64-pipe conversion).
__device__ __forceinline__ void load_mom(double& dst, double x) { dst = x; }
__device__ __forceinline__ void load_mom(df& dst, double x) { dst = df_from_double(x); }

template <class Proc, class R, int LB>
__device__ __forceinline__ double eval_point(const typename Proc::template mom_t<R> (&p)[Proc::NEXT][4],
                                             const PointDev& pt, int lane, unsigned gmask) {
  typename Proc::template mom_t<R> q[Proc::NEXT][4];
  bool inside = true;
  if (pt.reshuffle) {
    inside = Proc::template reshuffle<R>(p, pt.m_t, q);
  } else {
#pragma unroll
    for (int i = 0; i < Proc::NEXT; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) q[i][m] = p[i][m];
  }
  double v;
  if constexpr (Proc::template inline_me<R>())
    v = Proc::template me_body<R, LB>(q, pt, lane, gmask);
  else
    v = Proc::template me<R, LB>(q, pt, lane, gmask);
  return inside ? v : 0.0;
}

// MINB: resident blocks of 256 threads per SM the register allocation must
// allow (1: up to 255 registers; 2: 128, for small processes whose FP32
// kernels are latency-bound at 8 warps per SM).
template <class Proc, class R, int LB, int MINB = 1>
__global__ void __launch_bounds__(256, MINB) k_reweight(const __grid_constant__ RwArgs a) {
  constexpr int NEXT = Proc::NEXT;
  constexpr int LANES = 1 << LB;
  // dynamic shared memory: the amplitude code's current store (if any), then
  // the warp partial sums [nwarps][P+1]
  extern __shared__ __align__(16) unsigned char rw_dyn_bytes[];
  double2* sacc = reinterpret_cast<double2*>(rw_dyn_bytes + (size_t)Proc::template jstore_bytes<R, LB>() * blockDim.x);
  __shared__ double2 red[32];
  __shared__ int is_last;
  const int P = a.P;
  const int stride = P + 1;
  const int tid = threadIdx.x;
  const int nw = blockDim.x >> 5;
  const int warp = tid >> 5, wl = tid & 31;
  const int lane = tid & (LANES - 1);
  const unsigned gmask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << (wl & ~(LANES - 1)));
  if (!a.me_only)
    for (int i = tid; i < nw * stride; i += blockDim.x) sacc[i] = make_double2(0.0, 0.0);
  __syncthreads();
  const long long gpb = blockDim.x / LANES;
  const long long ngroups = (long long)gridDim.x * gpb;
  const long long g0 = (long long)blockIdx.x * gpb + tid / LANES;
  const long long E = a.E;
  const long long ldo = a.ldo ? a.ldo : a.E;
  unsigned long long nbad = 0;
  // Up to FEW points: per-thread compensated accumulators for the cross
  // sections (slot P = sigma of the original weights), reduced once at the end;
  // more points: a warp reduction per event into shared memory.
  constexpr int FEW = 3;
  const bool few = P <= FEW;
  double rs[FEW + 1], rc[FEW + 1];
#pragma unroll
  for (int q = 0; q <= FEW; ++q) rs[q] = rc[q] = 0.0;
  for (long long base = 0; base < E; base += ngroups) {
    const long long ev = base + g0;
    const bool valid = ev < E;
    const long long evc = valid ? ev : E - 1;
    typename Proc::template mom_t<R> p[NEXT][4];
#pragma unroll
    for (int i = 0; i < NEXT; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) load_mom(p[i][m], __ldg(a.mom + ((long long)(i * 4 + m)) * a.ld + evc));
    // One call site for every evaluation (original, then each point), so that
    // identical parameters give bitwise identical |M|^2 and r == 1 exactly.
    const bool leader = valid && lane == 0;
    const double w = __ldg(a.w + evc);
    double me0 = 0.0;
    bool ok = false;
    const int nev = a.me_only ? 1 : P + 1;
#pragma unroll 1
    for (int j = 0; j < nev; ++j) {
      const double me = eval_point<Proc, R, LB>(p, a.pt[j], lane, gmask);
      if (j == 0) {
        me0 = me;
        if (a.me_only) {
          if (leader) a.me0[ev] = me;
          break;
        }
        ok = isfinite(me0) && me0 != 0.0;
        if (leader && !ok) ++nbad;
        if (leader && a.me0) a.me0[ev] = me0;
        if (few) {
          if (leader) {
#pragma unroll
            for (int q = 0; q <= FEW; ++q)
              if (q == P) two_sum_acc(rs[q], rc[q], w, 0.0);
          }
        } else {
          warp_accumulate(sacc, warp, stride, P, leader ? w : 0.0);
        }
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
      if (few) {
        if (leader) {
#pragma unroll
          for (int q = 0; q < FEW; ++q)
            if (q == j - 1) two_sum_acc(rs[q], rc[q], wn, 0.0);
        }
      } else {
        warp_accumulate(sacc, warp, stride, j - 1, leader ? wn : 0.0);
      }
    }
  }
  if (a.me_only) return;
  if (few) {  // one warp reduction per slot for the whole launch
#pragma unroll
    for (int q = 0; q <= FEW; ++q) {
      if (q > P) break;
      double s = rs[q], c = rc[q];
      __syncwarp();
      warp_sum2(s, c);
      if (wl == 0) sacc[warp * stride + q] = make_double2(s, c);
    }
  }
  __syncthreads();
  for (int j = tid; j < stride; j += blockDim.x) {
    double s = 0.0, c = 0.0;
    for (int wi = 0; wi < nw; ++wi) two_sum_acc(s, c, sacc[wi * stride + j].x, sacc[wi * stride + j].y);
    a.block_part[(long long)blockIdx.x * stride + j] = make_double2(s, c);
  }
  if (nbad) atomicAdd(a.nbad_count, nbad);
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int j = 0; j < stride; ++j) {
    double s = 0.0, c = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += blockDim.x) {
      const double2 v = __ldcg(a.block_part + (long long)b * stride + j);
      two_sum_acc(s, c, v.x, v.y);
    }
    block_sum2(s, c, red);
    if (tid == 0) {
      if (a.sigma_acc) {  // chunked launches: carry (sum, compensation) in launch order
        double2 t = a.accumulate ? a.sigma_acc[j] : make_double2(0.0, 0.0);
        two_sum_acc(t.x, t.y, s, c);
        a.sigma_acc[j] = t;
        a.sigma[j] = t.x + t.y;
        if (a.sigma_pair) a.sigma_pair[j] = t;
      } else {
        a.sigma[j] = s + c;
        if (a.sigma_pair) a.sigma_pair[j] = make_double2(s, c);
      }
    }
  }
  if (tid == 0) {
    const unsigned long long nb = atomicExch(a.nbad_count, 0ull);
    *a.nbad_out = a.accumulate ? *a.nbad_out + nb : nb;
    *a.ticket = 0u;
  }
}

// ---------------------------------------------------------------------------
// Interpolation surrogate for many points on one parameter axis v (m_t,
// alpha_s, alpha, M_Z, ...): per event, |M|^2 exactly at the original point
// and at K Chebyshev nodes v_k = (a+b)/2 + (b-a)/2 x_k, x_k = cos(pi (k+1/2)/K),
// of the points' range [a, b]; y_k = log(|M(v_k)|^2/|M|^2) is interpolated by
// p(x) = sum_{i<K} c_i T_i(x), c = cheb . y, and log r at every point read off
// p.  log r is analytic in v on [a, b] for these processes, so the Chebyshev
// coefficients decay geometrically and |c_{K-1}| + |c_{K-2}| estimates the
// interpolation error.  Events whose estimate exceeds tol (or with a
// non-positive or non-finite node value) are listed for the exact path;
// events with |M|^2 == 0 or non-finite get W' = 0 and are counted as bad.
// ---------------------------------------------------------------------------
constexpr int MAX_NODES = 16;

struct InterpArgs {
  const double* mom;  // [N][4][ld]
  const double* w;    // [E]
  long long E, ld;
  double* wnew;                 // [P][E]; rows of listed events are left for the exact path
  unsigned char* flag;          // [E]: 1 listed for the exact path, or null
  unsigned long long* counts;   // [0] listed events, [1] bad events
  long long* list;              // [E] listed event indices
  int P, K;
  double tol;
  PointDev pt0;
  PointDev node[MAX_NODES];
  double cheb[MAX_NODES][MAX_NODES];  // c_i = sum_k cheb[i][k] y_k; zero for i or k >= K
  double x[MAX_POINTS];               // the points' abscissae in [-1, 1]
};

template <class Proc, class R, int LB, int MINB = 1>
__global__ void __launch_bounds__(256, MINB) k_interp(const __grid_constant__ InterpArgs a) {
  constexpr int NEXT = Proc::NEXT;
  constexpr int LANES = 1 << LB;
  const int tid = threadIdx.x;
  const int wl = tid & 31;
  const int lane = tid & (LANES - 1);
  const unsigned gmask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << (wl & ~(LANES - 1)));
  const long long gpb = blockDim.x / LANES;
  const long long ngroups = (long long)gridDim.x * gpb;
  const long long g0 = (long long)blockIdx.x * gpb + tid / LANES;
  const long long E = a.E;
  for (long long base = 0; base < E; base += ngroups) {
    const long long ev = base + g0;
    const bool valid = ev < E;
    const long long evc = valid ? ev : E - 1;
    typename Proc::template mom_t<R> p[NEXT][4];
#pragma unroll
    for (int i = 0; i < NEXT; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) load_mom(p[i][m], __ldg(a.mom + ((long long)(i * 4 + m)) * a.ld + evc));
    const double me0 = eval_point<Proc, R, LB>(p, a.pt0, lane, gmask);
    const bool ok = isfinite(me0) && me0 != 0.0;
    R y[MAX_NODES];
    bool good = ok;
#pragma unroll 1
    for (int k = 0; k < a.K; ++k) {
      const double t = eval_point<Proc, R, LB>(p, a.node[k], lane, gmask) / me0;
      good = good && isfinite(t) && t > 0.0;
      y[k] = good ? R(log(R(t))) : R(0);
    }
    if (!valid || lane != 0) continue;
    if (!ok) {
      atomicAdd(a.counts + 1, 1ull);
      if (a.flag) a.flag[ev] = 0;
      for (int j = 0; j < a.P; ++j) a.wnew[(long long)j * E + ev] = 0.0;
      continue;
    }
    // fixed-size register arrays (cheb is zero beyond K, so the padded
    // coefficients vanish and the 16-term Clenshaw sum equals the K-term one)
    R yr[MAX_NODES], c[MAX_NODES];
#pragma unroll
    for (int k = 0; k < MAX_NODES; ++k) yr[k] = k < a.K ? y[k] : R(0);
    double est = 0.0;
#pragma unroll
    for (int i = 0; i < MAX_NODES; ++i) {
      R s = R(0);
#pragma unroll
      for (int k = 0; k < MAX_NODES; ++k) s = fmadd(R(a.cheb[i][k]), yr[k], s);
      c[i] = s;
      if (i == a.K - 1 || i == a.K - 2) est += fabs((double)s);
    }
    if (!(good && est <= a.tol)) {
      if (a.flag) a.flag[ev] = 1;
      a.list[atomicAdd(a.counts, 1ull)] = ev;
      continue;
    }
    if (a.flag) a.flag[ev] = 0;
    const double w = __ldg(a.w + ev);
    for (int j = 0; j < a.P; ++j) {
      // Clenshaw: p(x) = sum_i c_i T_i(x)
      const R x = R(a.x[j]), x2 = R(2) * x;
      R b1 = R(0), b2 = R(0);
#pragma unroll
      for (int i = MAX_NODES - 1; i >= 1; --i) {
        const R b0 = fmadd(x2, b1, c[i] - b2);
        b2 = b1;
        b1 = b0;
      }
      const R lr = fmadd(x, b1, c[0] - b2);
      a.wnew[(long long)j * E + ev] = (double)exp(lr) * w;
    }
  }
}

}  // namespace rw
