/*
 * rwgt.h -- C ABI of librwgt.so: leading-order event reweighting on one GPU.
 *
 * The library follows the reweighting procedure of arXiv:2312.07440,
 * Sec. 3.2 ("Parallel LO scattering amplitudes and reweighting"):
 *   1) input reweight parameters          -> rw_set_params, rw_set_reweight_points
 *   2) parse events                        -> rw_load_events (device arrays)
 *   3) evaluate original |M|^2             -> rw_eval_me(point = -1), or fused in rw_reweight*
 *   4) overwrite physics parameters        -> the parameter points
 *   5) evaluate new |M'|^2                 -> rw_eval_me(point = p), or fused
 *   6) new weight W' = |M'|^2/|M|^2 W      (Sec. 2.2, Eq. 3)
 *   7) repeat 4-6 for all parameter sets   (all points in one launch)
 *   8) return new weights                  -> W'[P][E] and sigma'_p = sum_k W'_pk (Sec. 2.1, Eq. 2)
 * The validity condition of Eq. 3 (|M|^2 != 0, Sec. 2.2) is reported, not
 * fatal: an event with |M|^2 == 0 or non-finite gets r = W' = 0, is left out
 * of sigma' and is counted; the call then returns RW_WARN_BAD_EVENTS.
 *
 * |M|^2 is the tree-level squared matrix element averaged over initial spins
 * and colours and summed over final ones (1/n! for n identical outgoing
 * gluons).  Processes: e+e- -> mu+mu- (photon + Z), g g -> t tbar,
 * g g -> t tbar g, g g -> t tbar g g.
 *
 * Conventions
 *  - Momenta: float64, structure of arrays mom[N][4][E] (particle, component
 *    (E, px, py, pz), event), in GeV, partonic centre-of-mass frame, incoming
 *    partons first.  Particle order: e-, e+, mu-, mu+  |  g, g, t, tbar, g, g.
 *  - Weights: float64 w[E].  Outputs W'[P][E], r[P][E], |M|^2 [E] float64.
 *  - A top-mass change moves each event onto the new mass shell (outgoing
 *    3-momenta scaled by a common factor at fixed partonic energy) before
 *    |M'|^2 is evaluated; an event the new masses do not fit gets |M'|^2 = 0.
 *  - Ownership: the caller owns every event, output and workspace buffer
 *    (device memory unless the name says h_); the context owns only itself
 *    and a small pinned staging buffer.  Pointers passed to rw_load_events
 *    must stay valid until the next rw_load_events or rw_destroy.
 *  - Asynchrony: work is queued on the context's stream; only calls with
 *    h_ outputs (and rw_reweight_host) synchronise that stream.
 *  - Errors: every call returns RW_OK (0), a warning (> 0) or an error (< 0);
 *    rw_last_error() describes the last failure.  A context is not
 *    thread-safe; separate contexts are independent.
 */
#ifndef RWGT_H
#define RWGT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RW_OK 0
#define RW_WARN_BAD_EVENTS 1    /* some events had |M|^2 == 0 or non-finite */
#define RW_ERR_NULL (-1)        /* a required pointer is NULL */
#define RW_ERR_ARG (-2)         /* bad size, count or index */
#define RW_ERR_MODE (-3)        /* process/precision combination not available */
#define RW_ERR_PARAM (-4)       /* non-finite or unphysical model parameter */
#define RW_ERR_CUDA (-5)        /* a CUDA runtime call failed (message in rw_last_error) */
#define RW_ERR_STATE (-6)       /* call out of order (e.g. no process or events set) */
#define RW_ERR_ALIGN (-7)       /* buffer not 8-byte (16-byte for workspace) aligned */
#define RW_ERR_WORKSPACE (-8)   /* workspace smaller than rw_workspace_bytes() */

/* processes */
#define RW_EE_MUMU 0   /* e- e+ -> mu- mu+, 2 diagrams, 16 helicities */
#define RW_GG_TT 1     /* g g -> t tbar, 3 diagrams, 2 colour orderings */
#define RW_GG_TTG 2    /* g g -> t tbar g, 16 diagrams, 6 orderings */
#define RW_GG_TTGG 3   /* g g -> t tbar g g, 123 diagrams, 24 orderings */
#define RW_EE_5A 4     /* e- e+ -> 5 photons (the paper's benchmark process, Table 1): pure QED,
                          massless electrons, 120 diagrams, 128 helicities; FP64 and FP32 modes */

/* precision modes of the amplitude arithmetic; momenta, propagator
   invariants, r, W' and sigma are FP64 in every mode */
#define RW_FP64 0       /* FP64 amplitudes and colour sum */
#define RW_FP32 1       /* FP32 amplitudes and colour sum */
#define RW_MIXED_FP16 2 /* FP32 amplitudes, colour sum on the tensor cores in FP16 (power-of-two
                           scaled rows) with FP32 accumulation; QCD processes */
#define RW_MIXED_BF16 3 /* as RW_MIXED_FP16 with BF16 operands */

#define RW_MAX_POINTS 256

/* Model parameters (Sec. 3.2 step 1).  QCD processes use alpha_s and m_t
   (w_t must be 0: every top propagator here is off shell; yt_scale, the top
   Yukawa scale, enters no tree diagram of these processes).  e+e- -> mu+mu-
   uses alpha_em_inv = 1/alpha, G_F [GeV^-2], m_Z, w_Z [GeV]; M_W and s_W are
   derived: M_W^2 = M_Z^2/2 + sqrt(M_Z^4/4 - pi alpha M_Z^2/(sqrt2 G_F)).
   e+e- -> 5 photons uses alpha_em_inv only (e = sqrt(4 pi / alpha_em_inv)). */
typedef struct rw_params {
  double alpha_s, m_t, w_t, yt_scale;
  double alpha_em_inv, G_F, m_Z, w_Z;
} rw_params;

/* static description of a process (for flop accounting and checks) */
typedef struct rw_process_info {
  int n_external;      /* external particles N */
  int n_helicities;    /* 2^N */
  int n_colour_flows;  /* K: colour orderings (1 for e+e- -> mu+mu-) */
  int n_diagrams;      /* tree Feynman diagrams */
  int colour_den;      /* C = C_int / colour_den */
  long long flops_hel_sum; /* amplitude + colour-sum flops of one helicity-summed |M|^2 */
} rw_process_info;

typedef struct rw_ctx rw_ctx;

/* Create a context on CUDA device `device`, queuing work on `cuda_stream`
   (a cudaStream_t; NULL = the legacy default stream).  *ctx is NULL on error. */
int rw_create(rw_ctx** ctx, int device, void* cuda_stream);
int rw_destroy(rw_ctx* ctx);
/* description of the last error on this context (owned by the context) */
const char* rw_last_error(const rw_ctx* ctx);

int rw_process_info_get(int process, rw_process_info* out);

/* Select process and precision mode.  Resets parameters and events. */
int rw_set_process(rw_ctx* ctx, int process, int mode);
/* Step 1: the original parameters of the event sample. */
int rw_set_params(rw_ctx* ctx, const rw_params* orig);
/* Steps 4/7: P modified parameter points (1 <= P <= RW_MAX_POINTS). */
int rw_set_reweight_points(rw_ctx* ctx, const rw_params* pts, int P);
/* Launch shape: lanes per event = 2^lane_bits (-1 = default), threads per
   block (multiple of 32, <= 256; 0 = default). */
int rw_set_tuning(rw_ctx* ctx, int lane_bits, int block);

/* The launch shape in use (after rw_set_tuning or rw_autotune). */
int rw_get_tuning(const rw_ctx* ctx, int* lane_bits, int* block);
/* Autotuner: times every compiled lanes-per-event variant x block size in
   {64, 128, 256} on the first min(E, max_events) attached events (CUDA events
   on the context's stream, median of 3 launches after one warm-up), keeps the
   fastest with rw_set_tuning and returns its time per launch in *ms (may be
   NULL).  Events must be loaded.  cache_path (may be NULL): a JSON-lines file of
   {"key": "<gpu>|<process>|<mode>|P<points>|E<2^k>", "lane_bits", "block", "ms"};
   a matching entry is used without timing, a new result is appended.
   Synchronises the stream; results are unchanged by the choice (every variant
   computes the same sums; the sigma reduction order follows the grid). */
int rw_autotune(rw_ctx* ctx, int64_t max_events, const char* cache_path, double* ms);

/* Device workspace needed for E events with the current points (bytes).  In
   the mixed modes of g g -> t tbar g g with at most 3 points it includes the
   separate colour pass's amplitude buffers, (P+1) x 32 x 98 + (P+1) bytes per
   event (Sec. 3.1's colour sum done as its own tensor-core pass); with a
   smaller workspace those modes sum colours inside the amplitude kernel. */
size_t rw_workspace_bytes(const rw_ctx* ctx, int64_t n_events);
/* Step 2: attach a device event batch (SoA momenta [N][4][E], weights [E])
   and a device workspace, 16-byte aligned, of rw_workspace_bytes(E) bytes:
   the reduction slots for the current points are required (RW_ERR_WORKSPACE
   below them); the separate colour pass's buffers that the mixed modes of
   g g -> t tbar g g use beyond them are optional (without them those modes
   sum colours inside the amplitude kernel).  Clears the workspace counters
   (asynchronously). */
int rw_load_events(rw_ctx* ctx, const double* d_mom, const double* d_w, int64_t n_events, void* d_workspace,
                   size_t workspace_bytes);

/* Steps 3/5: |M|^2 of every event under the original parameters
   (point = -1) or under point p (momenta moved to its mass shell if m_t
   differs).  d_me_out: device [E]. */
int rw_eval_me(rw_ctx* ctx, int point, double* d_me_out);

/* Steps 3-7 fused, no host synchronisation: W'[P][E], r[P][E], |M|^2 [E]
   and |M'|^2 [P][E] are written where the pointer is not NULL; sigma'_p,
   sigma and the bad-event count stay in the workspace (rw_get_results). */
int rw_reweight_async(rw_ctx* ctx, double* d_wnew, double* d_ratio, double* d_me0, double* d_me_pts);
/* Copy the last reweight's sigma'_p [P], sigma (original) and bad-event count
   to the host; synchronises the stream.  Returns RW_WARN_BAD_EVENTS if any. */
int rw_get_results(rw_ctx* ctx, double* h_sigma, double* h_sigma_orig, int64_t* h_n_bad);
/* The same results as (sum, compensation) pairs before they are added:
   h_sum[j] + h_comp[j] is sigma'_j for j < P and sigma for j = P (arrays of
   P+1 doubles, both required).  For merging partial cross sections of event
   shards (Eq. 2 over all shards) without losing the compensation term.
   Synchronises the stream.  Returns RW_WARN_BAD_EVENTS if any. */
int rw_get_result_pairs(rw_ctx* ctx, double* h_sum, double* h_comp, int64_t* h_n_bad);
/* rw_reweight_async + rw_get_results. */
int rw_reweight(rw_ctx* ctx, double* d_wnew, double* d_ratio, double* h_sigma, double* h_sigma_orig,
                int64_t* h_n_bad);

/* End to end from host memory: copies momenta [N][4][E] and weights [E] to
   the device workspace, reweights, copies W'[P][E] back to h_wnew (may be
   NULL) and the sums to h_sigma/h_sigma_orig/h_n_bad; synchronises.  The
   device workspace must hold rw_workspace_bytes_host(E) bytes.  Host buffers
   should be pinned (cudaHostAlloc) for full copy bandwidth.  Large batches are
   pipelined: chunks of about E/8 events (a multiple of the threads one launch
   keeps resident) are copied in on a second stream the context creates on
   first use, and the reweight of chunk k starts as soon as its copy is in,
   overlapping the copies of the later chunks; W' of chunk k is copied out
   while chunk k+1 is reweighted.  The sums are carried across chunks in
   compensated form, in chunk order, so results stay deterministic.  The work starts after what is
   already queued on the context's stream and the call returns with all of
   it done. */
size_t rw_workspace_bytes_host(const rw_ctx* ctx, int64_t n_events);
int rw_reweight_host(rw_ctx* ctx, const double* h_mom, const double* h_w, int64_t n_events, double* h_wnew,
                     double* h_sigma, double* h_sigma_orig, int64_t* h_n_bad, void* d_workspace,
                     size_t workspace_bytes);

/* ---------------------------------------------------------------------------
   CUDA-graph batching: record rw_reweight_async / rw_eval_me calls of any
   number of contexts (processes, modes, point sets) that queue on one stream
   between rw_graph_begin and rw_graph_end, then replay them all with one
   rw_graph_launch.  Each replay recomputes every recorded reweight from the
   events and outputs bound at capture time (the kernels reset their own
   counters, so replays are independent).  Do not call functions that
   synchronise (rw_get_results, rw_autotune, ...) while capturing, and run
   rw_autotune (if used) before capturing. */
typedef struct rw_graph rw_graph;
int rw_graph_begin(void* cuda_stream);
int rw_graph_end(void* cuda_stream, rw_graph** graph);
int rw_graph_launch(rw_graph* graph, void* cuda_stream);
int rw_graph_destroy(rw_graph* graph);

/* ---------------------------------------------------------------------------
   Several processes in one persistent launch (Sec. 3.2 steps 3-7 for every
   process of a sample at once; Sec. 4: the real-emission events of an NLO
   sample are tree-level events of one more parton, reweighted by the same LO
   machinery).  Each process is a context with its process, mode, parameters,
   points, events and workspace set as for rw_reweight_async; one kernel walks
   tiles of all of their events grid-stride, so a cheap process fills the gaps
   a costly one leaves.  Per process: W'[P_i][E_i] and r[P_i][E_i] where the
   pointers given to rw_multi_add are not NULL, and its sigma'_p, sigma and
   bad-event count in its own workspace (rw_get_results(ctx) after the launch).
   Compiled process sets, each in one precision mode for all of its processes:
     {g g -> t tbar g, g g -> t tbar}                 RW_FP64, RW_FP32
     {g g -> t tbar g g, g g -> t tbar g, g g -> t tbar} RW_FP64
   (any other set or mode: RW_ERR_MODE at launch).  At most 420 parameter
   points in total over the processes, one original point counted per
   process (RW_ERR_ARG).  Threads per block: 128.  The launch is asynchronous
   on the stream given to rw_multi_create, which must order the launch after
   the work queued for the contexts' events.  Results are deterministic for a
   given set of contexts.  Not thread-safe; contexts must outlive the
   rw_multi that holds them. */
typedef struct rw_multi rw_multi;
int rw_multi_create(rw_multi** m, int device, void* cuda_stream);
int rw_multi_destroy(rw_multi* m);
const char* rw_multi_last_error(const rw_multi* m);
/* add a prepared context (RW_ERR_STATE when its events or points are
   missing, RW_ERR_MODE when its mode differs from those already added,
   RW_ERR_ARG for a second context of the same process or a fifth process) */
int rw_multi_add(rw_multi* m, rw_ctx* ctx, double* d_wnew, double* d_ratio);
/* device workspace of the launch itself (its ticket), 16-byte aligned */
size_t rw_multi_workspace_bytes(const rw_multi* m);
int rw_multi_reweight_async(rw_multi* m, void* d_workspace, size_t workspace_bytes);
/* the sample's totals: sigma'_p = sum over processes of each process's
   sigma'_p (P must be the same for every process, else RW_ERR_STATE),
   sigma and the bad-event count, merged from the (sum, compensation) pairs
   in the order the processes were added; synchronises the contexts' streams */
int rw_multi_get_results(rw_multi* m, double* h_sigma, double* h_sigma_orig, int64_t* h_n_bad);

/* ---------------------------------------------------------------------------
   Learned surrogate for log r (spec extension; the paper has none).
   An MLP n_in -> [hidden, SiLU] x n_layers -> 2 predicts mu = log r and
   s = log of its own error for a feature vector built from an event and a
   parameter point; BF16 weights/activations, FP32 accumulation on the tensor
   cores, FP32 master weights and Adam.  The object owns its device memory
   (parameters, optimiser state, activations for max_batch rows).
   Parameter vector layout: for each linear layer l = 0..n_layers,
   W_l [in_l][out_l] row-major then b_l [out_l]. */
typedef struct rw_mlp rw_mlp;
int rw_mlp_create(rw_mlp** m, int device, void* cuda_stream, int n_in, int hidden, int n_layers, int max_batch,
                  uint64_t seed);
int rw_mlp_destroy(rw_mlp* m);
const char* rw_mlp_last_error(const rw_mlp* m);
int64_t rw_mlp_n_params(const rw_mlp* m);
/* shape and stream the model was created with (pointers may be NULL) */
int rw_mlp_info(const rw_mlp* m, int* n_in, int* hidden, int* n_layers, void** cuda_stream);
/* checkpoint / resume: FP32 parameters, Adam moments (may be NULL) and step */
int rw_mlp_get_state(rw_mlp* m, float* h_params, float* h_m1, float* h_m2, int64_t* h_step);
int rw_mlp_set_state(rw_mlp* m, const float* h_params, const float* h_m1, const float* h_m2, int64_t step);
/* out [n][2] = (mu, s) for features x [n][n_in] (device, FP32).  With GEMM
   kind 0, hidden = 256, n_in <= 40 and n_layers <= 8 the whole network runs
   in one persistent tensor-core kernel for all n rows (activations stay in
   shared memory; the input layer as one BF16 MMA over the split operands
   [x_h | x_l | x_h] . [W_h ; W_h ; W_l], i.e. FP32 up to ~2^-16 relative; the
   last activation is not rounded to BF16), else max_batch rows at a time. */
int rw_mlp_forward(rw_mlp* m, const float* d_x, int64_t n, float* d_out);
/* loss and its gradient at the current parameters for n <= max_batch rows
   (no update): loss = mean ((y-mu)/tau)^2 + lam (r^2 e^{-2s}/2 + s), r = y - mu
   held constant in the second term; h_grad [n_params] may be NULL. Synchronises. */
int rw_mlp_gradient(rw_mlp* m, const float* d_x, const float* d_y, int64_t n, float tau, float lam, float* h_grad,
                    float* h_loss);
/* n_steps Adam steps on minibatches of `batch` rows drawn with a counter-based
   generator from (seed, step) out of x [n][n_in], y [n]; asynchronous. */
int rw_mlp_train(rw_mlp* m, const float* d_x, const float* d_y, int64_t n, int batch, int64_t n_steps, float lr,
                 float tau, float lam, uint64_t seed);

/* Forward GEMMs of the hidden layers (training and inference): kind 0 (the
   default) runs them on the 5th-generation tensor cores -- tcgen05.mma fed by
   TMA, FP32 accumulators in tensor memory, bias + SiLU fused into the
   epilogue and, in rw_mlp_forward, the output layer fused into the last
   hidden layer -- whenever hidden is a multiple of 64 and at most 256, and
   inference of the whole network in one kernel where rw_mlp_forward allows;
   kind 2 is kind 0 with inference layer by layer (FP32 input layer); kind 1
   uses the mma.sync kernel for every layer.  The hidden layers compute the
   same products of the same BF16 operands in FP32 on every path. */
int rw_mlp_set_gemm(rw_mlp* m, int kind);
/* Synchronise the model's stream and report a tensor-core pipeline wait that
   gave up (RW_ERR_CUDA; the kernel then stops early and its results are
   invalid), else RW_OK. */
int rw_mlp_status(rw_mlp* m);
/* One hidden layer l (1 <= l < n_layers) on the current GEMM path, for tests
   and benchmarks: d_z [n][hidden] (FP32) = d_h_in [n][hidden] (BF16) W_l + b_l,
   d_h_out [n][hidden] (BF16) = SiLU(d_z) rounded; device buffers, 16-byte
   aligned; asynchronous on the model's stream. */
int rw_mlp_hidden_layer(rw_mlp* m, int layer, const void* d_h_in, int64_t n, float* d_z, void* d_h_out);

/* Surrogate features of the attached events for every point p, row p*E + e:
   x = (p_i^mu / p_scale for all N particles after the rotation about the beam
   axis that puts the top's p_T along +x, (kappa_p - 1)/k_scale, then -- when
   n_in leaves room for them -- the logarithms of the N(N-1)/2 pairwise
   invariants, log(2 p_i.p_j / s-hat), zero padding) [n_in],
   kappa_p = m_t(point p) / m_t(original); and, when d_ratio [P][E] is not NULL,
   labels y [P*E] = log r / (kappa_p - 1) (0 where r <= 0 or kappa_p = 1): the
   network's mu predicts log r per unit shift and s the log of its error in
   log r per unit shift.  Device buffers. */
int rw_surrogate_features(rw_ctx* ctx, int n_in, double p_scale, double k_scale, const double* d_ratio, float* d_x,
                          float* d_y);
/* Surrogate reweighting of the attached events for every point (Sec. 3.2
   steps 5-7 with the MLP in place of |M'|^2/|M|^2): r = exp((kappa-1) mu);
   where the predicted log error of log r, s + log|kappa - 1|, exceeds s_max
   the event is recomputed by the exact fused kernel (its W' there is the exact
   path's, bit for bit): with P <= 6 points the events are grouped by the set
   of points they need and each group is one exact launch at just those
   points; with more points an event over the bound at any point is
   recomputed at every point.  W'[P][E], optional fallback flags [P][E]
   (1 = exact), sigma'_p (h_sigma [P]) and the fallback counts (h_n_fallback
   [P]: events recomputed at point p).  The model must be created on the
   context's stream with the width n_in used here.  Device workspace of
   rw_surrogate_workspace_bytes(ctx, n_in); synchronises. */
size_t rw_surrogate_workspace_bytes(const rw_ctx* ctx, int n_in);
int rw_surrogate_reweight(rw_ctx* ctx, rw_mlp* m, double p_scale, double k_scale, double s_max, double* d_wnew,
                          unsigned char* d_fallback, double* h_sigma, int64_t* h_n_fallback, void* d_workspace,
                          size_t workspace_bytes);

/* ---------------------------------------------------------------------------
   Allocation-free variant of rw_reweight_async.  The paper has no counterpart:
   it exists for callers that cannot allocate device memory -- code that runs
   inside a host framework owning the whole device memory budget up front
   (online/trigger-style services, plug-ins hooked into an event generator),
   or in a latency-critical loop where cudaMalloc's implicit device
   synchronisation is not acceptable.  The caller passes inputs and outputs
   only; the reduction scratch lives in a fixed array of RW_NOALLOC_SCRATCH_BYTES
   bytes in this library's device memory, which every GPU that loads the
   library holds until the process exits.
     d_mom [N][4][E], d_w [E]      device inputs (as rw_load_events)
     d_wnew [P][E], d_ratio [P][E] device outputs, may be NULL
     d_sigma [P+1]                 device output: sigma'_0..P-1, then sigma
     d_n_bad [1]                   device output: events with |M|^2 == 0/non-finite
   Process, mode, parameters and at most RW_NOALLOC_MAX_POINTS points come from
   the context (set beforehand).  No cudaMalloc/cudaFree or other allocation
   happens in the call; it returns without synchronising the stream.
   The first call on a device looks up the array's device address (once per
   device, with that device current); make that first call before any stream
   capture.  All calls share the one array and each call overwrites it: calls
   whose kernels overlap on the GPU (e.g. two streams at once) race and must
   be serialised by the caller.  More points than the maximum -> RW_ERR_ARG;
   error texts of this call are short (at most 15 characters). */
#define RW_NOALLOC_MAX_POINTS 16
#define RW_NOALLOC_SCRATCH_BYTES (256 + 2048 * (RW_NOALLOC_MAX_POINTS + 1) * 16)
int rw_reweight_noalloc(rw_ctx* ctx, const double* d_mom, const double* d_w, int64_t n_events, double* d_wnew,
                        double* d_ratio, double* d_sigma, unsigned long long* d_n_bad);

/* ---------------------------------------------------------------------------
   Interpolation surrogate for many points on one parameter axis (the paper
   has no counterpart; it is the second surrogate of the library, beside the
   learned one above).  The points must differ from the original parameters
   in one field only (m_t, alpha_s, alpha_em_inv, m_Z, ...), the same field
   for all.  Per event the kernel evaluates |M|^2 exactly at the original
   point and at n_nodes Chebyshev nodes of the points' range [a, b] of that
   field (n_nodes in [3, 16]), interpolates y = log(|M'|^2/|M|^2) by the
   Chebyshev series through the nodes and reads log r for every point off it:
   1 + n_nodes amplitude evaluations per event instead of 1 + P.  log r is
   analytic along these axes, so the series coefficients fall off
   geometrically and |c_{n-1}| + |c_{n-2}| estimates the error; an event whose
   estimate exceeds tol, or with a node |M|^2 <= 0 or non-finite (e.g. a top
   mass that does not fit), is recomputed on the exact path for all points
   (d_fallback[e] = 1).  Events with |M|^2 == 0 or non-finite get W' = 0 and
   are counted in h_n_bad (RW_WARN_BAD_EVENTS).  Outputs: d_wnew [P][E]
   (device), d_fallback [E] (device, may be NULL), sigma'_p and sigma as
   compensated sums of the final W' and W (h_sigma [P], h_sigma_orig), the
   number of recomputed events.  Works on the attached events; the workspace
   (rw_interp_workspace_bytes, with events and points set) is separate from
   rw_load_events'.  Synchronises.  RW_ERR_ARG when the points are not on one
   axis or n_nodes / tol are out of range; RW_ERR_MODE in the mixed modes. */
size_t rw_interp_workspace_bytes(const rw_ctx* ctx);
int rw_reweight_interp(rw_ctx* ctx, int n_nodes, double tol, double* d_wnew, unsigned char* d_fallback,
                       double* h_sigma, double* h_sigma_orig, int64_t* h_n_fallback, int64_t* h_n_bad,
                       void* d_workspace, size_t workspace_bytes);

/* ---------------------------------------------------------------------------
   Les Houches Event files (Sec. 3.2 step 2, "parse events", and step 8,
   "return new weights"; the format of hep-ph/0609017, per-event weight
   blocks as in its version 3.0).  Host-side, no GPU needed.
   rw_lhe_open loads the file and indexes its <event> blocks (RW_ERR_ARG when
   the file cannot be read or an <event> is not closed; no handle then).
   rw_lhe_read parses events [first, first+n) with n_threads threads into
   h_mom [N][4][ld] (E, px, py, pz; the process's particle order, matched by
   PDG code among the incoming (status -1) and outgoing (status +1) lines in
   file order, other lines skipped) and h_w [n] (XWGTUP), boosting each event
   along the beam axis into the partonic centre-of-mass frame the kernels
   assume.  RW_ERR_ARG with the event index in rw_lhe_last_error when an event
   does not match the process or a number does not parse.
   rw_lhe_write writes the file again to `path` with, for every event k, the
   lines <wgt id='ids[j]'> h_wnew[j*ld + k] </wgt> (j < P; the shortest
   decimal form that reads back as the same double) inside its <rwgt> block
   (created before </event> when absent); everything else is copied byte for
   byte.  ids must not contain ' < > &. */
typedef struct rw_lhe rw_lhe;
int rw_lhe_open(rw_lhe** out, const char* path);
int rw_lhe_close(rw_lhe* lhe);
const char* rw_lhe_last_error(const rw_lhe* lhe);
int64_t rw_lhe_n_events(const rw_lhe* lhe);
int rw_lhe_read(rw_lhe* lhe, int process, int64_t first, int64_t n, double* h_mom, int64_t ld, double* h_w,
                int n_threads);
int rw_lhe_write(rw_lhe* lhe, const char* path, const double* h_wnew, int P, int64_t ld, const char* const* ids);
/* The same output written in pieces, events in file order:
   rw_lhe_write_begin opens `path` (RW_ERR_STATE if a write is open),
   rw_lhe_write_events adds events [first, first + n) with their weights
   h_wnew[j*ld + i] (first must be the next unwritten event), rw_lhe_write_end
   writes the rest of the file and closes it (RW_ERR_STATE, with the file
   closed, when events are missing). */
int rw_lhe_write_begin(rw_lhe* lhe, const char* path, int P, const char* const* ids);
int rw_lhe_write_events(rw_lhe* lhe, int64_t first, int64_t n, const double* h_wnew, int64_t ld);
int rw_lhe_write_end(rw_lhe* lhe);
/* Event file to event file (Sec. 3.2: step 2, parse events; steps 3-7 on the
   GPU; step 8, return the new weights) with the host work hidden behind the
   GPU's: the file is cut into chunks of `chunk` events; while the GPU
   reweights chunk k (its momenta copied in, the fused kernel, W' copied back
   on the context's stream), n_threads host threads parse chunk k+1 and the
   calling thread writes chunk k-1 to out_path (as rw_lhe_write, the weights
   ids[0..P-1]).  The cross sections are carried from chunk to chunk in
   (sum, compensation) form (deterministic for a given chunk size); sigma'_p,
   sigma and the bad-event count as rw_get_results.  The events must match the
   context's process (RW_ERR_ARG otherwise, the output then incomplete).
   Device workspace of rw_lhe_workspace_bytes(ctx, chunk) bytes, 256-byte
   aligned (two chunks' momenta, weights and W', and the sums); the call
   attaches it as the context's events (as rw_reweight_host does), allocates
   three pinned host chunks for its duration and synchronises. */
size_t rw_lhe_workspace_bytes(const rw_ctx* ctx, int64_t chunk);
int rw_lhe_reweight(rw_ctx* ctx, rw_lhe* lhe, const char* out_path, const char* const* ids, int64_t chunk,
                    int n_threads, void* d_workspace, size_t workspace_bytes, double* h_sigma, double* h_sigma_orig,
                    int64_t* h_n_bad);
/* Samples with several processes (e.g. the Born and real-emission events of
   an NLO sample, Sec. 4): h_process_of_event[k] (one int per event) = the
   first of processes[0..n_processes-1] (1..8 RW_* ids) whose external
   particles event k matches exactly, or -1; n_threads threads. */
int rw_lhe_classify(rw_lhe* lhe, const int* processes, int n_processes, int* h_process_of_event, int n_threads);
/* rw_lhe_read for the events idx[0..n-1] (file indices, any order): event
   idx[i] goes to column i of h_mom [N][4][ld] and h_w[i].  RW_ERR_ARG for an
   index outside the file or an event that does not match the process. */
int rw_lhe_read_list(rw_lhe* lhe, int process, const int64_t* idx, int64_t n, double* h_mom, int64_t ld, double* h_w,
                     int n_threads);

/* ---------------------------------------------------------------------------
   Input conversion of the FP32 modes, exposed for verification.  The paper has
   no counterpart.  In RW_FP32 / RW_MIXED_* the g g -> t tbar (+g) kernels split
   every FP64 momentum component x into two floats, hi = the float nearest to x
   (ties to even) and lo = x - hi rounded to float, using integer operations
   (the kinematic invariants and the reshuffle are then done in double-float
   arithmetic on the FP32 pipe).  This call runs that split on n device doubles:
     d_x [n]  device input;   d_hi [n], d_lo [n]  device outputs (float)
   Zero and |x| < 2^-126 give +-0 (lo 0); |x| >= 2^128 gives +-inf; NaN stays
   NaN; lo is 0 for |x| < 2^-74.  Asynchronous on `stream` (a cudaStream_t,
   NULL = legacy default stream); n < 0 -> RW_ERR_ARG, a NULL pointer with
   n > 0 -> RW_ERR_NULL, a failed launch -> RW_ERR_CUDA (there is no context,
   so no message). */
int rw_split_double(const double* d_x, int64_t n, float* d_hi, float* d_lo, void* stream);

/* ---------------------------------------------------------------------------
   Measured plain-ALU peak of a GPU (the paper has no counterpart): the
   amplitude kernels are bound by the FP64 pipe in RW_FP64 and by the FP32 FMA
   pipe in the other modes, so their roofline denominators are these rates.
   kind 0 = FP64 (DFMA), 1 = FP32 (FFMA): every SM at full occupancy runs
   eight independent FMA chains per thread, one warm-up launch then the best
   of three, timed with CUDA events on cuda_stream (a cudaStream_t, NULL = the
   legacy default stream) of device `device`.  h_tflops: FLOP/s / 1e12
   (an FMA counts 2); h_ms (may be NULL): the best launch's duration.
   Synchronises the stream; allocates nothing.  RW_ERR_NULL, RW_ERR_ARG (bad
   kind) or RW_ERR_CUDA. */
int rw_alu_peak(int device, void* cuda_stream, int kind, double* h_tflops, double* h_ms);

#ifdef __cplusplus
}
#endif
#endif /* RWGT_H */
