/*
 * tt.h -- C ABI of libtt, a GPU (sm_103a) traveltime-parameter search.
 *
 * The library evaluates the semblance coherence of a traveltime operator
 * over prestack seismic gathers and searches the operator's parameters with
 * differential evolution plus an exchange of best individuals between
 * neighbouring zero-offset samples (evolution by neighborhood similarity),
 * after "Ultra-fast traveltime parameters search by a coevolutionary
 * optimization approach using GPUs" (arXiv 2304.11399).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every array argument is a DEVICE pointer owned by the caller, unless a
 *    comment says "host". Float arrays are IEEE float32, row-major, densely
 *    packed, with the shapes given in brackets.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). All work is enqueued on it and the call returns without
 *    waiting, except tt_ctx_create / tt_ctx_load_traces (which synchronise
 *    the stream before returning) and where stated.
 *  - No entry point other than tt_ctx_create allocates device memory.
 *  - Every entry point returns a tt_status; on failure nothing has been
 *    written to caller arrays unless the failure is TT_ERR_CUDA raised by an
 *    asynchronous launch. tt_last_error() gives a message.
 *  - A context may be used from one host thread at a time; calls on
 *    different streams that share a context's scratch (tt_search,
 *    tt_ens_search, tt_neighbor_exchange, tt_polish, split evaluations --
 *    see TT_OPT_SPLIT) must not overlap.
 *
 * Notation (the paper's): a domain is one zero-offset sample (m0, it0),
 * t0 = it0 dt (Sec. 2.1, "index-vector point (t, tr)"); its aperture is the
 * set of N traces used by one semblance call (T_a in eq. order); theta is a
 * parameter vector ("individual", Sec. 2) of D = 1 (CMP: C), D = 3
 * (ZO-CRS: A, B, C) or D = 5 (FO-CRS: Am, Ah, Bmm, Bmh, Bhh) values; NP
 * individuals form a domain's population.
 */
#ifndef TT_H
#define TT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tt_status;
enum {
  TT_OK = 0,
  TT_ERR_INVALID_ARG = 1,   /* bad pointer, size, index or configuration   */
  TT_ERR_CUDA = 2,          /* a CUDA runtime call or launch failed        */
  TT_ERR_OUT_OF_MEMORY = 3, /* tt_ctx_create could not allocate            */
  TT_ERR_TIMEOUT = 4,       /* a bounded device wait gave up               */
  TT_ERR_UNSUPPORTED = 5    /* valid request outside what is built         */
};

/* Traveltime operators (readings of the operators the paper cites, Sec. 1):
 *   TT_OP_CMP:   T = t0^2 + C h^2                         theta = (C)
 *   TT_OP_CRS:   T = (t0 + A dm)^2 + B dm^2 + C h^2       theta = (A, B, C)
 *   TT_OP_FOCRS: T = (t0 + Am dm + Ah dh)^2 + Bmm dm^2 + Bmh dm dh + Bhh dh^2
 *                theta = (Am, Ah, Bmm, Bmh, Bhh): the hyperbolic finite-offset
 *                CRS operator (two slopes, three curvatures) for the sample
 *                t0 of the common-offset section at central offset h0,
 *                dh = h - h0 (tt_problem.group_h0)
 * with dm = m - m0 the midpoint displacement and h the full offset of a
 * trace (metres), t = sqrt(T) (seconds); a trace with T < 0 contributes
 * zero amplitudes and still counts in N. */
enum { TT_OP_CMP = 0, TT_OP_CRS = 1, TT_OP_FOCRS = 2 };

/* Storage type of the context's copy of the traces (arithmetic is FP32). */
enum { TT_STORE_F32 = 0, TT_STORE_BF16 = 1 };

#define TT_MAX_DIM 8
#define TT_MAX_HALF_WINDOW 8

/* Prestack gathers (Sec. 4, "bucket": the traces of an interactive domain). */
typedef struct tt_gathers {
  int32_t n_traces;      /* number of traces                                 */
  int32_t ns;            /* samples per trace (NT)                           */
  int32_t storage;       /* TT_STORE_F32 or TT_STORE_BF16                    */
  int32_t reserved;
  const float* traces;   /* [n_traces][ns] amplitudes; the record is zero    */
                         /* outside samples 0..ns-1                          */
  const float* mid;      /* [n_traces] midpoint m of each trace (m)          */
  const float* off;      /* [n_traces] full source-receiver offset h (m)     */
} tt_gathers;

/* Domains and apertures. Domains sharing a midpoint, sample interval and
 * aperture form a group; apertures are CSR lists of trace indices. */
typedef struct tt_problem {
  int32_t op;            /* TT_OP_CMP, TT_OP_CRS or TT_OP_FOCRS             */
  int32_t half_window;   /* w: the window is the 2w+1 samples t + k dt,      */
                         /* k = -w..w (Sec. 2, W_l = 2w+1), 0 <= w <= 8      */
  int32_t n_groups;
  int32_t n_dom;
  const float* group_m0;    /* [n_groups] reference midpoint m0 (m)          */
  const float* group_dt;    /* [n_groups] sample interval dt (s), > 0        */
  const int32_t* ap_ptr;    /* [n_groups+1] CSR row pointers into ap_idx     */
  const int32_t* ap_idx;    /* [ap_ptr[n_groups]] trace indices              */
  const int32_t* dom_it0;   /* [n_dom] zero-offset sample index it0          */
  const int32_t* dom_group; /* [n_dom] group of each domain                  */
  int32_t n_m0, n_t0;    /* exchange grid: if n_m0 * n_t0 == n_dom the       */
                         /* domains are laid out m0-major, d = im0*n_t0+it;  */
                         /* 0, 0 = no grid (no exchange)                     */
  const float* group_h0; /* [n_groups] central full offset h0 (m) of each    */
                         /* group: TT_OP_FOCRS only (NULL otherwise)         */
} tt_problem;

/* Search settings (Sec. 2.1: NP, NG, p = 1; F and CR fixed, or adapted as
 * in JADE when `adapt` is 1). */
typedef struct tt_de_cfg {
  int32_t np;            /* population size NP, 4..1024                     */
  int32_t ng;            /* generations NG >= 0                             */
  float F, CR;           /* mutation factor in [0, 2], crossover rate in    */
                         /* [0, 1]; with adapt = 1 the initial mu_F in      */
                         /* (0, 1] and mu_CR in [0, 1] (JADE: 0.5, 0.5)     */
  uint64_t seed;         /* Philox4x32-10 key                               */
  float lo[TT_MAX_DIM];  /* parameter bounds, lo[d] <= hi[d]                */
  float hi[TT_MAX_DIM];
  int32_t exch_every;    /* neighbour exchange after the selection of every */
                         /* exch_every-th generation; 0 = never             */
  int32_t polish_steps;  /* projected gradient-ascent steps after DE        */
  float polish_lr;       /* step: theta += lr (hi-lo)^2 dS/dtheta           */
  int32_t adapt;         /* 0: fixed F, CR. 1: JADE adaptation (Sec. 2.1.4,  */
                         /* the cited JADE with c = 0.1): per member        */
                         /* CR_i ~ N(mu_CR, 0.1) clipped to [0, 1], F_i ~   */
                         /* Cauchy(mu_F, 0.1) redrawn while <= 0, capped at */
                         /* 1; r2 drawn from population + archive of the    */
                         /* parents of strictly better children (<= NP,     */
                         /* uniform replacement when full); mu moved by c   */
                         /* towards the mean CR and Lehmer-mean F of the    */
                         /* successes. tt_search, tt_de_step and the ENS    */
                         /* sweep (a fresh memory and archive per sample).  */
} tt_de_cfg;

typedef struct tt_ctx tt_ctx;

/* Message of the last failure on `ctx` (or of the calling thread's last
 * tt_ctx_create failure when ctx is NULL). Never NULL. */
const char* tt_last_error(const tt_ctx* ctx);

/* Version string of the library build. */
const char* tt_version(void);

/* Create a context: validates the problem on the device, copies the traces
 * into a zero-padded, aligned device layout of the chosen storage type,
 * builds the per-aperture geometry table, copies the domain arrays and
 * allocates the search scratch (sized by cfg->np and D). The caller's
 * arrays may be freed once this returns. Synchronises `stream`.
 * Errors: INVALID_ARG (NULL pointers, sizes, out-of-range indices, an
 * unsorted ap_ptr, dt <= 0, bad cfg), OUT_OF_MEMORY, CUDA. On failure
 * *out is NULL. `cfg` may be NULL when no search will be run. */
tt_status tt_ctx_create(tt_ctx** out, const tt_gathers* gathers, const tt_problem* problem,
                        const tt_de_cfg* cfg, void* stream);

/* Reload the context's copy of the traces from `traces` ([n_traces][ns],
 * same shape as at creation); `host` != 0 means a host pointer (pinned
 * memory gives an asynchronous-speed copy). Synchronises `stream`. */
tt_status tt_ctx_load_traces(tt_ctx* ctx, const float* traces, int32_t host, void* stream);

void tt_ctx_destroy(tt_ctx* ctx);

/* Semblance (Sec. 1, Neidell-Taner; Sec. 2.2 eq. S, values in [0, 1]) of P
 * parameter vectors at every domain:
 *   u_i = sqrt(T_i)/dt, j = floor(u_i), f = u_i - j,
 *   a_ik = (1-f) x_i[j+k] + f x_i[j+k+1], k = -w..w,
 *   S = sum_k (sum_i a_ik)^2 / (N sum_ik a_ik^2), 0 when the energy is 0.
 * theta [n_dom][P][D], S [n_dom][P]. P >= 1. FP32 arithmetic. */
tt_status tt_semblance_eval(tt_ctx* ctx, const float* theta, int32_t P, float* S, void* stream);

/* Semblance and its gradient dS/dtheta (an addition to the paper's method,
 * used to polish the DE winner) by the adjoint of the interpolation and
 * traveltime: inside an interpolation cell da_ik/du_i = x_i[j+k+1]-x_i[j+k].
 * theta [n_dom][P][D], S [n_dom][P], dS [n_dom][P][D]. */
tt_status tt_semblance_grad(tt_ctx* ctx, const float* theta, int32_t P, float* S, float* dS,
                            void* stream);

/* Stacked zero-offset output along one operator per domain: the output
 * sample at (m0, t0) is the mean, over the domain's N aperture traces, of the
 * amplitude at the operator's traveltime, read by the same clamped linear
 * interpolation as the centre sample of the semblance window:
 *   out[d] = (1/N) sum_i ((1-f_i) x_i[j_i] + f_i x_i[j_i+1]),
 * a trace with T < 0 or past the record adding 0, and out[d] = 0 when N = 0.
 * This is the enhanced zero-offset sample that the operator rebuilds (Sec.
 * 1) and the stacking panels of Sec. 5.1 show, taken at the searched
 * parameters. theta [n_dom][D] (device, e.g. tt_search's best_theta), out
 * [n_dom] (device), both owned by the caller; FP32 with a fixed summation
 * order (per-lane strided sums, then a butterfly across the warp), so a
 * call's result does not depend on the launch. Errors: TT_ERR_INVALID_ARG
 * for NULL arrays. */
tt_status tt_stack(tt_ctx* ctx, const float* theta, float* out, void* stream);

/* One differential-evolution step per domain (Sec. 2.1.1-2.1.4, p = 1):
 *  gen == 0:  initialise pop [n_dom][NP][D] uniformly in [lo, hi]; other
 *             arrays are ignored and may be NULL.
 *  gen >= 1:  if trial != NULL, greedy selection: member i takes
 *             (trial[i], trial_fit[i]) when trial_fit[i] >= fit[i] (NaN
 *             ranks lowest); then best_idx[d] = argmax fit (lowest index on
 *             ties); then, if next_trial != NULL, DE/current-to-best/1/bin:
 *             v = x_i + F (x_best - x_i) + F (x_r1 - x_r2), binomial
 *             crossover with j_rand, repair v<lo -> (lo+x_i)/2,
 *             v>hi -> (hi+x_i)/2, written to next_trial [n_dom][NP][D].
 *  cfg.adapt: the JADE state (mu_CR, mu_F, archive, the trial's F_i and
 *             CR_i) lives in the context: gen 0 resets it; a selection
 *             updates the archive and mu (the trial selected is that of
 *             generation gen - 1 when next_trial != NULL, else of gen);
 *             the mutation draws F_i, CR_i and takes r2 from population +
 *             archive. One search per context at a time.
 * Random numbers: Philox4x32-10, key = seed, counter = (i, gen, domain,
 * block); FP32 arithmetic with one rounding per operation, so results are
 * bit-reproducible. pop and fit [n_dom][NP] are updated in place;
 * best_idx [n_dom] may be NULL. */
tt_status tt_de_step(tt_ctx* ctx, int32_t gen, float* pop, float* fit, const float* trial,
                     const float* trial_fit, float* next_trial, int32_t* best_idx,
                     void* stream);

/* Copy the JADE adaptation state of a context created with cfg.adapt = 1
 * out to (save = 1) or in from (save = 0) caller arrays, for checkpointing an
 * adaptive search driven by tt_de_step: mu [n_dom][2] (mu_CR, mu_F), n_arc
 * [n_dom] (archive fill), archive [n_dom][NP][D], F and CR [n_dom][NP] (the
 * pending trial's F_i, CR_i). Device pointers owned by the caller; the paper
 * has no counterpart (with Philox stateless, pop, fit, the pending trial and
 * its fitness, the generation and this state are the whole search state).
 * Asynchronous on `stream`. Errors: TT_ERR_INVALID_ARG without adaptation or
 * for NULL arrays. */
tt_status tt_jade_state(tt_ctx* ctx, int32_t save, float* mu, int32_t* n_arc, float* archive,
                        float* F, float* CR, void* stream);

/* best_theta [n_dom][D] and best_S [n_dom] (either may be NULL) = the
 * member with the highest fitness of each domain (lowest index on ties). */
tt_status tt_best_snapshot(tt_ctx* ctx, const float* pop, const float* fit, float* best_theta,
                           float* best_S, void* stream);

/* Neighbour exchange (Sec. 3.3 "Information propagation"): on the m0-major
 * grid n_m0 x n_t0 (n_m0 * n_t0 == n_dom), every domain imports the
 * snapshot best_theta [n_dom][D] of its present neighbours, in the order
 * (it0-1), (it0+1), (m0-1), (m0+1), into its worst members ranked by
 * (fitness ascending, index ascending) excluding its own best, and
 * evaluates each import's semblance at its own (m0, t0) into fit.
 * imports [n_dom][4][D] and slots [n_dom][4] (-1 = absent neighbour)
 * record what was done; either may be NULL. */
tt_status tt_neighbor_exchange(tt_ctx* ctx, int32_t n_m0, int32_t n_t0, const float* best_theta,
                               float* pop, float* fit, float* imports, int32_t* slots,
                               void* stream);

/* Projected gradient ascent from theta [n_dom][D] (in/out): `steps`
 * iterations of theta <- clip(theta + lr (hi-lo)^2 dS/dtheta, lo, hi),
 * S evaluated at every iterate, keeping the best iterate (first on ties);
 * S [n_dom] receives its semblance. Uses the context's scratch. */
tt_status tt_polish(tt_ctx* ctx, float* theta, float* S, int32_t steps, float lr, void* stream);

/* Evolution by neighborhood similarity in sweep mode (Sec. 3.3-3.6): the
 * grid's traces (m0) are cut into buckets of n_bucket consecutive traces;
 * every bucket runs a forward exploration (NP_f x NG_f, seeded with the best
 * of the same sample on the previous trace) and n_cycle backward-and-forward
 * cycles (NP_bf x NG_bf, seeded with the bests of samples t-1, t+1, of
 * sample t on the previous trace of the sweep, and the own best); each stage
 * estimates every (n_skip+1)-th sample and interpolates the others linearly
 * in t, keeping the higher semblance (Sec. 3.5). In the backward-and-forward
 * stages a sample's own best seed is not evaluated again: its stored
 * semblance is its fitness (the call count of eq. ens_semblance leaves it
 * out as well). */
typedef struct tt_ens_cfg {
  int32_t np_f, ng_f;    /* forward exploration: population, generations      */
  int32_t np_bf, ng_bf;  /* backward-and-forward stages                       */
  int32_t n_skip;        /* samples interpolated between estimated ones       */
  int32_t n_cycle;       /* backward-and-forward cycles (<= 64)               */
  int32_t n_bucket;      /* traces per bucket (interactive domain), >= 1      */
  int32_t reserved;
} tt_ens_cfg;

/* Run the ENS sweep over the context's (m0, t0) grid (n_m0 * n_t0 == n_dom)
 * with F, CR, seed, bounds and adapt from the context's tt_de_cfg (with
 * adapt, every estimated sample starts a fresh JADE memory and archive),
 * whose np must be at least np_f and np_bf (both >= 4). Writes best_theta [n_dom][D] and
 * best_S [n_dom]; *n_evals (host, may be NULL) receives the semblance-call
 * count of eq. ens_semblance for the estimated and interpolated samples
 * actually visited. Uses the context's search scratch (not concurrently with
 * tt_search). Captured into a CUDA graph on first use like tt_search. */
tt_status tt_ens_search(tt_ctx* ctx, const tt_ens_cfg* cfg, float* best_theta, float* best_S,
                        uint64_t* n_evals, void* stream);

/* Counters of a context, accumulated on the host since the last reset:
 * `launches` = kernels this context enqueued; `semblance_launches` and
 * `trace_evals` = semblance/gradient launches and the (aperture trace x
 * parameter vector) pairs they evaluated; `semblance_ms` = their summed
 * device time, measured with CUDA events recorded on the launching stream
 * around each of them while profiling is enabled (0 otherwise). */
typedef struct tt_stats {
  uint64_t launches;
  uint64_t semblance_launches;
  double trace_evals;
  double semblance_ms;
  uint64_t timed_launches;   /* semblance launches covered by semblance_ms */
} tt_stats;

/* Enable (1) or disable (0) event timing of semblance launches. Enabling
 * creates a fixed pool of events (no device memory); launches beyond the
 * pool between two tt_ctx_stats calls are counted but not timed. */
tt_status tt_ctx_profile(tt_ctx* ctx, int32_t enable);

/* Copy the counters to *out (host) and, if `reset`, zero them. When timed
 * launches are pending this waits for the last recorded event. */
tt_status tt_ctx_stats(tt_ctx* ctx, tt_stats* out, int32_t reset);

/* L1 load-bandwidth probe (no passage in the paper: a measurement aid for
 * the semblance kernel's roofline). Enqueues on `stream` one kernel in which
 * one wave of resident 256-thread blocks (at most 8 per SM) each stream
 * `iters` x 32 coalesced 4-byte
 * loads per thread (32 consecutive floats per warp request, the load K1
 * gathers its windows with) from a 24 KiB window of the context's scratch
 * that stays in L1, each iteration at other lines of the window;
 * *bytes (host) receives the bytes it loads. Time it with events on
 * `stream`. It reads the scratch's contents, whatever they are, and may
 * write one float of it (the scratch holds nothing between launches).
 * Errors: INVALID_ARG for iters < 1 or a NULL bytes. */
tt_status tt_ctx_probe_l1(tt_ctx* ctx, int32_t iters, double* bytes, void* stream);

/* Launch options of a context (tt_ctx_set_option / tt_ctx_get_option):
 *  TT_OPT_KERNEL  semblance kernel variant for forward evaluations:
 *                 TT_KERNEL_PACKED (default; two parameter vectors per thread
 *                 with packed FP32x2 arithmetic, one launch covering every
 *                 (domain, vector) pair), TT_KERNEL_PERSISTENT (the same work
 *                 in a persistent grid sized to the GPU, warps taking 64-pair
 *                 work units from an atomic counter -- load balance for
 *                 uneven apertures), TT_KERNEL_SCALAR (one pair per thread).
 *                 All variants perform the same operations in the same order
 *                 and give bit-identical S.
 *  TT_OPT_BLOCK   threads per block, 128 or 256 (default 256).
 *  TT_OPT_SEARCH_GRAPH  1 (default): tt_search captures its whole launch
 *                 sequence into a CUDA graph on first use and replays it;
 *                 0: launch eagerly. Searches run eagerly while profiling is
 *                 enabled.
 *  TT_OPT_SPLIT   1 (default): a forward evaluation of fewer than
 *                 n_sm x 32 x 64 (domain, vector) pairs, n_sm the device's
 *                 multiprocessor count (TT_OPT_SPLIT_MAX_PAIRS reads the
 *                 figure) -- too few to fill the GPU at one warp per 64
 *                 pairs -- runs a kernel in which
 *                 the S warps of a block (8, 16 or 32, more for smaller
 *                 launches) share 64 pairs, each warp summing a contiguous
 *                 slice of every pair's aperture, the partial sums added in
 *                 slice order; every variant then launches that kernel, so S
 *                 still does not depend on TT_OPT_KERNEL / TT_OPT_BLOCK, but
 *                 its rounding differs from the unsplit kernels' (all stay
 *                 within 1e-5 of the exact semblance). The smallest launches
 *                 also spread a unit over up to 9 blocks that combine their
 *                 sums through the context's scratch, so split evaluations on
 *                 one context must not overlap on the GPU (one stream, or
 *                 events between streams). 0: never split.
 *  TT_OPT_MEMBER_ORDER  1: before each generation's evaluation inside
 *                 tt_search / tt_search_slab (NP <= 256), the members of
 *                 every domain are put in the order of their window position
 *                 on the domain's middle aperture entry, so that the lanes of
 *                 a warp read windows that lie close together; the results go
 *                 back to each member's own slot, and S, the search and its
 *                 call count are bit-identical to 0 (the index order). The
 *                 reordered copy uses the trial buffer that the generation's
 *                 selection has just consumed. 2 (default): 1 when the
 *                 apertures hold at least 768 traces on average (long
 *                 apertures scatter the members' windows most and carry the
 *                 most work per member), else 0.
 *  TT_OPT_SPLIT_MAX_PAIRS  (read only) the split threshold above, in pairs.
 *  TT_OPT_SM_COUNT  (read only) multiprocessors of the context's device,
 *                 queried at tt_ctx_create; the split thresholds and the
 *                 persistent grid scale with it.
 *  Changing an option drops a captured graph. */
enum {
  TT_OPT_KERNEL = 1,
  TT_OPT_BLOCK = 2,
  TT_OPT_SEARCH_GRAPH = 3,
  TT_OPT_SPLIT = 4,
  TT_OPT_SPLIT_MAX_PAIRS = 5,
  TT_OPT_SM_COUNT = 6,
  TT_OPT_MEMBER_ORDER = 7
};
enum { TT_KERNEL_PACKED = 1, TT_KERNEL_PERSISTENT = 2, TT_KERNEL_SCALAR = 3 };
#define TT_N_TUNE_CANDIDATES 6
tt_status tt_ctx_set_option(tt_ctx* ctx, int32_t option, int64_t value);
tt_status tt_ctx_get_option(const tt_ctx* ctx, int32_t option, int64_t* value);

/* Autotuner: times every (kernel variant, block size) candidate -- in the
 * order packed/256, packed/128, persistent/256, persistent/128, scalar/256,
 * scalar/128 -- on one evaluation of theta [n_dom][P][D] (S [n_dom][P]
 * receives it), keeps the fastest as the context's TT_OPT_KERNEL and
 * TT_OPT_BLOCK, and writes the mean time of each candidate in ms to
 * times_ms (host, TT_N_TUNE_CANDIDATES entries, may be NULL). A persistent
 * candidate is kept only if it is more than 3% faster than the fastest
 * packed or scalar one; otherwise that one is kept (the persistent form's
 * work queue gives up the L1 sharing between adjacent domains that a
 * converged population has and a first-generation trial does not show).
 * Synchronises `stream`. */
tt_status tt_ctx_autotune(tt_ctx* ctx, const float* theta, int32_t P, float* S,
                          float* times_ms, void* stream);

/* The whole search (JADE loop of Sec. 2.1 with the exchange of Sec. 3.3):
 * init, NG generations of select/mutate/evaluate, an exchange after every
 * exch_every-th selection, then cfg polish_steps of polishing. Writes
 * best_theta [n_dom][D] and best_S [n_dom] (device). *n_evals (host, may be
 * NULL) receives the number of semblance evaluations issued:
 * NP (1 + NG) n_dom (eq. jade_semblance) + imports + polish calls.
 * Requires a cfg at tt_ctx_create. Uses the context's scratch. */
tt_status tt_search(tt_ctx* ctx, float* best_theta, float* best_S, uint64_t* n_evals,
                    void* stream);

/* One slab of a search sharded over several GPUs by midpoint (Sec. 4: the
 * data is cut into buckets processed independently; Sec. 5.5: the buckets
 * run on up to 16 GPUs). A long line is cut into contiguous slabs of CMPs,
 * one per GPU; each GPU's context holds its slab's domains (an m0-major
 * n_m0 x n_t0 grid) over a copy of only the traces their apertures read
 * (the slab plus a read-only halo of the aperture radius). The slabs share
 * one thing: at every exchange generation, the neighbour exchange of the
 * first (last) row of a slab imports the bests of the previous (next)
 * slab's last (first) row. The library writes its own edge rows to
 * send_first / send_last and then calls `exchange`, which must fill
 * recv_prev / recv_next with the neighbouring slabs' rows of the same
 * generation -- by NCCL send/recv into this GPU's own memory, by host
 * staging, or otherwise -- before returning, or enqueue that on `stream`
 * (the library's next launch on `stream` reads them). With dom_base the
 * global index of the slab's first domain on the whole line's grid (its
 * Philox keys), the slabs together compute exactly what tt_search computes
 * on the whole line, bit for bit. */
typedef int32_t (*tt_halo_fn)(void* user, int32_t gen, void* stream);
typedef struct tt_slab {
  int64_t dom_base;        /* global index of the context's first domain       */
  int32_t has_prev;        /* 1: a slab lies before this one (m0 - 1 exists)   */
  int32_t has_next;        /* 1: a slab lies after this one                    */
  float* send_first;       /* [n_t0][D] device, caller-owned: the bests of the */
  float* send_last;        /* slab's first / last m0 row, written by the       */
                           /* library on `stream` before each exchange call    */
  const float* recv_prev;  /* [n_t0][D] device: the previous slab's last row  */
  const float* recv_next;  /* [n_t0][D] device: the next slab's first row     */
  tt_halo_fn exchange;     /* called on the host at every exchange generation;*/
                           /* a non-zero return aborts the search             */
  void* user;              /* passed to exchange                              */
} tt_slab;

/* The search of tt_search on one slab (see tt_slab): same loop, draws keyed
 * by dom_base + domain, the exchange's edge rows taken from recv_prev /
 * recv_next. Runs eagerly (no graph: the exchange calls back to the host).
 * *n_evals counts this slab's calls, imports from the neighbouring slabs
 * included. Errors: INVALID_ARG (no grid, NULL slab or rows, dom_base out
 * of range, exchange missing while a neighbour exists and exch_every > 0,
 * or a non-zero return of exchange), CUDA. */
tt_status tt_search_slab(tt_ctx* ctx, const tt_slab* slab, float* best_theta, float* best_S,
                         uint64_t* n_evals, void* stream);

/* Allocation-free semblance evaluation. The paper has no counterpart: this
 * entry point serves callers that cannot allocate device memory, such as a
 * plug-in whose host application owns every device buffer, or a service loop
 * in which cudaMalloc (which may synchronise the device and can fail once
 * memory is fragmented) is not allowed after start-up. Such callers cannot
 * create a context, so this call evaluates exactly what tt_semblance_eval
 * evaluates, directly on the caller's arrays: gathers (storage must be
 * TT_STORE_F32; the traces are read in place), problem, theta
 * [n_dom][P][D] and S [n_dom][P], all device pointers owned by the caller.
 * It calls no cudaMalloc or cudaFree. Its scratch (the aperture geometry
 * table and a validation flag) is a fixed device array of
 * TT_NOALLOC_SCRATCH_BYTES inside the library, held by every GPU that loads
 * the library until the process exits; problems whose aperture lists hold
 * more than TT_NOALLOC_MAX_APERTURE_ENTRIES entries, and TT_OP_FOCRS problems,
 * are rejected with TT_ERR_UNSUPPORTED. Positions follow tt_semblance_eval's
 * two forms (direct up to 2048 samples, the moveout form for longer
 * records), so S agrees with the exact semblance to the same 1e-5. Every
 * call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing), so a device reset by the
 * host application between calls is harmless. Every call synchronises
 * `stream` twice -- to read ap_ptr, then the result of the on-device
 * validation (INVALID_ARG as for tt_ctx_create) -- and then enqueues the
 * evaluation without waiting. All calls share the scratch array, which keeps the last call's contents: calls
 * that overlap on the GPU race on it, so serialise them (one stream, or
 * events). Error messages: tt_last_error(NULL). */
#define TT_NOALLOC_SCRATCH_BYTES (4u << 20)
#define TT_NOALLOC_MAX_APERTURE_ENTRIES 262128
tt_status tt_semblance_eval_noalloc(const tt_gathers* gathers, const tt_problem* problem,
                                    const float* theta, int32_t P, float* S, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TT_H */
