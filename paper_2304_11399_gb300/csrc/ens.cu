// Evolution by neighborhood similarity in sweep mode (tt_ens_search): the
// paper's ENS (Sec. 3.3-3.6) on the m0-major (m0, t0) grid, cut into buckets
// of n_bucket consecutive traces (CMPs).
//
// Stages: a forward exploration (NP_f x NG_f, one seed: the best of the same
// sample on the previous trace), then n_cycle backward-and-forward cycles
// (NP_bf x NG_bf, four seeds: the bests of samples t-1 and t+1 on the trace,
// of sample t on the previous trace of the sweep, and the own best). Each
// stage estimates every (n_skip+1)-th sample from an offset (0 for the
// exploration; 0 or 1 backward; n_skip forward) and interpolates the others
// linearly in t, keeping the higher semblance.
//
// GPU mapping: the sweep is sequential over the traces of a bucket, so one
// step handles the current trace of every bucket at once -- all estimated
// samples of all buckets in each launch. Per step: seed and initialise the
// populations (the same kernel writes the step's local-to-global domain map),
// evaluate, run the DE generations (the ordinary DE and semblance kernels on
// the mapped subset; the last selection also writes the bests), interpolate
// the skipped samples (writing their map), evaluate them and keep the higher.
// Random numbers: Philox keyed by the global domain, with the counter's
// generation field (stage + 1) * 65536 + g. Scratch: the context's search
// buffers (the context's NP must be at least NP_f and NP_bf). The whole
// sweep is captured into a CUDA graph on first use.
#include <algorithm>

#include "tt_internal.cuh"

tt::DeArgs tt_make_de_args(const tt_ctx* c, int gen);

namespace {

struct StepGeo {
  int n_m0, n_t0, nb, n_buckets, tb, init, stride, n_est, n_skp, dirn;
};

__device__ __forceinline__ int bucket_len(const StepGeo& g, int b) {
  return min(g.nb, g.n_m0 - b * g.nb);
}

// r-th estimated sample of this step (bucket-major): global domain or -1
__device__ __forceinline__ int est_domain(const StepGeo& g, int r) {
  const int b = r / g.n_est, k = r - b * g.n_est;
  const int t = g.init + k * g.stride;
  if (g.tb >= bucket_len(g, b) || t >= g.n_t0) return -1;
  return (b * g.nb + g.tb) * g.n_t0 + t;
}

// r-th non-estimated sample of this step: the samples before init, then the
// stride - 1 samples after each estimated one
__device__ __forceinline__ int skip_domain(const StepGeo& g, int r) {
  const int b = r / g.n_skp, k = r - b * g.n_skp;
  int t;
  if (k < g.init) {
    t = k;
  } else {
    const int kk = k - g.init, per = g.stride - 1;
    t = g.init + (kk / per) * g.stride + 1 + kk % per;
  }
  if (g.tb >= bucket_len(g, b) || t >= g.n_t0) return -1;
  return (b * g.nb + g.tb) * g.n_t0 + t;
}

__device__ __forceinline__ bool unset(const float* th) { return isnan(th[0]); }

// One thread per (local domain r, population slot i): the i-th present seed
// in the order (t-1, t+1, previous trace, own best) -- only the previous
// trace in the exploration stage -- or a random member drawn from Philox.
// In the backward and forward stages the own best, the last seed, is not
// evaluated again: its semblance at this sample is the stored best_S, written
// to fit here (every sample has a best once the exploration has passed, so the
// own best is always there; were it not, the last slot would be passed over
// with a NaN fitness, which ranks lowest). The other NP - 1 members are also
// copied to the rows of cth [r][NP - 1][D], with cslot [r][NP - 1] naming each
// one's slot in pop, so that the evaluation reads them contiguously and
// scatters their semblance into fit.
__global__ void k_ens_init(StepGeo g, int bf, int NP, int D, int* map, const float* best_th,
                           const float* best_S, float* pop, float* fit, float* cth, int* cslot,
                           uint32_t key0, uint32_t key1, uint32_t gen, const float* lo,
                           const float* hi, float* jade_mu, int* jade_na, float F0, float CR0) {
  const long long n = (long long)g.n_buckets * g.n_est * NP;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int r = int(q / NP), i = int(q - (long long)r * NP);
  const int d = est_domain(g, r);
  if (i == 0) map[r] = d;  // the step's map for the kernels that follow
  if (d < 0) return;
  if (jade_mu && i == 0) {  // a fresh JADE memory and an empty archive per sample
    jade_mu[2 * (size_t)r] = CR0;
    jade_mu[2 * (size_t)r + 1] = F0;
    jade_na[r] = 0;
  }
  const int t = d % g.n_t0, b = r / g.n_est;
  const bool has_prev = (g.tb - g.dirn) >= 0 && (g.tb - g.dirn) < bucket_len(g, b);
  const int dprev = d - g.dirn * g.n_t0;
  const float* seed[4];
  int ns = 0;
  if (!bf) {
    if (has_prev && !unset(best_th + (size_t)dprev * D)) seed[ns++] = best_th + (size_t)dprev * D;
  } else {
    if (t - 1 >= 0 && !unset(best_th + (size_t)(d - 1) * D)) seed[ns++] = best_th + (size_t)(d - 1) * D;
    if (t + 1 < g.n_t0 && !unset(best_th + (size_t)(d + 1) * D))
      seed[ns++] = best_th + (size_t)(d + 1) * D;
    if (has_prev && !unset(best_th + (size_t)dprev * D)) seed[ns++] = best_th + (size_t)dprev * D;
    if (!unset(best_th + (size_t)d * D)) seed[ns++] = best_th + (size_t)d * D;
  }
  float* out = pop + ((size_t)r * NP + i) * D;
  float* cout = nullptr;  // the member's compact row (none for the own best)
  if (bf) {
    const bool own = !unset(best_th + (size_t)d * D);
    const int sk = own ? ns - 1 : NP - 1;
    if (i == sk) {
      fit[(size_t)r * NP + sk] = own ? best_S[d] : __int_as_float(0x7fc00000);
    } else {
      const size_t c = (size_t)r * (NP - 1) + (i > sk ? i - 1 : i);
      cslot[c] = i;
      cout = cth + c * D;
    }
  }
  if (i < ns) {
    for (int k = 0; k < D; ++k) out[k] = seed[i][k];
    if (cout)
      for (int k = 0; k < D; ++k) cout[k] = seed[i][k];
    return;
  }
  tt::Words w(key0, key1, uint32_t(d), gen, uint32_t(i), D);
  for (int k = 0; k < D; ++k) {
    const float v = __fadd_rn(lo[k], __fmul_rn(tt::unit_float(w.w[k]), __fsub_rn(hi[k], lo[k])));
    out[k] = v;
    if (cout) cout[k] = v;
  }
}

// One warp per local domain: the population's best becomes the sample's best.
__global__ void k_ens_update(int n, int NP, int D, const int* map, const float* pop,
                             const float* fit, float* best_th, float* best_S) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int d = map[warp];
  if (d < 0) return;
  const int b = tt::warp_argmax(fit + (size_t)warp * NP, NP, lane);
  if (lane < D) best_th[(size_t)d * D + lane] = pop[((size_t)warp * NP + b) * D + lane];
  if (lane == 0) best_S[d] = fit[(size_t)warp * NP + b];
}

// Linear interpolation in t of each skipped sample between the bests of the
// nearest estimated samples of its trace (FP32, one rounding per operation);
// beyond the first or last estimated sample the nearest one is copied.
__global__ void k_ens_interp(StepGeo g, int D, int* map, const float* best_th, float* th_out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.n_buckets * g.n_skp) return;
  const int d = skip_domain(g, r);
  map[r] = d;  // the map of the evaluation and keep that follow
  if (d < 0) return;
  const int t = d % g.n_t0, row = d - t;
  const int ta = t >= g.init ? g.init + ((t - g.init) / g.stride) * g.stride : -1;
  const int tb = t < g.init ? g.init : ta + g.stride;
  const bool has_a = ta >= 0, has_b = tb < g.n_t0;
  float* out = th_out + (size_t)r * D;
  const float* A = best_th + (size_t)(row + (has_a ? ta : tb)) * D;
  const float* B = best_th + (size_t)(row + (has_b ? tb : ta)) * D;
  if (has_a && has_b) {
    const float w = __fdiv_rn(float(t - ta), float(tb - ta));
    for (int k = 0; k < D; ++k) out[k] = __fadd_rn(A[k], __fmul_rn(w, __fsub_rn(B[k], A[k])));
  } else {
    for (int k = 0; k < D; ++k) out[k] = A[k];
  }
}

__global__ void k_ens_keep(int n, int D, const int* map, const float* th, const float* S,
                           float* best_th, float* best_S) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int d = map[r];
  if (d < 0) return;
  if (tt::rank_key(S[r]) > tt::rank_key(best_S[d])) {
    best_S[d] = S[r];
    for (int k = 0; k < D; ++k) best_th[(size_t)d * D + k] = th[(size_t)r * D + k];
  }
}

__global__ void k_ens_clear(int n, int D, float* best_th, float* best_S) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  best_S[d] = -INFINITY;
  for (int k = 0; k < D; ++k) best_th[(size_t)d * D + k] = __int_as_float(0x7fc00000);
}

int blocks(long long n, int b = 256) { return int(std::max<long long>(1, (n + b - 1) / b)); }

struct Stage {
  bool bf;
  int dirn, init;
};

// Enqueue the whole sweep on `s` into (bth, bS); returns the call count.
tt_status ens_body(tt_ctx* c, const tt_ens_cfg& e, float* bth, float* bS, cudaStream_t s,
                   unsigned long long* n_calls) {
  const int D = c->D, n_m0 = c->n_m0, n_t0 = c->n_t0;
  const int nb = e.n_bucket, n_buckets = (n_m0 + nb - 1) / nb;
  unsigned long long calls = 0;
  tt_status st = TT_OK;
#define STEP(expr, what)                                 \
  do {                                                   \
    st = tt_cuda_check(c, (expr), what);                 \
    if (st != TT_OK) return st;                          \
  } while (0)
  k_ens_clear<<<blocks(c->n_dom), 256, 0, s>>>(c->n_dom, D, bth, bS);
  STEP(c->counted(cudaGetLastError()), "ens clear");
  Stage stages[1 + 2 * 64];
  int n_st = 0;
  stages[n_st++] = {false, +1, 0};
  for (int k = 0; k < e.n_cycle; ++k) {
    stages[n_st++] = {true, -1, e.n_skip == 0 ? 0 : 1};
    stages[n_st++] = {true, +1, e.n_skip};
  }
  // The interpolated samples of a step (interpolate, evaluate, keep) only
  // touch that trace's skipped samples, which the next steps of the stage do
  // not read; they run on the side stream, overlapping the next step, with
  // their maps and buffers double-buffered by step parity and their own
  // split scratch. A step waits for the side work of the step two before it
  // (which used the same buffers); every stage ends with a join.
  if (!c->side_stream) {
    cudaError_t r = cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking);
    for (int k = 0; r == cudaSuccess && k < 4; ++k)
      r = cudaEventCreateWithFlags(&c->side_ev[k], cudaEventDisableTiming);
    if (r != cudaSuccess) return tt_cuda_check(c, r, "side stream");
  }
  cudaStream_t s2 = c->side_stream;
  cudaEvent_t* fork_ev = c->side_ev;      // [parity]: main -> side
  cudaEvent_t* join_ev = c->side_ev + 2;  // [parity]: side work of that parity done
  bool side_busy[2] = {false, false};
  int* map_est = c->best_idx;
  // compact rows and slot map of the evaluation that passes over the own best:
  // the second trial buffers, which no step uses before its second generation
  float* cth = c->trial[1];
  int* cslot = reinterpret_cast<int*>(c->tfit[1]);
  int* map_skp2[2] = {c->slots, c->slots + c->n_dom};
  float* th_skp2[2] = {c->imports, c->imports + size_t(c->n_dom) * D};
  float* S_skp2[2] = {c->pol_S, c->pol_bS};
  auto join = [&](int par) -> cudaError_t {
    if (!side_busy[par]) return cudaSuccess;
    side_busy[par] = false;
    return cudaStreamWaitEvent(s, join_ev[par], 0);
  };
  const uint32_t key0 = uint32_t(c->cfg.seed & 0xffffffffull), key1 = uint32_t(c->cfg.seed >> 32);
  for (int si = 0; si < n_st; ++si) {
    const Stage& sg = stages[si];
    const int NP = sg.bf ? e.np_bf : e.np_f, NG = sg.bf ? e.ng_bf : e.ng_f;
    StepGeo g{};
    g.n_m0 = n_m0;
    g.n_t0 = n_t0;
    g.nb = nb;
    g.n_buckets = n_buckets;
    g.init = sg.init;
    g.stride = e.n_skip + 1;
    g.n_est = sg.init < n_t0 ? (n_t0 - sg.init + g.stride - 1) / g.stride : 0;
    g.n_skp = n_t0 - g.n_est;
    g.dirn = sg.dirn;
    const int n_est_loc = n_buckets * g.n_est, n_skp_loc = n_buckets * g.n_skp;
    for (int step = 0; step < nb; ++step) {
      g.tb = sg.dirn > 0 ? step : nb - 1 - step;
      int active = 0;  // traces of this step (buckets long enough)
      for (int b = 0; b < n_buckets; ++b) active += g.tb < std::min(nb, n_m0 - b * nb);
      if (active == 0) continue;
      const int par = step & 1;
      STEP(join(par), "ens join");
      int* map_skp = map_skp2[par];
      float* th_skp = th_skp2[par];
      float* S_skp = S_skp2[par];
      if (g.n_est > 0) {
        const uint32_t gen0 = uint32_t(si + 1) * 65536u;
        k_ens_init<<<blocks((long long)n_est_loc * NP), 256, 0, s>>>(
            g, sg.bf ? 1 : 0, NP, D, map_est, bth, bS, c->pop, c->fit, cth, cslot, key0, key1,
            gen0, c->bounds, c->bounds + D, c->cfg.adapt ? c->jade_mu : nullptr, c->jade_na,
            c->cfg.F, c->cfg.CR);
        STEP(c->counted(cudaGetLastError()), "ens init");
        tt::EvalArgs ea = c->eval_args(c->pop, NP, c->fit);
        ea.n_dom = n_est_loc;
        ea.dom_map = map_est;
        if (sg.bf) {  // the own best's semblance is known: NP - 1 pairs per sample
          ea.theta = cth;
          ea.P = NP - 1;
          ea.slots = cslot;
          ea.np_out = NP;
        }
        STEP(c->semblance(ea, s, false), "ens evaluate");
        calls += (unsigned long long)active * g.n_est * (sg.bf ? NP - 1 : NP);
        int cur = 0;
        bool pending = false;
        for (int gi = 1; gi <= NG; ++gi) {
          tt::DeArgs a = tt_make_de_args(c, int(gen0) + gi);
          a.n_dom = n_est_loc;
          a.NP = NP;
          a.dom_map = map_est;
          a.pop = c->pop;
          a.fit = c->fit;
          a.trial = pending ? c->trial[cur ^ 1] : nullptr;
          a.tfit = pending ? c->tfit[cur ^ 1] : nullptr;
          a.next = c->trial[cur];
          STEP(c->counted(tt::launch_de_step(a, s)), "ens de step");
          tt::EvalArgs et = c->eval_args(c->trial[cur], NP, c->tfit[cur]);
          et.n_dom = n_est_loc;
          et.dom_map = map_est;
          STEP(c->semblance(et, s, false), "ens evaluate trial");
          calls += (unsigned long long)active * g.n_est * NP;
          pending = true;
          cur ^= 1;
        }
        if (pending) {
          tt::DeArgs a = tt_make_de_args(c, int(gen0) + NG + 1);
          a.sel_gen = int(gen0) + NG;  // select-only: the last trial
          a.n_dom = n_est_loc;
          a.NP = NP;
          a.dom_map = map_est;
          a.pop = c->pop;
          a.fit = c->fit;
          a.trial = c->trial[cur ^ 1];
          a.tfit = c->tfit[cur ^ 1];
          a.ens_best_th = bth;  // the bests written by the selecting kernel
          a.ens_best_S = bS;
          STEP(c->counted(tt::launch_de_step(a, s)), "ens select");
        } else {
          k_ens_update<<<blocks((long long)n_est_loc * 32), 256, 0, s>>>(
              n_est_loc, NP, D, map_est, c->pop, c->fit, bth, bS);
          STEP(c->counted(cudaGetLastError()), "ens update");
        }
      }
      if (g.n_skp > 0 && g.n_est > 0) {
        STEP(cudaEventRecord(fork_ev[par], s), "ens fork");
        STEP(cudaStreamWaitEvent(s2, fork_ev[par], 0), "ens fork");
        k_ens_interp<<<blocks(n_skp_loc), 256, 0, s2>>>(g, D, map_skp, bth, th_skp);
        STEP(c->counted(cudaGetLastError()), "ens interpolate");
        tt::EvalArgs ei = c->eval_args(th_skp, 1, S_skp);
        ei.n_dom = n_skp_loc;
        ei.dom_map = map_skp;
        ei.split_part = c->split_part2;
        ei.split_part_d = c->split_part_d2;
        ei.split_ticket = c->split_ticket2;
        STEP(c->semblance(ei, s2, false), "ens evaluate interpolated");
        calls += (unsigned long long)active * g.n_skp;
        k_ens_keep<<<blocks(n_skp_loc), 256, 0, s2>>>(n_skp_loc, D, map_skp, th_skp, S_skp, bth,
                                                      bS);
        STEP(c->counted(cudaGetLastError()), "ens keep");
        STEP(cudaEventRecord(join_ev[par], s2), "ens join");
        side_busy[par] = true;
      }
    }
    STEP(join(0), "ens join");
    STEP(join(1), "ens join");
  }
#undef STEP
  *n_calls = calls;
  return TT_OK;
}

bool same_cfg(const tt_ens_cfg& a, const tt_ens_cfg& b) {
  return a.np_f == b.np_f && a.ng_f == b.ng_f && a.np_bf == b.np_bf && a.ng_bf == b.ng_bf &&
         a.n_skip == b.n_skip && a.n_cycle == b.n_cycle && a.n_bucket == b.n_bucket;
}

}  // namespace

extern "C" tt_status tt_ens_search(tt_ctx* c, const tt_ens_cfg* e, float* best_theta,
                                   float* best_S, uint64_t* n_evals, void* stream) {
  if (!c) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (!e) return tt_fail(c, TT_ERR_INVALID_ARG, "ens cfg is NULL");
  if (!c->has_cfg) return tt_fail(c, TT_ERR_INVALID_ARG, "context was created without a cfg");
  if (c->n_m0 <= 0 || c->n_t0 <= 0 || (long long)c->n_m0 * c->n_t0 != c->n_dom)
    return tt_fail(c, TT_ERR_INVALID_ARG, "the problem has no (m0, t0) grid");
  if (e->np_f < 4 || e->np_bf < 4 || e->np_f > c->cfg.np || e->np_bf > c->cfg.np)
    return tt_fail(c, TT_ERR_INVALID_ARG,
                   "np_f and np_bf must be in [4, the context's np = %d]", c->cfg.np);
  if (e->ng_f < 0 || e->ng_bf < 0 || e->n_skip < 0 || e->n_cycle < 0 || e->n_cycle > 64 ||
      e->n_bucket < 1)
    return tt_fail(c, TT_ERR_INVALID_ARG, "bad ENS settings");
  if (!best_theta || !best_S) return tt_fail(c, TT_ERR_INVALID_ARG, "NULL output array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long calls = 0;
  if (!c->use_graph || c->profiling) {
    tt_status st = ens_body(c, *e, best_theta, best_S, s, &calls);
    if (st == TT_OK && n_evals) *n_evals = calls;
    return st;
  }
  if (!c->ens_exec || !same_cfg(c->ens_cfg, *e)) {
    if (c->ens_exec) {
      cudaGraphExecDestroy(c->ens_exec);
      c->ens_exec = nullptr;
    }
    if (!c->cap_stream) {
      cudaError_t r = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
      if (r != cudaSuccess) return tt_cuda_check(c, r, "capture stream");
    }
    const unsigned long long l0 = c->n_launch, s0 = c->n_sem;
    const double t0 = c->trace_evals;
    cudaError_t r = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (r != cudaSuccess) return tt_cuda_check(c, r, "begin capture");
    tt_status st = ens_body(c, *e, c->out_th, c->out_S, c->cap_stream, &c->ens_calls);
    cudaGraph_t graph = nullptr;
    r = cudaStreamEndCapture(c->cap_stream, &graph);
    if (st == TT_OK && r != cudaSuccess) st = tt_cuda_check(c, r, "end capture");
    if (st == TT_OK) {
      r = cudaGraphInstantiate(&c->ens_exec, graph, 0);
      if (r != cudaSuccess) {
        c->ens_exec = nullptr;
        st = tt_cuda_check(c, r, "graph instantiate");
      }
    }
    if (graph) cudaGraphDestroy(graph);
    c->ens_launch = c->n_launch - l0;
    c->ens_sem = c->n_sem - s0;
    c->ens_trace_evals = c->trace_evals - t0;
    c->n_launch = l0;
    c->n_sem = s0;
    c->trace_evals = t0;
    if (st != TT_OK) return st;
    c->ens_cfg = *e;
  }
  cudaError_t r = cudaGraphLaunch(c->ens_exec, s);
  if (r == cudaSuccess)
    r = cudaMemcpyAsync(best_theta, c->out_th, size_t(c->n_dom) * c->D * 4,
                        cudaMemcpyDeviceToDevice, s);
  if (r == cudaSuccess)
    r = cudaMemcpyAsync(best_S, c->out_S, size_t(c->n_dom) * 4, cudaMemcpyDeviceToDevice, s);
  if (r != cudaSuccess) return tt_cuda_check(c, r, "graph launch");
  c->n_launch += c->ens_launch;
  c->n_sem += c->ens_sem;
  c->trace_evals += c->ens_trace_evals;
  if (n_evals) *n_evals = c->ens_calls;
  return TT_OK;
}
