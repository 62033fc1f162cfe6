// Host driver of the whole search: the JADE loop of Sec. 2.1 (p = 1, fixed
// F and CR) over every domain at once, the neighbour exchange of Sec. 3.3
// after every exch_every-th selection, and the gradient polish. Everything
// is enqueued on one stream; nothing synchronises. The selection of
// generation g is fused into the step that mutates generation g+1 unless an
// exchange must run between them.
#include <utility>

#include "tt_internal.cuh"

tt::DeArgs tt_make_de_args(const tt_ctx* c, int gen);

namespace {

tt_status polish_impl(tt_ctx* c, const float* theta_in, float* theta_out, float* S_out,
                      int steps, float lr, cudaStream_t s) {
  const int n = c->n_dom, D = c->D;
  if (n == 0) return TT_OK;
  const float* lo = c->bounds;
  const float* hi = c->bounds ? c->bounds + D : nullptr;
  if (!lo) return tt_fail(c, TT_ERR_INVALID_ARG, "polish needs parameter bounds (a cfg)");
  tt_status st = tt_cuda_check(
      c, cudaMemcpyAsync(c->pol_th, theta_in, size_t(n) * D * 4, cudaMemcpyDeviceToDevice, s),
      "polish copy");
  if (st != TT_OK) return st;
  for (int k = 0; k < steps; ++k) {
    tt::EvalArgs a = c->eval_args(c->pol_th, 1, c->pol_S);
    a.dS = c->pol_g;
    st = tt_cuda_check(c, c->semblance(a, s, true), "polish gradient");
    if (st != TT_OK) return st;
    st = tt_cuda_check(c, c->counted(tt::launch_polish_update(n, D, c->pol_th, c->pol_g, c->pol_S,
                                                   c->pol_bth, c->pol_bS, lo, hi, lr, k == 0, 0,
                                                   s)),
                       "polish update");
    if (st != TT_OK) return st;
  }
  tt::EvalArgs a = c->eval_args(c->pol_th, 1, c->pol_S);
  st = tt_cuda_check(c, c->semblance(a, s, false), "polish evaluation");
  if (st != TT_OK) return st;
  st = tt_cuda_check(c, c->counted(tt::launch_polish_update(n, D, c->pol_th, c->pol_g,
                                                            c->pol_S, c->pol_bth, c->pol_bS, lo,
                                                            hi, lr, steps == 0, 1, s)),
                     "polish final");
  if (st != TT_OK) return st;
  st = tt_cuda_check(c, cudaMemcpyAsync(theta_out, c->pol_bth, size_t(n) * D * 4,
                                        cudaMemcpyDeviceToDevice, s),
                     "polish copy out");
  if (st != TT_OK) return st;
  if (S_out)
    st = tt_cuda_check(c, cudaMemcpyAsync(S_out, c->pol_bS, size_t(n) * 4,
                                          cudaMemcpyDeviceToDevice, s),
                       "polish copy out");
  return st;
}

}  // namespace

extern "C" tt_status tt_polish(tt_ctx* c, float* theta, float* S, int32_t steps, float lr,
                               void* stream) {
  if (!c) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (steps < 0) return tt_fail(c, TT_ERR_INVALID_ARG, "steps < 0");
  if (c->n_dom > 0 && !theta) return tt_fail(c, TT_ERR_INVALID_ARG, "theta is NULL");
  return polish_impl(c, theta, theta, S, steps, lr, static_cast<cudaStream_t>(stream));
}

namespace {

// Enqueue the whole search on `s`, writing the result to (best_theta, best_S).
// `slab` (may be NULL) makes it one slab of a sharded line.
tt_status search_body(tt_ctx* c, float* best_theta, float* best_S, cudaStream_t s,
                      unsigned long long* n_evals, const tt_slab* slab = nullptr) {
  const tt_de_cfg& cfg = c->cfg;
  const int NP = cfg.np, NG = cfg.ng;
  const bool grid = cfg.exch_every > 0 && c->n_m0 > 0 && c->n_t0 > 0 &&
                    (long long)c->n_m0 * c->n_t0 == c->n_dom;
  const int base = slab ? int(slab->dom_base) : 0;
  const bool prev = slab && slab->has_prev, next = slab && slab->has_next;
  // imports per exchange: the grid's inner edges both ways, plus one per
  // domain of an edge row with a neighbouring slab
  const unsigned long long edges =
      grid ? 2ull * ((unsigned long long)c->n_m0 * (c->n_t0 - 1) +
                     (unsigned long long)c->n_t0 * (c->n_m0 - 1)) +
                 (unsigned long long)c->n_t0 * ((prev ? 1 : 0) + (next ? 1 : 0))
           : 0ull;
  unsigned long long evals = 0;
  tt_status st = TT_OK;
#define STEP(expr, what)                                         \
  do {                                                           \
    st = tt_cuda_check(c, (expr), what);                         \
    if (st != TT_OK) return st;                                  \
  } while (0)
  auto de_args = [&](int gen) {
    tt::DeArgs d = tt_make_de_args(c, gen);
    d.dom_base = base;
    return d;
  };
  // Evaluate population th [n_dom][NP] into fit, in member order when the
  // option is on: the order kernel writes the reordered copy and its slot map
  // to the free trial buffers (tmp, tmp_fit), and the evaluation scatters
  // each member's semblance back to its own slot.
  const bool long_apertures = c->sum_N >= tt::kOrderMinMeanAperture * double(c->n_dom);
  const bool order = (c->member_order == 1 || (c->member_order == 2 && long_apertures)) &&
                     NP > 1 && NP <= tt::kOrderMaxP;
  auto evaluate = [&](const float* th, float* fit, float* tmp, float* tmp_fit) -> tt_status {
    if (!order) return tt_cuda_check(c, c->semblance(c->eval_args(th, NP, fit), s, false),
                                     "evaluate");
    int* map = reinterpret_cast<int*>(tmp_fit);
    tt_status r = tt_cuda_check(
        c, c->counted(tt::launch_member_order(c->eval_args(th, NP, nullptr), tmp, map, s)),
        "member order");
    if (r != TT_OK) return r;
    tt::EvalArgs ea = c->eval_args(tmp, NP, fit);
    ea.slots = map;
    ea.np_out = NP;
    return tt_cuda_check(c, c->semblance(ea, s, false), "evaluate");
  };
  // generation 0: initialise and evaluate
  tt::DeArgs a = de_args(0);
  a.pop = c->pop;
  a.fit = c->fit;
  STEP(c->counted(tt::launch_de_step(a, s)), "init");
  st = evaluate(c->pop, c->fit, c->trial[0], c->tfit[0]);
  if (st != TT_OK) return st;
  evals += (unsigned long long)NP * c->n_dom;
  int cur = 0;            // trial buffer written by the next mutation
  bool pending = false;   // trial[cur ^ 1] awaits selection
  for (int g = 1; g <= NG; ++g) {
    a = de_args(g);
    a.pop = c->pop;
    a.fit = c->fit;
    a.trial = pending ? c->trial[cur ^ 1] : nullptr;
    a.tfit = pending ? c->tfit[cur ^ 1] : nullptr;
    a.next = c->trial[cur];
    STEP(c->counted(tt::launch_de_step(a, s)), "de step");
    // the selection above has consumed trial[cur ^ 1]: free for the reordered copy
    st = evaluate(c->trial[cur], c->tfit[cur], c->trial[cur ^ 1], c->tfit[cur ^ 1]);
    if (st != TT_OK) return st;
    evals += (unsigned long long)NP * c->n_dom;
    pending = true;
    cur ^= 1;
    if (grid && g % cfg.exch_every == 0) {
      a = de_args(g);
      a.sel_gen = g;  // select-only: the trial of this generation
      a.pop = c->pop;
      a.fit = c->fit;
      a.trial = c->trial[cur ^ 1];
      a.tfit = c->tfit[cur ^ 1];
      STEP(c->counted(tt::launch_de_step(a, s)), "select");
      pending = false;
      STEP(c->counted(tt::launch_best_snapshot(c->n_dom, NP, c->D, c->pop, c->fit, c->snap,
                                                nullptr, s)),
           "snapshot");
      if (prev || next) {
        // the edge rows out, the neighbouring slabs' rows in
        const size_t row = size_t(c->n_t0) * c->D * sizeof(float);
        STEP(cudaMemcpyAsync(slab->send_first, c->snap, row, cudaMemcpyDeviceToDevice, s),
             "send first row");
        STEP(cudaMemcpyAsync(slab->send_last, c->snap + size_t(c->n_m0 - 1) * c->n_t0 * c->D,
                             row, cudaMemcpyDeviceToDevice, s),
             "send last row");
        if (slab->exchange(slab->user, g, s) != 0)
          return tt_fail(c, TT_ERR_INVALID_ARG, "slab exchange callback failed at gen %d", g);
      }
      STEP(c->counted(tt::launch_exchange_plan(c->n_m0, c->n_t0, NP, c->D, c->snap, c->pop,
                                               c->fit, c->imports, c->slots, s,
                                               prev ? slab->recv_prev : nullptr,
                                               next ? slab->recv_next : nullptr)),
           "exchange");
      tt::EvalArgs ea = c->eval_args(c->imports, 4, c->fit);
      ea.slots = c->slots;
      ea.np_out = NP;
      STEP(c->semblance(ea, s, false), "evaluate imports");
      evals += edges;
    }
  }
  if (pending) {
    a = de_args(NG + 1);
    a.sel_gen = NG;  // select-only: the last trial
    a.pop = c->pop;
    a.fit = c->fit;
    a.trial = c->trial[cur ^ 1];
    a.tfit = c->tfit[cur ^ 1];
    STEP(c->counted(tt::launch_de_step(a, s)), "final select");
  }
  STEP(c->counted(tt::launch_best_snapshot(c->n_dom, NP, c->D, c->pop, c->fit, best_theta,
                                           best_S, s)),
       "best");
#undef STEP
  if (cfg.polish_steps > 0) {
    st = polish_impl(c, best_theta, best_theta, best_S, cfg.polish_steps, cfg.polish_lr, s);
    if (st != TT_OK) return st;
    evals += (unsigned long long)c->n_dom * (cfg.polish_steps + 1);
  }
  *n_evals = evals;
  return TT_OK;
}

}  // namespace

extern "C" tt_status tt_search(tt_ctx* c, float* best_theta, float* best_S, uint64_t* n_evals,
                               void* stream) {
  if (!c) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->has_cfg) return tt_fail(c, TT_ERR_INVALID_ARG, "context was created without a cfg");
  if (c->n_dom > 0 && (!best_theta || !best_S))
    return tt_fail(c, TT_ERR_INVALID_ARG, "NULL output array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long evals = 0;
  if (!c->use_graph || c->profiling || c->n_dom == 0) {
    tt_status st = search_body(c, best_theta, best_S, s, &evals);
    if (st == TT_OK && n_evals) *n_evals = evals;
    return st;
  }
  if (!c->graph_exec) {
    // capture once on a private stream into context-owned outputs; the
    // counters advanced during capture are moved to the per-replay deltas
    if (!c->cap_stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return tt_cuda_check(c, e, "capture stream");
    }
    const unsigned long long l0 = c->n_launch, s0 = c->n_sem;
    const double t0 = c->trace_evals;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return tt_cuda_check(c, e, "begin capture");
    tt_status st = search_body(c, c->out_th, c->out_S, c->cap_stream, &c->g_evals);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (st == TT_OK && e != cudaSuccess) st = tt_cuda_check(c, e, "end capture");
    if (st == TT_OK) {
      e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
      if (e != cudaSuccess) {
        c->graph_exec = nullptr;
        st = tt_cuda_check(c, e, "graph instantiate");
      }
    }
    if (graph) cudaGraphDestroy(graph);
    c->g_launch = c->n_launch - l0;
    c->g_sem = c->n_sem - s0;
    c->g_trace_evals = c->trace_evals - t0;
    c->n_launch = l0;
    c->n_sem = s0;
    c->trace_evals = t0;
    if (st != TT_OK) return st;
  }
  cudaError_t e = cudaGraphLaunch(c->graph_exec, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(best_theta, c->out_th, size_t(c->n_dom) * c->D * 4,
                        cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(best_S, c->out_S, size_t(c->n_dom) * 4, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return tt_cuda_check(c, e, "graph launch");
  c->n_launch += c->g_launch;
  c->n_sem += c->g_sem;
  c->trace_evals += c->g_trace_evals;
  if (n_evals) *n_evals = c->g_evals;
  return TT_OK;
}

extern "C" tt_status tt_search_slab(tt_ctx* c, const tt_slab* slab, float* best_theta,
                                    float* best_S, uint64_t* n_evals, void* stream) {
  if (!c) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->has_cfg) return tt_fail(c, TT_ERR_INVALID_ARG, "context was created without a cfg");
  if (!slab) return tt_fail(c, TT_ERR_INVALID_ARG, "slab is NULL");
  if (c->n_m0 <= 0 || c->n_t0 <= 0 || (long long)c->n_m0 * c->n_t0 != c->n_dom)
    return tt_fail(c, TT_ERR_INVALID_ARG, "a slab needs the (m0, t0) grid of its domains");
  if (slab->dom_base < 0 || slab->dom_base + c->n_dom > 0x7fffffffll)
    return tt_fail(c, TT_ERR_INVALID_ARG, "dom_base out of range");
  const bool edges = c->cfg.exch_every > 0 && (slab->has_prev || slab->has_next);
  if (edges && (!slab->exchange || !slab->send_first || !slab->send_last ||
                (slab->has_prev && !slab->recv_prev) || (slab->has_next && !slab->recv_next)))
    return tt_fail(c, TT_ERR_INVALID_ARG, "a slab with neighbours needs exchange and its rows");
  if (!best_theta || !best_S) return tt_fail(c, TT_ERR_INVALID_ARG, "NULL output array");
  unsigned long long evals = 0;
  tt_status st = search_body(c, best_theta, best_S, static_cast<cudaStream_t>(stream), &evals,
                             slab);
  if (st == TT_OK && n_evals) *n_evals = evals;
  return st;
}
