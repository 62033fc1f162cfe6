// Context life cycle: argument validation, the padded device copy of the
// gathers, the per-aperture geometry table and the search scratch.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>

#include "tt_internal.cuh"

static thread_local std::string g_create_err = "no error";
static constexpr size_t kStageBytes = size_t(32) << 20;  // bf16 reload staging

tt_status tt_fail(tt_ctx* ctx, tt_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf; else g_create_err = buf;
  return code;
}

tt_status tt_cuda_check(tt_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TT_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return tt_fail(ctx, TT_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
  }
  return tt_fail(ctx, TT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char* tt_last_error(const tt_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

extern "C" const char* tt_version(void) { return "libtt 0.1 sm_103a"; }

tt::EvalArgs tt_ctx::eval_args(const float* theta, int P, float* S) const {
  tt::EvalArgs a{};
  a.traces = traces;
  a.ap_tab = ap_tab;
  a.ap_ptr = ap_ptr;
  a.g_inv_dt = g_inv_dt;
  a.dom_it0 = dom_it0;
  a.dom_group = dom_group;
  a.n_dom = n_dom;
  a.P = P;
  a.D = D;
  a.op = op;
  a.W = W;
  a.storage = storage;
  a.umax = float(ns + W);
  a.theta = theta;
  a.S = S;
  a.dS = nullptr;
  a.slots = nullptr;
  a.np_out = 0;
  a.dom_map = nullptr;
  a.kernel = kernel;
  a.block = block;
  a.split = split ? 1 : 0;
  a.split_blocks = 1;
  a.n_sm = n_sm;
  a.split_part = split_part;
  a.split_part_d = split_part_d;
  a.split_ticket = split_ticket;
  a.queue = queue;
  return a;
}

void tt_ctx_drop_graph(tt_ctx* c) {
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  if (c->ens_exec) {
    cudaGraphExecDestroy(c->ens_exec);
    c->ens_exec = nullptr;
  }
}

extern "C" tt_status tt_ctx_set_option(tt_ctx* c, int32_t option, int64_t value) {
  if (!c) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  switch (option) {
    case TT_OPT_KERNEL:
      if (value != TT_KERNEL_PACKED && value != TT_KERNEL_PERSISTENT && value != TT_KERNEL_SCALAR)
        return tt_fail(c, TT_ERR_INVALID_ARG, "unknown kernel variant %lld", (long long)value);
      c->kernel = int(value);
      break;
    case TT_OPT_BLOCK:
      if (value != 128 && value != 256)
        return tt_fail(c, TT_ERR_INVALID_ARG, "block must be 128 or 256");
      c->block = int(value);
      break;
    case TT_OPT_SEARCH_GRAPH:
      c->use_graph = value != 0;
      break;
    case TT_OPT_SPLIT:
      c->split = value != 0;
      break;
    case TT_OPT_MEMBER_ORDER:
      if (value < 0 || value > 2)
        return tt_fail(c, TT_ERR_INVALID_ARG, "member order must be 0, 1 or 2 (automatic)");
      c->member_order = int(value);
      break;
    case TT_OPT_SPLIT_MAX_PAIRS:
    case TT_OPT_SM_COUNT:
      return tt_fail(c, TT_ERR_INVALID_ARG, "option %d is read only", option);
    default:
      return tt_fail(c, TT_ERR_INVALID_ARG, "unknown option %d", option);
  }
  tt_ctx_drop_graph(c);
  return TT_OK;
}

extern "C" tt_status tt_ctx_get_option(const tt_ctx* c, int32_t option, int64_t* value) {
  if (!c || !value) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx or value is NULL");
  switch (option) {
    case TT_OPT_KERNEL: *value = c->kernel; return TT_OK;
    case TT_OPT_BLOCK: *value = c->block; return TT_OK;
    case TT_OPT_SEARCH_GRAPH: *value = c->use_graph ? 1 : 0; return TT_OK;
    case TT_OPT_SPLIT: *value = c->split ? 1 : 0; return TT_OK;
    case TT_OPT_MEMBER_ORDER: *value = c->member_order; return TT_OK;
    case TT_OPT_SPLIT_MAX_PAIRS: *value = (int64_t)c->n_sm * tt::kSplitUnitsPerSm * 64; return TT_OK;
    case TT_OPT_SM_COUNT: *value = c->n_sm; return TT_OK;
  }
  return tt_fail(nullptr, TT_ERR_INVALID_ARG, "unknown option %d", option);
}

constexpr float kPersistentMargin = 0.03f;

extern "C" tt_status tt_ctx_autotune(tt_ctx* c, const float* theta, int32_t P, float* S,
                                     float* times_ms, void* stream) {
  if (!c) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (P < 1) return tt_fail(c, TT_ERR_INVALID_ARG, "P must be >= 1");
  if (c->n_dom > 0 && (!theta || !S)) return tt_fail(c, TT_ERR_INVALID_ARG, "NULL array");
  static const int cand[TT_N_TUNE_CANDIDATES][2] = {
      {TT_KERNEL_PACKED, 256},     {TT_KERNEL_PACKED, 128}, {TT_KERNEL_PERSISTENT, 256},
      {TT_KERNEL_PERSISTENT, 128}, {TT_KERNEL_SCALAR, 256}, {TT_KERNEL_SCALAR, 128}};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaError_t r = cudaEventCreate(&e0);
  if (r == cudaSuccess) r = cudaEventCreate(&e1);
  if (r != cudaSuccess) return tt_cuda_check(c, r, "event create");
  float t[TT_N_TUNE_CANDIDATES] = {};
  tt_status st = TT_OK;
  for (int i = 0; i < TT_N_TUNE_CANDIDATES && st == TT_OK; ++i) {
    tt::EvalArgs a = c->eval_args(theta, P, S);
    a.kernel = cand[i][0];
    a.block = cand[i][1];
    r = tt::launch_semblance(a, s);  // warm-up
    if (r == cudaSuccess) r = cudaEventRecord(e0, s);
    for (int k = 0; k < 3 && r == cudaSuccess; ++k) r = tt::launch_semblance(a, s);
    if (r == cudaSuccess) r = cudaEventRecord(e1, s);
    if (r == cudaSuccess) r = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
    if (r != cudaSuccess) {
      st = tt_cuda_check(c, r, "autotune");
      break;
    }
    t[i] = ms / 3.f;
    if (times_ms) times_ms[i] = t[i];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TT_OK) return st;
  int best = 0;
  for (int i = 1; i < TT_N_TUNE_CANDIDATES; ++i)
    if (t[i] < t[best]) best = i;
  // The trial population is usually a first generation, whose windows are
  // scattered. Once a search's populations converge, the warps of a
  // grid-mapped block (adjacent domains) read the same trace lines at the
  // same time and share them in L1, which the work queue's scattered unit
  // order loses; so the persistent form is kept only when it wins the trial
  // by more than kPersistentMargin.
  if (cand[best][0] == TT_KERNEL_PERSISTENT) {
    int alt = -1;
    for (int i = 0; i < TT_N_TUNE_CANDIDATES; ++i)
      if (cand[i][0] != TT_KERNEL_PERSISTENT && (alt < 0 || t[i] < t[alt])) alt = i;
    if (alt >= 0 && t[alt] <= t[best] * (1.f + kPersistentMargin)) best = alt;
  }
  c->kernel = cand[best][0];
  c->block = cand[best][1];
  tt_ctx_drop_graph(c);
  return TT_OK;
}

cudaError_t tt_ctx::semblance(const tt::EvalArgs& a, cudaStream_t s, bool grad) {
  const bool timed = profiling && ev_used + 2 <= ev.size();
  if (timed) cudaEventRecord(ev[ev_used], s);
  cudaError_t e = grad ? tt::launch_semblance_grad(a, s) : tt::launch_semblance(a, s);
  if (timed) {
    cudaEventRecord(ev[ev_used + 1], s);
    ev_used += 2;
  }
  ++n_launch;
  ++n_sem;
  // a mapped (subset) launch is counted at the mean aperture size
  trace_evals += double(a.P) * (a.dom_map ? sum_N / double(n_dom > 0 ? n_dom : 1) * a.n_dom
                                          : sum_N);
  return e;
}

extern "C" tt_status tt_ctx_profile(tt_ctx* c, int32_t enable) {
  if (!c) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (enable && c->ev.empty()) {
    c->ev.resize(8192);
    for (auto& e : c->ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return tt_cuda_check(c, r, "event create");
    }
  }
  c->profiling = enable != 0;
  return TT_OK;
}

extern "C" tt_status tt_ctx_stats(tt_ctx* c, tt_stats* out, int32_t reset) {
  if (!c) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  double ms = 0.0;
  if (c->ev_used) {
    cudaError_t r = cudaEventSynchronize(c->ev[c->ev_used - 1]);
    if (r != cudaSuccess) return tt_cuda_check(c, r, "event sync");
    for (size_t i = 0; i < c->ev_used; i += 2) {
      float t = 0.f;
      r = cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]);
      if (r != cudaSuccess) return tt_cuda_check(c, r, "event time");
      ms += t;
    }
  }
  if (out) {
    out->launches = c->n_launch;
    out->semblance_launches = c->n_sem;
    out->trace_evals = c->trace_evals;
    out->semblance_ms = ms;
    out->timed_launches = c->ev_used / 2;
  }
  if (reset) {
    c->n_launch = c->n_sem = 0;
    c->trace_evals = 0;
    c->ev_used = 0;
  }
  return TT_OK;
}

namespace {

enum : int {
  kErrApPtr = 1, kErrApIdx = 2, kErrGroup = 3, kErrDt = 4, kErrIt0 = 5, kErrGeom = 6
};

__device__ void flag(int* err, int code) { atomicCAS(err, 0, code); }

__global__ void k_validate(int n_traces, int G, int n_dom, const float* g_dt, const float* g_m0,
                           const float* g_h0, const int* ap_ptr, const int* ap_idx,
                           long long nnz, const int* dom_it0, const int* dom_group, int* err) {
  long long stride = (long long)gridDim.x * blockDim.x;
  long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long i = i0; i < G; i += stride) {
    if (ap_ptr[i] > ap_ptr[i + 1]) flag(err, kErrApPtr);
    float dt = g_dt[i];
    if (!(dt > 0.f) || !isfinite(dt)) flag(err, kErrDt);
    if (!isfinite(g_m0[i]) || (g_h0 && !isfinite(g_h0[i]))) flag(err, kErrGeom);
  }
  for (long long i = i0; i < nnz; i += stride) {
    int r = ap_idx[i];
    if (r < 0 || r >= n_traces) flag(err, kErrApIdx);
  }
  for (long long i = i0; i < n_dom; i += stride) {
    int g = dom_group[i];
    if (g < 0 || g >= G) flag(err, kErrGroup);
    int it = dom_it0[i];
    if (it < 0 || it >= (1 << 24)) flag(err, kErrIt0);
  }
}

__global__ void k_check_geom(int n, const float* mid, const float* off, int* err) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (!isfinite(mid[i]) || !isfinite(off[i])) flag(err, kErrGeom);
}

// dst rows of `pitch` elements; src rows of `ns` floats; zero padding around.
template <typename T>
__global__ void k_pad_rows(const float* __restrict__ src, T* __restrict__ dst, long long row0,
                           long long rows, int ns, int pitch) {
  long long total = rows * pitch;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    long long r = i / pitch;
    int c = int(i - r * pitch) - tt::kPadFront;
    float v = (c >= 0 && c < ns) ? src[r * ns + c] : 0.f;
    if constexpr (sizeof(T) == 2)
      dst[(row0 + r) * pitch + c + tt::kPadFront] = __float2bfloat16_rn(v);
    else
      dst[(row0 + r) * pitch + c + tt::kPadFront] = v;
  }
}

// One warp per group: aperture entry e of group g -> (dm, dm^2, h^2, row base),
// or for FO-CRS (g_h0 != NULL) -> (dm, dh = h - h0, 0, row base).
__global__ void k_ap_table(int G, const int* ap_ptr, const int* ap_idx, const float* g_m0,
                           const float* g_h0, const float* mid, const float* off, int pitch,
                           float4* tab) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= G) return;
  float m0 = g_m0[warp];
  for (int e = ap_ptr[warp] + lane; e < ap_ptr[warp + 1]; e += 32) {
    int r = ap_idx[e];
    float dm = mid[r] - m0;
    float h = off[r];
    unsigned base = unsigned(r) * unsigned(pitch) + unsigned(tt::kPadFront);
    if (g_h0)
      tab[e] = make_float4(dm, h - g_h0[warp], 0.f, __uint_as_float(base));
    else
      tab[e] = make_float4(dm, dm * dm, h * h, __uint_as_float(base));
  }
}

__global__ void k_inv(int n, const float* x, float* y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = 1.0f / x[i];
}

// blocks of a grid-stride loop over n items: enough to cover them, at most
// 32 blocks per SM of the context's device
int grid_for(const tt_ctx* c, long long n, int block = 256) {
  long long b = (n + block - 1) / block;
  const long long cap = 32ll * c->n_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return int(b);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

void free_ctx(tt_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->traces, c->mid, c->off, c->stage, c->g_inv_dt, c->ap_ptr, c->ap_tab,
                  c->dom_it0, c->dom_group, c->bounds, c->pop, c->fit, c->trial[0],
                  c->trial[1], c->tfit[0], c->tfit[1], c->snap, c->imports, c->slots,
                  c->best_idx, c->pol_th, c->pol_g, c->pol_S, c->pol_bth, c->pol_bS, c->d_err,
                  c->queue, c->split_part, c->split_part_d, c->split_ticket, c->split_part2,
                  c->split_part_d2, c->split_ticket2, c->out_th,
                  c->out_S, c->jade_mu, c->jade_arc, c->jade_F,
                  c->jade_CR, c->jade_na};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto e : c->ev) cudaEventDestroy(e);
  tt_ctx_drop_graph(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  for (cudaEvent_t e : c->side_ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

tt_status fill_traces(tt_ctx* c, const float* src, bool host, cudaStream_t s) {
  const long long n_tr = c->n_traces;
  if (c->storage == TT_STORE_F32) {
    float* dst = static_cast<float*>(c->traces) + tt::kPadFront;
    if (n_tr == 0 || c->ns == 0) return TT_OK;
    cudaError_t e = cudaMemcpy2DAsync(dst, size_t(c->pitch) * 4, src, size_t(c->ns) * 4,
                                      size_t(c->ns) * 4, size_t(n_tr),
                                      host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                      s);
    return tt_cuda_check(c, e, "copy traces");
  }
  // bf16 storage: convert rows in chunks (directly from a device source,
  // through the staging buffer from a host source)
  auto* dst = static_cast<__nv_bfloat16*>(c->traces);
  long long rows_per = host ? (long long)(kStageBytes / (size_t(c->ns) * 4)) : n_tr;
  if (rows_per < 1) rows_per = 1;
  for (long long r0 = 0; r0 < n_tr; r0 += rows_per) {
    long long rows = n_tr - r0 < rows_per ? n_tr - r0 : rows_per;
    const float* from = src + r0 * c->ns;
    if (host) {
      cudaError_t e = cudaMemcpyAsync(c->stage, from, size_t(rows) * c->ns * 4,
                                      cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return tt_cuda_check(c, e, "stage traces");
      from = c->stage;
    }
    k_pad_rows<__nv_bfloat16><<<grid_for(c, rows * c->pitch), 256, 0, s>>>(from, dst, r0, rows,
                                                                        c->ns, c->pitch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tt_cuda_check(c, e, "convert traces");
  }
  return TT_OK;
}

}  // namespace

extern "C" tt_status tt_ctx_create(tt_ctx** out, const tt_gathers* ga, const tt_problem* pr,
                                   const tt_de_cfg* cfg, void* stream) {
  if (!out) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ga || !pr) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "gathers/problem is NULL");
  if (ga->n_traces < 0 || ga->ns < 0 || pr->n_groups < 0 || pr->n_dom < 0)
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "negative size");
  if (ga->storage != TT_STORE_F32 && ga->storage != TT_STORE_BF16)
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "storage must be TT_STORE_F32 or TT_STORE_BF16");
  if (pr->op != TT_OP_CMP && pr->op != TT_OP_CRS && pr->op != TT_OP_FOCRS)
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "op must be TT_OP_CMP, TT_OP_CRS or TT_OP_FOCRS");
  if (pr->op == TT_OP_FOCRS && pr->n_groups > 0 && !pr->group_h0)
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "FO-CRS needs group_h0");
  if (pr->half_window < 0 || pr->half_window > TT_MAX_HALF_WINDOW)
    return tt_fail(nullptr, TT_ERR_UNSUPPORTED, "half_window %d outside 0..%d", pr->half_window,
                   TT_MAX_HALF_WINDOW);
  if (ga->n_traces > 0 && ga->ns > 0 && (!ga->traces || !ga->mid || !ga->off))
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "NULL trace/geometry pointer");
  if (pr->n_groups > 0 && (!pr->group_m0 || !pr->group_dt || !pr->ap_ptr))
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "NULL group array");
  if (pr->n_dom > 0 && (!pr->dom_it0 || !pr->dom_group || pr->n_groups == 0))
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "NULL domain array or no groups");
  if (pr->n_m0 < 0 || pr->n_t0 < 0)
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "negative exchange grid");
  long long pitch = tt::padded_pitch(ga->ns);
  if ((long long)ga->n_traces * pitch >= (1ll << 32))
    return tt_fail(nullptr, TT_ERR_UNSUPPORTED, "padded trace buffer exceeds 2^32 samples");
  const int D = tt::op_dim(pr->op);
  if (cfg) {
    if (cfg->np < 4 || cfg->np > 1024)
      return tt_fail(nullptr, TT_ERR_INVALID_ARG, "np %d outside 4..1024", cfg->np);
    if (cfg->ng < 0) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ng < 0");
    if (!(cfg->F >= 0.f && cfg->F <= 2.f) || !(cfg->CR >= 0.f && cfg->CR <= 1.f))
      return tt_fail(nullptr, TT_ERR_INVALID_ARG, "F must be in [0,2], CR in [0,1]");
    for (int d = 0; d < D; ++d)
      if (!(cfg->lo[d] <= cfg->hi[d]) || !std::isfinite(cfg->lo[d]) || !std::isfinite(cfg->hi[d]))
        return tt_fail(nullptr, TT_ERR_INVALID_ARG, "bad bounds in dimension %d", d);
    if (cfg->exch_every < 0 || cfg->polish_steps < 0 || !std::isfinite(cfg->polish_lr))
      return tt_fail(nullptr, TT_ERR_INVALID_ARG, "bad exchange/polish settings");
    if (cfg->adapt != 0 && cfg->adapt != 1)
      return tt_fail(nullptr, TT_ERR_INVALID_ARG, "adapt must be 0 or 1");
    if (cfg->adapt && !(cfg->F > 0.f && cfg->F <= 1.f))
      return tt_fail(nullptr, TT_ERR_INVALID_ARG, "adaptive search: initial F in (0, 1]");
    if (cfg->adapt && cfg->ng >= (1 << 30) - 1)
      return tt_fail(nullptr, TT_ERR_INVALID_ARG, "adaptive search: ng must be below 2^30 - 1");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tt_ctx* c = new tt_ctx();
  {
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess || c->n_sm < 1) {
      free_ctx(c);
      return tt_cuda_check(nullptr, e != cudaSuccess ? e : cudaErrorInvalidDevice,
                           "query the device's multiprocessor count");
    }
  }
  c->n_traces = ga->n_traces;
  c->ns = ga->ns;
  c->storage = ga->storage;
  c->pitch = int(pitch);
  c->op = pr->op;
  c->W = pr->half_window;
  c->D = D;
  c->n_groups = pr->n_groups;
  c->n_dom = pr->n_dom;
  c->n_m0 = pr->n_m0;
  c->n_t0 = pr->n_t0;
  if (cfg) {
    c->has_cfg = true;
    c->cfg = *cfg;
  }
  tt_status st = TT_OK;
#define TRY(expr, what)                                              \
  do {                                                               \
    st = tt_cuda_check(nullptr, (expr), what);                       \
    if (st != TT_OK) { free_ctx(c); return st; }                     \
  } while (0)
  // group arrays and the aperture size
  int ap0 = 0, apn = 0;
  if (pr->n_groups > 0) {
    TRY(cudaMemcpyAsync(&ap0, pr->ap_ptr, 4, cudaMemcpyDeviceToHost, s), "read ap_ptr[0]");
    TRY(cudaMemcpyAsync(&apn, pr->ap_ptr + pr->n_groups, 4, cudaMemcpyDeviceToHost, s),
        "read ap_ptr[G]");
    TRY(cudaStreamSynchronize(s), "sync");
    if (ap0 != 0 || apn < 0) {
      free_ctx(c);
      return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ap_ptr must start at 0 and end >= 0");
    }
    if (apn > 0 && !pr->ap_idx) {
      free_ctx(c);
      return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ap_idx is NULL");
    }
  }
  c->nnz = apn;
  TRY(dalloc(&c->d_err, 1), "alloc flag");
  TRY(cudaMemsetAsync(c->d_err, 0, 4, s), "clear flag");
  if (pr->n_groups > 0 || pr->n_dom > 0) {
    k_validate<<<grid_for(c, std::max<long long>({(long long)pr->n_groups, c->nnz,
                                               (long long)pr->n_dom})),
                 256, 0, s>>>(ga->n_traces, pr->n_groups, pr->n_dom, pr->group_dt,
                              pr->group_m0, pr->op == TT_OP_FOCRS ? pr->group_h0 : nullptr,
                              pr->ap_ptr, pr->ap_idx, c->nnz, pr->dom_it0, pr->dom_group,
                              c->d_err);
    TRY(cudaGetLastError(), "validate");
  }
  if (ga->n_traces > 0 && ga->ns > 0) {
    k_check_geom<<<grid_for(c, ga->n_traces), 256, 0, s>>>(ga->n_traces, ga->mid, ga->off,
                                                        c->d_err);
    TRY(cudaGetLastError(), "validate geometry");
  }
  int herr = 0;
  TRY(cudaMemcpyAsync(&herr, c->d_err, 4, cudaMemcpyDeviceToHost, s), "read flag");
  TRY(cudaStreamSynchronize(s), "sync validation");
  if (herr) {
    static const char* msg[] = {"", "ap_ptr is not non-decreasing",
                                "ap_idx holds a trace index outside [0, n_traces)",
                                "dom_group holds a group outside [0, n_groups)",
                                "group_dt must be finite and > 0",
                                "dom_it0 must be in [0, 2^24)",
                                "non-finite midpoint or offset"};
    free_ctx(c);
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "%s", msg[herr]);
  }
  // padded traces
  size_t elem = c->storage == TT_STORE_F32 ? 4 : 2;
  size_t tbytes = size_t(c->n_traces) * size_t(c->pitch) * elem;
  TRY(cudaMalloc(&c->traces, tbytes ? tbytes : 16), "alloc traces");
  TRY(cudaMemsetAsync(c->traces, 0, tbytes ? tbytes : 16, s), "clear traces");
  if (c->storage == TT_STORE_BF16) TRY(dalloc(&c->stage, kStageBytes / 4), "alloc staging");
  if (c->n_traces > 0 && c->ns > 0) {
    st = fill_traces(c, ga->traces, false, s);
    if (st != TT_OK) {
      g_create_err = c->err;
      free_ctx(c);
      return st;
    }
  }
  // geometry copies and the aperture table
  TRY(dalloc(&c->mid, c->n_traces), "alloc mid");
  TRY(dalloc(&c->off, c->n_traces), "alloc off");
  if (c->n_traces > 0) {
    TRY(cudaMemcpyAsync(c->mid, ga->mid, size_t(c->n_traces) * 4, cudaMemcpyDeviceToDevice, s),
        "copy mid");
    TRY(cudaMemcpyAsync(c->off, ga->off, size_t(c->n_traces) * 4, cudaMemcpyDeviceToDevice, s),
        "copy off");
  }
  TRY(dalloc(&c->g_inv_dt, c->n_groups), "alloc dt");
  TRY(dalloc(&c->ap_ptr, c->n_groups + 1), "alloc ap_ptr");
  TRY(dalloc(&c->ap_tab, size_t(c->nnz)), "alloc ap_tab");
  TRY(dalloc(&c->dom_it0, c->n_dom), "alloc it0");
  TRY(dalloc(&c->dom_group, c->n_dom), "alloc groups");
  if (c->n_groups > 0) {
    TRY(cudaMemcpyAsync(c->ap_ptr, pr->ap_ptr, size_t(c->n_groups + 1) * 4,
                        cudaMemcpyDeviceToDevice, s), "copy ap_ptr");
    k_inv<<<(c->n_groups + 255) / 256, 256, 0, s>>>(c->n_groups, pr->group_dt, c->g_inv_dt);
    TRY(cudaGetLastError(), "inv dt");
    k_ap_table<<<(c->n_groups * 32 + 255) / 256, 256, 0, s>>>(
        c->n_groups, pr->ap_ptr, pr->ap_idx, pr->group_m0,
        pr->op == TT_OP_FOCRS ? pr->group_h0 : nullptr, ga->mid, ga->off, c->pitch, c->ap_tab);
    TRY(cudaGetLastError(), "aperture table");
  }
  if (c->n_dom > 0) {
    TRY(cudaMemcpyAsync(c->dom_it0, pr->dom_it0, size_t(c->n_dom) * 4, cudaMemcpyDeviceToDevice,
                        s), "copy it0");
    TRY(cudaMemcpyAsync(c->dom_group, pr->dom_group, size_t(c->n_dom) * 4,
                        cudaMemcpyDeviceToDevice, s), "copy groups");
  }
  // sum over domains of the aperture size (for the trace-evaluation counter)
  if (c->n_dom > 0) {
    std::vector<int> hp(size_t(c->n_groups) + 1), hg(size_t(c->n_dom));
    TRY(cudaMemcpyAsync(hp.data(), pr->ap_ptr, hp.size() * 4, cudaMemcpyDeviceToHost, s),
        "read ap_ptr");
    TRY(cudaMemcpyAsync(hg.data(), pr->dom_group, hg.size() * 4, cudaMemcpyDeviceToHost, s),
        "read groups");
    TRY(cudaStreamSynchronize(s), "sync");
    double sn = 0;
    for (int g : hg) sn += hp[g + 1] - hp[g];
    c->sum_N = sn;
  }
  // search scratch
  if (c->has_cfg) {
    size_t nd = size_t(c->n_dom), np = size_t(cfg->np), Dz = size_t(D);
    float hb[2 * TT_MAX_DIM];
    for (int d = 0; d < D; ++d) {
      hb[d] = cfg->lo[d];
      hb[D + d] = cfg->hi[d];
    }
    TRY(dalloc(&c->bounds, 2 * Dz), "alloc bounds");
    TRY(cudaMemcpyAsync(c->bounds, hb, 2 * Dz * 4, cudaMemcpyHostToDevice, s), "copy bounds");
    TRY(dalloc(&c->pop, nd * np * Dz), "alloc pop");
    TRY(dalloc(&c->fit, nd * np), "alloc fit");
    for (int k = 0; k < 2; ++k) {
      TRY(dalloc(&c->trial[k], nd * np * Dz), "alloc trial");
      TRY(dalloc(&c->tfit[k], nd * np), "alloc trial fit");
    }
    TRY(dalloc(&c->snap, nd * Dz), "alloc snapshot");
    TRY(dalloc(&c->imports, nd * 4 * Dz), "alloc imports");
    TRY(dalloc(&c->slots, nd * 4), "alloc slots");
    TRY(dalloc(&c->best_idx, nd), "alloc best");
    if (cfg->adapt) {
      TRY(dalloc(&c->jade_mu, nd * 2), "alloc adaptation");
      TRY(dalloc(&c->jade_na, nd), "alloc adaptation");
      TRY(dalloc(&c->jade_arc, nd * np * Dz), "alloc archive");
      TRY(dalloc(&c->jade_F, nd * np), "alloc adaptation");
      TRY(dalloc(&c->jade_CR, nd * np), "alloc adaptation");
    }
  }
  TRY(dalloc(&c->queue, 1), "alloc queue");
  TRY(dalloc(&c->split_part, size_t(tt::split_part_sets(c->n_sm)) * 64 * tt::kSplitPartStride),
      "alloc split scratch");
  TRY(dalloc(&c->split_part_d, size_t(tt::split_part_sets(c->n_sm)) * 64), "alloc split scratch");
  TRY(dalloc(&c->split_ticket, size_t(tt::split_tickets(c->n_sm))), "alloc split tickets");
  TRY(cudaMemsetAsync(c->split_ticket, 0, size_t(tt::split_tickets(c->n_sm)) * sizeof(unsigned), s),
      "clear split tickets");
  TRY(dalloc(&c->split_part2, size_t(tt::split_part_sets(c->n_sm)) * 64 * tt::kSplitPartStride),
      "alloc split scratch");
  TRY(dalloc(&c->split_part_d2, size_t(tt::split_part_sets(c->n_sm)) * 64), "alloc split scratch");
  TRY(dalloc(&c->split_ticket2, size_t(tt::split_tickets(c->n_sm))), "alloc split tickets");
  TRY(cudaMemsetAsync(c->split_ticket2, 0, size_t(tt::split_tickets(c->n_sm)) * sizeof(unsigned), s),
      "clear split tickets");
  {
    size_t nd = size_t(c->n_dom), Dz = size_t(D);
    TRY(dalloc(&c->out_th, nd * Dz), "alloc search output");
    TRY(dalloc(&c->out_S, nd), "alloc search output");
    TRY(dalloc(&c->pol_th, nd * Dz), "alloc polish");
    TRY(dalloc(&c->pol_g, nd * Dz), "alloc polish");
    TRY(dalloc(&c->pol_S, nd), "alloc polish");
    TRY(dalloc(&c->pol_bth, nd * Dz), "alloc polish");
    TRY(dalloc(&c->pol_bS, nd), "alloc polish");
  }
  TRY(cudaStreamSynchronize(s), "sync create");
#undef TRY
  c->err = "no error";
  *out = c;
  return TT_OK;
}

extern "C" tt_status tt_ctx_load_traces(tt_ctx* c, const float* traces, int32_t host,
                                        void* stream) {
  if (!c) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (!traces && c->n_traces > 0 && c->ns > 0)
    return tt_fail(c, TT_ERR_INVALID_ARG, "traces is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tt_status st = fill_traces(c, traces, host != 0, s);
  if (st != TT_OK) return st;
  return tt_cuda_check(c, cudaStreamSynchronize(s), "sync reload");
}

extern "C" void tt_ctx_destroy(tt_ctx* c) { free_ctx(c); }
