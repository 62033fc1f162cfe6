// Allocation-free semblance evaluation (tt_semblance_eval_noalloc).
//
// For callers that cannot allocate device memory -- a plug-in whose host
// application owns every device buffer and hands it fixed pools, or a
// latency-bound service loop in which cudaMalloc (which may synchronise the
// device and fail under fragmentation) is not allowed after start-up. Such a
// caller cannot create a context, so this entry point works directly on the
// caller's gathers and problem arrays.
//
// Its only scratch -- the per-aperture geometry table and a validation flag
// -- lives in the file-scope device array below: TT_NOALLOC_SCRATCH_BYTES
// (4 MiB) that every GPU which loads the library holds until the process
// exits. Host code may not use the array's name as a device address (in host
// code it names a host-side stand-in), so the first call on each device, with
// that device current, asks the runtime for the array's device address with
// cudaGetSymbolAddress and every later call on that device reuses it; make
// that first call before any stream capture. All calls share the array and
// it keeps the last call's contents: the flag is cleared by every call, the
// table is rewritten, and calls that overlap on the GPU (different streams
// or threads) race on it.
#include <algorithm>
#include <mutex>

#include "tt_internal.cuh"

namespace {

constexpr size_t kScratchBytes = TT_NOALLOC_SCRATCH_BYTES;
constexpr size_t kHeaderBytes = 256;  // validation flag, then padding
constexpr long long kMaxEntries = TT_NOALLOC_MAX_APERTURE_ENTRIES;
static_assert(kHeaderBytes + size_t(kMaxEntries) * sizeof(float4) <= kScratchBytes,
              "table does not fit the scratch array");

static __device__ __align__(256) unsigned char tt_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
tt_status scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return tt_fail(nullptr, TT_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, tt_noalloc_scratch);
    if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "cudaGetSymbolAddress(scratch)");
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return TT_OK;
}

__device__ void raise_flag(int* flag, int code) { atomicCAS(flag, 0, code); }

__global__ void k_na_validate(int n_traces, int G, int n_dom, const float* g_dt,
                              const float* g_m0, const int* ap_ptr, const int* ap_idx,
                              long long nnz, const int* dom_it0, const int* dom_group,
                              const float* mid, const float* off, int* flag) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long i = i0; i < G; i += stride) {
    if (ap_ptr[i] > ap_ptr[i + 1]) raise_flag(flag, 1);
    const float dt = g_dt[i];
    if (!(dt > 0.f) || !isfinite(dt) || !isfinite(g_m0[i])) raise_flag(flag, 2);
  }
  for (long long i = i0; i < nnz; i += stride) {
    const int r = ap_idx[i];
    if (r < 0 || r >= n_traces) raise_flag(flag, 3);
    else if (!isfinite(mid[r]) || !isfinite(off[r])) raise_flag(flag, 2);
  }
  for (long long i = i0; i < n_dom; i += stride) {
    const int g = dom_group[i];
    if (g < 0 || g >= G) raise_flag(flag, 4);
    const int it = dom_it0[i];
    if (it < 0 || it >= (1 << 24)) raise_flag(flag, 5);
  }
}

// One warp per group: entry e -> (dm, dm^2, h^2, trace index).
__global__ void k_na_table(int G, const int* ap_ptr, const int* ap_idx, const float* g_m0,
                           const float* mid, const float* off, float4* tab) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= G) return;
  const float m0 = g_m0[warp];
  for (int e = ap_ptr[warp] + lane; e < ap_ptr[warp + 1]; e += 32) {
    const int r = ap_idx[e];
    const float dm = mid[r] - m0, h = off[r];
    tab[e] = make_float4(dm, dm * dm, h * h, __int_as_float(r));
  }
}

// One (domain, individual) pair per thread, samples read from the caller's
// [n_traces][ns] traces with the record's zero extension done by bounds
// checks (no padded copy).
template <int OP, int W>
__global__ void __launch_bounds__(256)
    k_na_semblance(const float* __restrict__ traces, int ns, const float4* __restrict__ tab,
                   const int* ap_ptr, const float* g_dt, const int* dom_it0,
                   const int* dom_group, int n_dom, int P, const float* theta, float* S) {
  constexpr int K = 2 * W + 1;
  constexpr int D = OP == TT_OP_CMP ? 1 : 3;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)n_dom * P) return;
  const int d = int(q / P);
  const int g = dom_group[d];
  const float inv_dt = 1.0f / g_dt[g];
  const float p0 = float(dom_it0[d]);
  const float* th = theta + q * D;
  const float ca = OP == TT_OP_CMP ? 0.f : th[0] * inv_dt;
  const float cb = OP == TT_OP_CMP ? 0.f : th[1] * inv_dt * inv_dt;
  const float cc = th[D - 1] * inv_dt * inv_dt;
  const float umax = float(ns + W);
  float s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = 0.f;
  float E = 0.f;
  const int e0 = ap_ptr[g], e1 = ap_ptr[g + 1];
  for (int e = e0; e < e1; ++e) {
    const float4 t4 = tab[e];
    const float qv = fmaf(ca, t4.x, p0);
    const float U = fmaf(cb, t4.y, fmaf(cc, t4.z, qv * qv));
    const float u = fminf(sqrtf(U), umax);  // NaN (U < 0) -> umax: all-zero window
    const float fl = truncf(u);
    const float f = u - fl;
    const int j0 = int(fl) - W;
    const float* row = traces + (size_t)__float_as_int(t4.w) * ns;
    float xv[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) {
      const int n = j0 + k;
      xv[k] = (n >= 0 && n < ns) ? __ldg(row + n) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float ak = fmaf(f, xv[k + 1] - xv[k], xv[k]);
      s[k] += ak;
      E = fmaf(ak, ak, E);
    }
  }
  float Q = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) Q = fmaf(s[k], s[k], Q);
  const float N = float(e1 - e0);
  S[q] = (E > 0.f) ? Q / (N * E) : 0.f;
}

using NaFn = void (*)(const float*, int, const float4*, const int*, const float*, const int*,
                      const int*, int, int, const float*, float*);

template <int OP>
NaFn pick(int W) {
  switch (W) {
    case 0: return k_na_semblance<OP, 0>;
    case 1: return k_na_semblance<OP, 1>;
    case 2: return k_na_semblance<OP, 2>;
    case 3: return k_na_semblance<OP, 3>;
    case 4: return k_na_semblance<OP, 4>;
    case 5: return k_na_semblance<OP, 5>;
    case 6: return k_na_semblance<OP, 6>;
    case 7: return k_na_semblance<OP, 7>;
    case 8: return k_na_semblance<OP, 8>;
  }
  return nullptr;
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return int(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

}  // namespace

extern "C" tt_status tt_semblance_eval_noalloc(const tt_gathers* ga, const tt_problem* pr,
                                               const float* theta, int32_t P, float* S,
                                               void* stream) {
  if (!ga || !pr) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "gathers/problem is NULL");
  if (ga->storage != TT_STORE_F32)
    return tt_fail(nullptr, TT_ERR_INVALID_ARG,
                   "the allocation-free path reads float32 traces in place (storage must be "
                   "TT_STORE_F32)");
  if (pr->op == TT_OP_FOCRS)
    return tt_fail(nullptr, TT_ERR_UNSUPPORTED,
                   "the allocation-free path evaluates TT_OP_CMP and TT_OP_CRS only");
  if (pr->op != TT_OP_CMP && pr->op != TT_OP_CRS)
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "op must be TT_OP_CMP or TT_OP_CRS");
  if (pr->half_window < 0 || pr->half_window > TT_MAX_HALF_WINDOW)
    return tt_fail(nullptr, TT_ERR_UNSUPPORTED, "half_window %d outside 0..%d", pr->half_window,
                   TT_MAX_HALF_WINDOW);
  if (ga->n_traces < 0 || ga->ns < 0 || pr->n_groups < 0 || pr->n_dom < 0 || P < 1)
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "negative size or P < 1");
  if (pr->n_dom == 0) return TT_OK;
  if (pr->n_groups == 0 || !pr->group_m0 || !pr->group_dt || !pr->ap_ptr || !pr->dom_it0 ||
      !pr->dom_group || !theta || !S)
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "NULL problem, theta or S array");
  if (ga->n_traces > 0 && (!ga->traces || !ga->mid || !ga->off))
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "NULL trace/geometry pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* scratch = nullptr;
  tt_status st = scratch_address(&scratch);
  if (st != TT_OK) return st;
  int* flag = reinterpret_cast<int*>(scratch);
  float4* tab = reinterpret_cast<float4*>(scratch + kHeaderBytes);
  int ap_end[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(&ap_end[0], pr->ap_ptr, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&ap_end[1], pr->ap_ptr + pr->n_groups, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "read ap_ptr");
  const long long nnz = ap_end[1];
  if (ap_end[0] != 0 || nnz < 0)
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ap_ptr must start at 0 and end >= 0");
  if (nnz > kMaxEntries)
    return tt_fail(nullptr, TT_ERR_UNSUPPORTED,
                   "aperture lists hold %lld entries; the allocation-free path holds at most "
                   "%lld (TT_NOALLOC_MAX_APERTURE_ENTRIES)",
                   nnz, kMaxEntries);
  if (nnz > 0 && !pr->ap_idx) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ap_idx is NULL");
  e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "clear flag");
  k_na_validate<<<grid_for(std::max<long long>((long long)pr->n_groups,
                                              std::max<long long>(nnz, pr->n_dom))),
                  256, 0, s>>>(ga->n_traces, pr->n_groups, pr->n_dom, pr->group_dt,
                               pr->group_m0, pr->ap_ptr, pr->ap_idx, nnz, pr->dom_it0,
                               pr->dom_group, ga->mid, ga->off, flag);
  int herr = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, flag, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "validate");
  if (herr) {
    static const char* msg[] = {"", "ap_ptr is not non-decreasing",
                                "non-finite dt, midpoint or offset (or dt <= 0)",
                                "ap_idx holds a trace index outside [0, n_traces)",
                                "dom_group holds a group outside [0, n_groups)",
                                "dom_it0 must be in [0, 2^24)"};
    return tt_fail(nullptr, TT_ERR_INVALID_ARG, "%s", msg[herr]);
  }
  k_na_table<<<(pr->n_groups * 32 + 255) / 256, 256, 0, s>>>(
      pr->n_groups, pr->ap_ptr, pr->ap_idx, pr->group_m0, ga->mid, ga->off, tab);
  e = cudaGetLastError();
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "aperture table");
  NaFn fn = pr->op == TT_OP_CMP ? pick<TT_OP_CMP>(pr->half_window)
                                : pick<TT_OP_CRS>(pr->half_window);
  const long long n = (long long)pr->n_dom * P;
  fn<<<unsigned((n + 255) / 256), 256, 0, s>>>(ga->traces, ga->ns, tab, pr->ap_ptr,
                                                pr->group_dt, pr->dom_it0, pr->dom_group,
                                                pr->n_dom, P, theta, S);
  e = cudaGetLastError();
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "allocation-free semblance");
  return TT_OK;
}
