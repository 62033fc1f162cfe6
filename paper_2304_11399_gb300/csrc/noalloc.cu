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
// code it names a host-side stand-in), so every call asks the runtime for the
// array's device address on the current device with cudaGetSymbolAddress
// (a lookup, no allocation); looking it up each time keeps a call correct
// after the host application has reset the device. All calls share the array
// and it keeps the last call's contents: the flag is cleared by every call,
// the table is rewritten, and calls that overlap on the GPU (different
// streams or threads) race on it. Every call synchronises its stream twice:
// to read ap_ptr, then the validation flag.
#include <algorithm>

#include "tt_internal.cuh"

namespace {

constexpr size_t kScratchBytes = TT_NOALLOC_SCRATCH_BYTES;
constexpr size_t kHeaderBytes = 256;  // validation flag, then padding
constexpr long long kMaxEntries = TT_NOALLOC_MAX_APERTURE_ENTRIES;
static_assert(kHeaderBytes + size_t(kMaxEntries) * sizeof(float4) <= kScratchBytes,
              "table does not fit the scratch array");

static __device__ __align__(256) unsigned char tt_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device, and that
// device's multiprocessor count (for grid-stride launches).
tt_status scratch_address(unsigned char** out, int* n_sm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "multiprocessor count");
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, tt_noalloc_scratch);
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "cudaGetSymbolAddress(scratch)");
  *out = static_cast<unsigned char*>(p);
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

// One warp per group (grid-stride over groups): entry e -> (dm, dm^2, h^2,
// trace index).
__global__ void k_na_table(int G, const int* ap_ptr, const int* ap_idx, const float* g_m0,
                           const float* mid, const float* off, float4* tab) {
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G;
       g += warps) {
    const float m0 = g_m0[g];
    for (int e = ap_ptr[g] + lane; e < ap_ptr[g + 1]; e += 32) {
      const int r = ap_idx[e];
      const float dm = mid[r] - m0, h = off[r];
      tab[e] = make_float4(dm, dm * dm, h * h, __int_as_float(r));
    }
  }
}

// One (domain, individual) pair per thread (grid-stride over pairs), samples
// read from the caller's [n_traces][ns] traces with the record's zero
// extension done by bounds checks (no padded copy). The window centre
// u = t / dt (samples) is found directly, u = sqrt(U), for records of up to
// 2048 samples (MV false); longer records (MV true) take u = it0 + du, with
// the moveout du the root of du^2 + 2 it0 du - V = 0, V = U - it0^2 formed
// from its small terms, from one reciprocal-square-root estimate and one
// Newton step: it0 is an exact integer and du is small, so the interpolation
// weight keeps ~1e-5-sample accuracy where u itself (thousands of samples)
// would round at ~1e-4 samples. U < 0 (no real traveltime) gives NaN, which
// the clamp to ns + w maps to a window of zeros.
template <int OP, int W, bool MV>
__global__ void __launch_bounds__(256)
    k_na_semblance(const float* __restrict__ traces, int ns, const float4* __restrict__ tab,
                   const int* ap_ptr, const float* g_dt, const int* dom_it0,
                   const int* dom_group, int n_dom, int P, const float* theta, float* S) {
  constexpr int K = 2 * W + 1;
  constexpr int D = OP == TT_OP_CMP ? 1 : 3;
  const long long n = (long long)n_dom * P;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const int d = int(q / P);
    const int g = dom_group[d];
    const float inv_dt = 1.0f / g_dt[g];
    const int it0 = dom_it0[d];
    const float p0 = float(it0);
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
      float f;
      int j;
      if (!MV) {
        const float qv = fmaf(ca, t4.x, p0);
        const float U = fmaf(cb, t4.y, fmaf(cc, t4.z, qv * qv));
        const float u = fminf(sqrtf(U), umax);
        const float fl = truncf(u);
        f = u - fl;
        j = int(fl);
      } else {
        const float x = ca * t4.x;
        const float V = fmaf(x, x + 2.f * p0, fmaf(cb, t4.y, cc * t4.z));
        const float U = fmaf(p0, p0, 1e-30f) + V;  // the bias keeps U = 0 finite
        const float r = rsqrtf(U);
        const float du0 = fmaf(U, r, -p0);
        float du = fmaf(-0.5f * r, fmaf(du0, du0 + 2.f * p0, -V), du0);
        du = fmaxf(fminf(du, umax - p0), -p0);
        const float fl = floorf(du);
        f = du - fl;
        j = it0 + int(fl);
      }
      const int j0 = j - W;
      const float* row = traces + (size_t)__float_as_int(t4.w) * ns;
      float xv[K + 1];
#pragma unroll
      for (int k = 0; k <= K; ++k) {
        const int m = j0 + k;
        xv[k] = (m >= 0 && m < ns) ? __ldg(row + m) : 0.f;
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
}

using NaFn = void (*)(const float*, int, const float4*, const int*, const float*, const int*,
                      const int*, int, int, const float*, float*);

template <int OP, bool MV>
NaFn pick_w(int W) {
  switch (W) {
    case 0: return k_na_semblance<OP, 0, MV>;
    case 1: return k_na_semblance<OP, 1, MV>;
    case 2: return k_na_semblance<OP, 2, MV>;
    case 3: return k_na_semblance<OP, 3, MV>;
    case 4: return k_na_semblance<OP, 4, MV>;
    case 5: return k_na_semblance<OP, 5, MV>;
    case 6: return k_na_semblance<OP, 6, MV>;
    case 7: return k_na_semblance<OP, 7, MV>;
    case 8: return k_na_semblance<OP, 8, MV>;
  }
  return nullptr;
}

// positions by the moveout form for records longer than this many samples
constexpr int kDirectMax = 2048;

NaFn pick(int op, int W, bool mv) {
  if (op == TT_OP_CMP) return mv ? pick_w<TT_OP_CMP, true>(W) : pick_w<TT_OP_CMP, false>(W);
  return mv ? pick_w<TT_OP_CRS, true>(W) : pick_w<TT_OP_CRS, false>(W);
}

// blocks of a grid-stride launch over n items, threads_per_item threads each:
// enough to cover them, at most 32 blocks of 256 threads per SM
unsigned grid_for(long long n, int n_sm, int threads_per_item = 1) {
  long long b = (n * threads_per_item + 255) / 256;
  const long long cap = 32ll * (n_sm > 0 ? n_sm : 1);
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return unsigned(b);
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
  int n_sm = 1;
  tt_status st = scratch_address(&scratch, &n_sm);
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
                                              std::max<long long>(nnz, pr->n_dom)),
                           n_sm),
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
  k_na_table<<<grid_for(pr->n_groups, n_sm, 32), 256, 0, s>>>(
      pr->n_groups, pr->ap_ptr, pr->ap_idx, pr->group_m0, ga->mid, ga->off, tab);
  e = cudaGetLastError();
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "aperture table");
  NaFn fn = pick(pr->op, pr->half_window, ga->ns + pr->half_window > kDirectMax);
  const long long n = (long long)pr->n_dom * P;
  fn<<<grid_for(n, n_sm), 256, 0, s>>>(ga->traces, ga->ns, tab, pr->ap_ptr, pr->group_dt,
                                       pr->dom_it0, pr->dom_group, pr->n_dom, P, theta, S);
  e = cudaGetLastError();
  if (e != cudaSuccess) return tt_cuda_check(nullptr, e, "allocation-free semblance");
  return TT_OK;
}
