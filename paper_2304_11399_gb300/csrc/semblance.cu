// Launch logic and entry points of the semblance kernels (semblance_kernels.cuh):
// forward evaluation (K1 in its packed, persistent, scalar and small-launch
// split forms), the adjoint gradient (K2) and the stacked output.
#include "semblance_kernels.cuh"

namespace tt {
namespace sk {
extern template KFn pick_kernel<TT_OP_CMP>(int, int, int, bool);
extern template KFn pick_kernel<TT_OP_CRS>(int, int, int, bool);
extern template KFn pick_kernel<TT_OP_FOCRS>(int, int, int, bool);
extern template SFn pick_stack<TT_OP_CMP>(int, bool);
extern template SFn pick_stack<TT_OP_CRS>(int, bool);
extern template SFn pick_stack<TT_OP_FOCRS>(int, bool);
extern template OFn pick_order<TT_OP_CMP>(bool);
extern template OFn pick_order<TT_OP_CRS>(bool);
extern template OFn pick_order<TT_OP_FOCRS>(bool);
}  // namespace sk

namespace {

using sk::KFn;

constexpr int kDirectMax = 2048;  // direct position up to u = 2048 samples

KFn pick(int kind, const EvalArgs& a, bool mv) {
  switch (a.op) {
    case TT_OP_CMP: return sk::pick_kernel<TT_OP_CMP>(kind, a.storage, a.W, mv);
    case TT_OP_CRS: return sk::pick_kernel<TT_OP_CRS>(kind, a.storage, a.W, mv);
    case TT_OP_FOCRS: return sk::pick_kernel<TT_OP_FOCRS>(kind, a.storage, a.W, mv);
  }
  return nullptr;
}

cudaError_t launch(const EvalArgs& a, cudaStream_t s, bool grad) {
  const long long n = (long long)a.n_dom * a.P;
  if (n == 0) return cudaSuccess;
  const int block = (a.block == 128) ? 128 : 256;
  // records longer than kDirectMax samples use the moveout form of the position
  const bool mv = a.umax > float(kDirectMax);
  KFn fn;
  long long blocks;
  EvalArgs b = a;
  if (grad) {
    fn = pick(sk::kKindGrad, a, mv);
    blocks = (n + block - 1) / block;
  } else if (a.split && (n + 63) / 64 < (long long)a.n_sm * kSplitUnitsPerSm) {
    // too few units to fill the GPU: each unit's aperture split over the
    // warps of B blocks, (S, B) by launch size only
    fn = pick(sk::kKindSplit, a, mv);
    if (!fn) return cudaErrorInvalidValue;
    const long long units = (n + 63) / 64;
    int S = sk::split_warps(units, a.n_sm);
    b.split_blocks = 1;
    if (a.split_part && a.split_ticket) {
      if (units <= (long long)a.n_sm * kSplitSmallPerSm) {
        S = sk::kSplitMultiWarps;
        b.split_blocks = units * 2 <= a.n_sm ? kSplitTinyBlocks : kSplitSmallBlocks;
      } else if (units < (long long)a.n_sm * kSplitMultiPerSm) {
        S = 8;
        b.split_blocks = 2;
      }
    }
    const size_t smem = sk::split_smem_bytes(S, a.W);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(sk::split_smem_bytes(sk::kSplitMaxWarps, a.W)));
    if (e != cudaSuccess) return e;
    fn<<<unsigned(units * b.split_blocks), 32 * S, smem, s>>>(b);
    return cudaGetLastError();
  } else if (a.kernel == TT_KERNEL_SCALAR) {
    fn = pick(sk::kKindScalar, a, mv);
    blocks = (n + block - 1) / block;
  } else {
    fn = pick(sk::kKindPacked, a, mv);
    const long long units = (n + 63) / 64;
    blocks = (units + block / 32 - 1) / (block / 32);
    if (a.kernel == TT_KERNEL_PERSISTENT && a.queue) {
      int per_sm = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0);
      if (e != cudaSuccess) return e;
      const long long resident = (long long)a.n_sm * (per_sm > 0 ? per_sm : 1);
      if (resident < blocks) blocks = resident;
      e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s);
      if (e != cudaSuccess) return e;
    } else {
      b.queue = nullptr;
    }
  }
  if (!fn) return cudaErrorInvalidValue;
  if (blocks > 0x7fffffffll) return cudaErrorInvalidConfiguration;
  fn<<<unsigned(blocks), block, 0, s>>>(b);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_semblance(const EvalArgs& a, cudaStream_t s) { return launch(a, s, false); }

cudaError_t launch_stack(const EvalArgs& a, float* out, cudaStream_t s) {
  if (a.n_dom == 0) return cudaSuccess;
  if (a.P != 1) return cudaErrorInvalidValue;
  const bool mv = a.umax > float(kDirectMax);
  sk::SFn fn = nullptr;
  switch (a.op) {
    case TT_OP_CMP: fn = sk::pick_stack<TT_OP_CMP>(a.storage, mv); break;
    case TT_OP_CRS: fn = sk::pick_stack<TT_OP_CRS>(a.storage, mv); break;
    case TT_OP_FOCRS: fn = sk::pick_stack<TT_OP_FOCRS>(a.storage, mv); break;
  }
  if (!fn) return cudaErrorInvalidValue;
  const long long blocks = ((long long)a.n_dom * 32 + 255) / 256;
  if (blocks > 0x7fffffffll) return cudaErrorInvalidConfiguration;
  fn<<<unsigned(blocks), 256, 0, s>>>(a, out);
  return cudaGetLastError();
}

cudaError_t launch_semblance_grad(const EvalArgs& a, cudaStream_t s) { return launch(a, s, true); }

cudaError_t launch_member_order(const EvalArgs& a, float* theta_out, int* slots,
                                cudaStream_t s) {
  if (a.n_dom == 0) return cudaSuccess;
  if (a.P < 1 || a.P > kOrderMaxP || a.dom_map) return cudaErrorInvalidValue;
  const bool mv = a.umax > float(kDirectMax);
  sk::OFn fn = nullptr;
  switch (a.op) {
    case TT_OP_CMP: fn = sk::pick_order<TT_OP_CMP>(mv); break;
    case TT_OP_CRS: fn = sk::pick_order<TT_OP_CRS>(mv); break;
    case TT_OP_FOCRS: fn = sk::pick_order<TT_OP_FOCRS>(mv); break;
  }
  if (!fn) return cudaErrorInvalidValue;
  const long long blocks = ((long long)a.n_dom + sk::kOrderWarps - 1) / sk::kOrderWarps;
  if (blocks > 0x7fffffffll) return cudaErrorInvalidConfiguration;
  fn<<<unsigned(blocks), 32 * sk::kOrderWarps, 0, s>>>(a, theta_out, slots);
  return cudaGetLastError();
}

// L1 load-bandwidth probe: every warp streams 4-byte loads (the instruction
// K1 gathers its windows with), 32 consecutive floats per warp request, from
// a 24 KiB window that stays in L1. Each iteration starts at another line of
// the window (a multiple of 37 lines, modulo 64), so no load repeats an
// earlier iteration's address and none can be moved out of the loop; their
// sum is written so that none is dropped. The grid is one wave of resident
// blocks (at most 8 of 256 threads per SM).
constexpr int kProbeThreads = 256, kProbeBlocksPerSm = 8, kProbeLoads = 32;
__global__ void __launch_bounds__(kProbeThreads, 4) k_l1_probe(const float* buf, int iters,
                                                               float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* base = buf + ((warp & 1) * 3072 + lane);
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int it = 0; it < iters; ++it) {
    const float* p = base + ((it * 37) & 63) * 32;
#pragma unroll
    for (int u = 0; u < kProbeLoads; ++u) acc[u & 7] += __ldg(p + u * 32);
  }
  float t = 0.f;
#pragma unroll
  for (int u = 0; u < 8; ++u) t += acc[u];
  if (t == 1.2345f) out[0] = t;  // practically never: keeps the loads live
}

cudaError_t launch_l1_probe(const float* buf, float* out, int n_sm, int iters, double* bytes,
                            cudaStream_t s) {
  // one wave: as many blocks as stay resident on every SM at once
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_l1_probe,
                                                                kProbeThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  if (per_sm > kProbeBlocksPerSm) per_sm = kProbeBlocksPerSm;
  const long long blocks = (long long)n_sm * per_sm;
  *bytes = double(blocks) * kProbeThreads * double(iters) * kProbeLoads * sizeof(float);
  k_l1_probe<<<unsigned(blocks), kProbeThreads, 0, s>>>(buf, iters, out);
  return cudaGetLastError();
}

}  // namespace tt

extern "C" tt_status tt_semblance_eval(tt_ctx* ctx, const float* theta, int32_t P, float* S,
                                       void* stream) {
  if (!ctx) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (P < 1) return tt_fail(ctx, TT_ERR_INVALID_ARG, "P must be >= 1");
  if (ctx->n_dom > 0 && (!theta || !S)) return tt_fail(ctx, TT_ERR_INVALID_ARG, "NULL array");
  tt::EvalArgs a = ctx->eval_args(theta, P, S);
  return tt_cuda_check(ctx, ctx->semblance(a, static_cast<cudaStream_t>(stream), false),
                       "semblance launch");
}

extern "C" tt_status tt_stack(tt_ctx* ctx, const float* theta, float* out, void* stream) {
  if (!ctx) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->n_dom > 0 && (!theta || !out)) return tt_fail(ctx, TT_ERR_INVALID_ARG, "NULL array");
  tt::EvalArgs a = ctx->eval_args(theta, 1, nullptr);
  return tt_cuda_check(ctx, ctx->counted(tt::launch_stack(a, out, static_cast<cudaStream_t>(stream))),
                       "stack launch");
}

extern "C" tt_status tt_semblance_grad(tt_ctx* ctx, const float* theta, int32_t P, float* S,
                                       float* dS, void* stream) {
  if (!ctx) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (P < 1) return tt_fail(ctx, TT_ERR_INVALID_ARG, "P must be >= 1");
  if (ctx->n_dom > 0 && (!theta || !S || !dS))
    return tt_fail(ctx, TT_ERR_INVALID_ARG, "NULL array");
  tt::EvalArgs a = ctx->eval_args(theta, P, S);
  a.dS = dS;
  return tt_cuda_check(ctx, ctx->semblance(a, static_cast<cudaStream_t>(stream), true),
                       "semblance gradient launch");
}

extern "C" tt_status tt_ctx_probe_l1(tt_ctx* ctx, int32_t iters, double* bytes, void* stream) {
  if (!ctx) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (iters < 1 || !bytes) return tt_fail(ctx, TT_ERR_INVALID_ARG, "iters < 1 or bytes is NULL");
  // the window and the sink live in the context's split scratch (no allocation)
  return tt_cuda_check(ctx,
                       ctx->counted(tt::launch_l1_probe(ctx->split_part, ctx->split_part + 8192,
                                                        ctx->n_sm, iters, bytes,
                                                        static_cast<cudaStream_t>(stream))),
                       "L1 probe launch");
}
