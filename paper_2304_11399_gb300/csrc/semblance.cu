// Semblance of a traveltime operator (K1) and its adjoint gradient (K2).
//
// Work decomposition: one thread per (domain, individual) pair, pairs laid
// out domain-major so that a warp covers consecutive individuals of one
// domain (P >= 32) or several consecutive domains of one group (P < 32).
// Consecutive domains share a group (same m0, same aperture), so every lane
// of a warp walks the same aperture entries in the same order: the
// geometry-table loads are warp-uniform broadcasts and the 2w+2 samples that
// each lane reads from a trace row sit at nearby addresses for nearby t0 and
// for a converging population, which the L1 cache turns into reuse.
//
// Per aperture trace i (Sec. 2, the W_l x T_a inner loop of eq. order):
//   U = (it0 + (A/dt) dm)^2 + (B/dt^2) dm^2 + (C/dt^2) h^2   (samples^2)
//   u = min(sqrt(U), ns + w)  -- NaN from U < 0 also maps to ns + w, where
//                                the whole window reads padding zeros
//   j = floor(u), f = u - j, a_k = x[j+k] + f (x[j+k+1] - x[j+k])
//   s_k += a_k, E += a_k^2
// S = sum_k s_k^2 / (N E) (0 when E = 0).
#include "tt_internal.cuh"

namespace tt {
namespace {

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <typename T>
__device__ __forceinline__ float ld_sample(const T* p);
template <>
__device__ __forceinline__ float ld_sample<float>(const float* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float ld_sample<__nv_bfloat16>(const __nv_bfloat16* p) {
  unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(p));
  return __uint_as_float(unsigned(u) << 16);
}

// Per-lane prologue shared by K1 and K2.
struct Lane {
  int d, p, e0, e1;
  float p0, ca, cb, cc, inv_dt;
};

template <int OP>
__device__ __forceinline__ bool lane_setup(const EvalArgs& a, long long q, Lane& L) {
  if (q >= (long long)a.n_dom * a.P) return false;
  L.d = int(q / a.P);
  L.p = int(q - (long long)L.d * a.P);
  int g = a.dom_group[L.d];
  L.inv_dt = a.g_inv_dt[g];
  L.e0 = a.ap_ptr[g];
  L.e1 = a.ap_ptr[g + 1];
  L.p0 = float(a.dom_it0[L.d]);
  const float* th = a.theta + q * (OP == TT_OP_CMP ? 1 : 3);
  float i2 = L.inv_dt * L.inv_dt;
  if (OP == TT_OP_CMP) {
    L.ca = 0.f;
    L.cb = 0.f;
    L.cc = th[0] * i2;
  } else {
    L.ca = th[0] * L.inv_dt;
    L.cb = th[1] * i2;
    L.cc = th[2] * i2;
  }
  return true;
}

template <int OP>
__device__ __forceinline__ float position_sq(const Lane& L, float4 t4, float& qv) {
  if (OP == TT_OP_CMP) {
    qv = L.p0;
    return fmaf(L.cc, t4.z, __fmul_rn(L.p0, L.p0));
  }
  qv = fmaf(L.ca, t4.x, L.p0);
  return fmaf(L.cb, t4.y, fmaf(L.cc, t4.z, __fmul_rn(qv, qv)));
}

// Final normalisation S = Q / (N E). FP32-stored traces: E is one FP32
// sum over the aperture. BF16-stored traces (long apertures, reduced-
// precision data): E is accumulated in FP32 within chunks of 32 aperture
// traces and the chunk sums are added in FP64, so the energy's rounding
// error stays that of a 32-trace FP32 sum; the division is done in FP64.
template <typename T>
struct Chunk {
  static constexpr bool kF64 = false;
  static constexpr int kTraces = 1 << 30;  // one chunk: the whole aperture
};
template <>
struct Chunk<__nv_bfloat16> {
  static constexpr bool kF64 = true;
  static constexpr int kTraces = 32;
};

template <typename T>
__device__ __forceinline__ float normalise(float Q, int N, float E, double Ed) {
  if (Chunk<T>::kF64) return (Ed > 0.0) ? float(double(Q) / (double(N) * Ed)) : 0.f;
  return (E > 0.f) ? Q / (float(N) * E) : 0.f;
}

// Scalar evaluation of one (domain, individual) pair over its aperture.
template <int OP, int W, typename T>
__device__ __forceinline__ float eval_scalar(const EvalArgs& a, const Lane& L) {
  constexpr int K = 2 * W + 1;
  const T* __restrict__ tr = static_cast<const T*>(a.traces);
  float s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = 0.f;
  double Ed = 0.0;  // FP64 sum of per-chunk energies (BF16 storage only)
  float E = 0.f;
  for (int c0 = L.e0, c1; c0 < L.e1; c0 = c1) {
    c1 = (L.e1 - c0 > Chunk<T>::kTraces) ? c0 + Chunk<T>::kTraces : L.e1;
    float Ec = 0.f;
    for (int e = c0; e < c1; ++e) {
      const float4 t4 = __ldg(a.ap_tab + e);
      float qv;
      const float U = position_sq<OP>(L, t4, qv);
      const float u = fminf(sqrt_approx(U), a.umax);
      const float fl = truncf(u);
      const float f = u - fl, g = 1.f - f;
      const T* x = tr + (__float_as_uint(t4.w) + int(fl) - W);
      float xv[K + 1];
#pragma unroll
      for (int k = 0; k <= K; ++k) xv[k] = ld_sample<T>(x + k);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        // same operations, in the same order, as one lane of the packed path
        const float ak = fmaf(f, xv[k + 1], __fmul_rn(g, xv[k]));
        s[k] = __fadd_rn(s[k], ak);
        Ec = fmaf(ak, ak, Ec);
      }
    }
    if (Chunk<T>::kF64) Ed += double(Ec); else E = Ec;
  }
  float Q = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) Q = fmaf(s[k], s[k], Q);
  const int N = L.e1 - L.e0;
  return normalise<T>(Q, N, E, Ed);
}

__device__ __forceinline__ void store_S(const EvalArgs& a, long long q, int d, float S) {
  if (a.slots) {
    const int slot = a.slots[q];
    if (slot >= 0) a.S[(size_t)d * a.np_out + slot] = S;
  } else {
    a.S[q] = S;
  }
}

// K1. Each thread evaluates two (domain, individual) pairs, q and q + 32 of
// its warp's 64 consecutive pairs. When both lie in one group (the common
// case: same aperture, possibly different t0) the aperture is walked once
// and the two windows are processed with packed FP32x2 arithmetic: sample
// k of the two pairs forms one register pair, so every interpolation,
// stack and energy update is one f32x2 instruction for both. Otherwise
// (a group boundary inside the warp, or no second pair) each pair is
// evaluated on its own.
template <int OP, int W, typename T>
__global__ void __launch_bounds__(kBlock) k_semblance(const EvalArgs a) {
  constexpr int K = 2 * W + 1;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const long long q0 = warp * 64 + lane, q1 = q0 + 32;
  Lane L0, L1;
  const bool v0 = lane_setup<OP>(a, q0, L0);
  if (!v0) return;
  const bool v1 = lane_setup<OP>(a, q1, L1);
  if (!v1 || L1.e0 != L0.e0 || L1.e1 != L0.e1 || L1.inv_dt != L0.inv_dt) {
    store_S(a, q0, L0.d, eval_scalar<OP, W, T>(a, L0));
    if (v1) store_S(a, q1, L1.d, eval_scalar<OP, W, T>(a, L1));
    return;
  }
  const T* __restrict__ tr = static_cast<const T*>(a.traces);
  const float2 ca = make_float2(L0.ca, L1.ca), cb = make_float2(L0.cb, L1.cb),
               cc = make_float2(L0.cc, L1.cc), p0 = make_float2(L0.p0, L1.p0);
  const float2 p0sq = __fmul2_rn(p0, p0);
  float2 s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = make_float2(0.f, 0.f);
  float2 E = make_float2(0.f, 0.f);
  double Ed0 = 0.0, Ed1 = 0.0;  // FP64 chunk sums (BF16 storage only)
  for (int c0 = L0.e0, c1; c0 < L0.e1; c0 = c1) {
  c1 = (L0.e1 - c0 > Chunk<T>::kTraces) ? c0 + Chunk<T>::kTraces : L0.e1;
  float2 Ec = make_float2(0.f, 0.f);
  for (int e = c0; e < c1; ++e) {
    const float4 t4 = __ldg(a.ap_tab + e);
    float2 U;
    if (OP == TT_OP_CMP) {
      U = __ffma2_rn(cc, make_float2(t4.z, t4.z), p0sq);
    } else {
      const float2 qv = __ffma2_rn(ca, make_float2(t4.x, t4.x), p0);
      U = __ffma2_rn(cc, make_float2(t4.z, t4.z), __fmul2_rn(qv, qv));
      U = __ffma2_rn(cb, make_float2(t4.y, t4.y), U);
    }
    const float u0 = fminf(sqrt_approx(U.x), a.umax);
    const float u1 = fminf(sqrt_approx(U.y), a.umax);
    const float fl0 = truncf(u0), fl1 = truncf(u1);
    const float2 f = make_float2(u0 - fl0, u1 - fl1);
    const float2 g = make_float2(1.f - f.x, 1.f - f.y);
    const unsigned base = __float_as_uint(t4.w) - W;
    const T* x0 = tr + (base + int(fl0));
    const T* x1 = tr + (base + int(fl1));
    float2 xv[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) xv[k] = make_float2(ld_sample<T>(x0 + k), ld_sample<T>(x1 + k));
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float2 ak = __ffma2_rn(f, xv[k + 1], __fmul2_rn(g, xv[k]));
      s[k] = __fadd2_rn(s[k], ak);
      Ec = __ffma2_rn(ak, ak, Ec);
    }
  }
  if (Chunk<T>::kF64) {
    Ed0 += double(Ec.x);
    Ed1 += double(Ec.y);
  } else {
    E = Ec;
  }
  }
  float2 Q = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < K; ++k) Q = __ffma2_rn(s[k], s[k], Q);
  const int N = L0.e1 - L0.e0;
  store_S(a, q0, L0.d, normalise<T>(Q.x, N, E.x, Ed0));
  store_S(a, q1, L1.d, normalise<T>(Q.y, N, E.y, Ed1));
}

// K2: two passes over the aperture. Pass 1 = K1 (s_k, E, S). With
// alpha = 2/(N E), beta = 2 S / E, dS/da_ik = alpha s_k - beta a_ik, so pass 2
// forms dS/du_i = sum_k (alpha s_k - beta a_ik)(x[j+k+1] - x[j+k]) and
// chains it through du/dtheta:
//   du/dA = (it0 + A dm/dt) dm / (u dt),  du/dB = dm^2 / (2 u dt^2),
//   du/dC = h^2 / (2 u dt^2).
template <int OP, int W, typename T>
__global__ void __launch_bounds__(kBlock) k_semblance_grad(const EvalArgs a) {
  constexpr int K = 2 * W + 1;
  constexpr int D = OP == TT_OP_CMP ? 1 : 3;
  const long long q = (long long)blockIdx.x * kBlock + threadIdx.x;
  Lane L;
  if (!lane_setup<OP>(a, q, L)) return;
  const T* __restrict__ tr = static_cast<const T*>(a.traces);
  float s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = 0.f;
  float E = 0.f;
  for (int e = L.e0; e < L.e1; ++e) {
    const float4 t4 = __ldg(a.ap_tab + e);
    float qv;
    const float u = fminf(sqrt_approx(position_sq<OP>(L, t4, qv)), a.umax);
    const float fl = truncf(u);
    const float f = u - fl;
    const T* x = tr + (__float_as_uint(t4.w) + int(fl) - W);
    float xv[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) xv[k] = ld_sample<T>(x + k);
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
  const float N = float(L.e1 - L.e0);
  const float S = (E > 0.f) ? Q / (N * E) : 0.f;
  float G0 = 0.f, G1 = 0.f, G2 = 0.f;
  if (E > 0.f) {
    const float alpha = 2.f / (N * E);
    const float beta = 2.f * S / E;
    for (int e = L.e0; e < L.e1; ++e) {
      const float4 t4 = __ldg(a.ap_tab + e);
      float qv;
      const float u = fminf(sqrt_approx(position_sq<OP>(L, t4, qv)), a.umax);
      const float fl = truncf(u);
      const float f = u - fl;
      const T* x = tr + (__float_as_uint(t4.w) + int(fl) - W);
      float xv[K + 1];
#pragma unroll
      for (int k = 0; k <= K; ++k) xv[k] = ld_sample<T>(x + k);
      float sg = 0.f, ag = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float gk = xv[k + 1] - xv[k];
        const float ak = fmaf(f, gk, xv[k]);
        sg = fmaf(s[k], gk, sg);
        ag = fmaf(ak, gk, ag);
      }
      const float dSdu = fmaf(alpha, sg, -beta * ag);
      const float inv_u = (u > 0.f && u < a.umax) ? 1.f / u : 0.f;
      const float c = dSdu * inv_u;
      if (OP == TT_OP_CRS) {
        G0 = fmaf(c * qv, t4.x, G0);
        G1 = fmaf(0.5f * c, t4.y, G1);
      }
      G2 = fmaf(0.5f * c, t4.z, G2);
    }
  }
  a.S[q] = S;
  float* out = a.dS + q * D;
  const float i2 = L.inv_dt * L.inv_dt;
  if (OP == TT_OP_CRS) {
    out[0] = G0 * L.inv_dt;
    out[1] = G1 * i2;
    out[2] = G2 * i2;
  } else {
    out[0] = G2 * i2;
  }
}

using KFn = void (*)(const EvalArgs);

template <int OP, typename T>
KFn pick_fwd(int W) {
  switch (W) {
    case 0: return k_semblance<OP, 0, T>;
    case 1: return k_semblance<OP, 1, T>;
    case 2: return k_semblance<OP, 2, T>;
    case 3: return k_semblance<OP, 3, T>;
    case 4: return k_semblance<OP, 4, T>;
    case 5: return k_semblance<OP, 5, T>;
    case 6: return k_semblance<OP, 6, T>;
    case 7: return k_semblance<OP, 7, T>;
    case 8: return k_semblance<OP, 8, T>;
  }
  return nullptr;
}

template <int OP, typename T>
KFn pick_grad(int W) {
  switch (W) {
    case 0: return k_semblance_grad<OP, 0, T>;
    case 1: return k_semblance_grad<OP, 1, T>;
    case 2: return k_semblance_grad<OP, 2, T>;
    case 3: return k_semblance_grad<OP, 3, T>;
    case 4: return k_semblance_grad<OP, 4, T>;
    case 5: return k_semblance_grad<OP, 5, T>;
    case 6: return k_semblance_grad<OP, 6, T>;
    case 7: return k_semblance_grad<OP, 7, T>;
    case 8: return k_semblance_grad<OP, 8, T>;
  }
  return nullptr;
}

KFn select_kernel(const EvalArgs& a, bool grad) {
  const bool bf = a.storage == TT_STORE_BF16;
  if (a.op == TT_OP_CMP)
    return grad ? (bf ? pick_grad<TT_OP_CMP, __nv_bfloat16>(a.W) : pick_grad<TT_OP_CMP, float>(a.W))
                : (bf ? pick_fwd<TT_OP_CMP, __nv_bfloat16>(a.W) : pick_fwd<TT_OP_CMP, float>(a.W));
  return grad ? (bf ? pick_grad<TT_OP_CRS, __nv_bfloat16>(a.W) : pick_grad<TT_OP_CRS, float>(a.W))
              : (bf ? pick_fwd<TT_OP_CRS, __nv_bfloat16>(a.W) : pick_fwd<TT_OP_CRS, float>(a.W));
}

cudaError_t launch(const EvalArgs& a, cudaStream_t s, bool grad) {
  const long long n = (long long)a.n_dom * a.P;
  if (n == 0) return cudaSuccess;
  KFn fn = select_kernel(a, grad);
  if (!fn) return cudaErrorInvalidValue;
  const long long per_block = grad ? kBlock : 2ll * kBlock;  // K1: two pairs per thread
  const long long blocks = (n + per_block - 1) / per_block;
  if (blocks > 0x7fffffffll) return cudaErrorInvalidConfiguration;
  fn<<<unsigned(blocks), kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_semblance(const EvalArgs& a, cudaStream_t s) { return launch(a, s, false); }
cudaError_t launch_semblance_grad(const EvalArgs& a, cudaStream_t s) { return launch(a, s, true); }

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
