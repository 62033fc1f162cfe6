// Semblance kernels: K1 (forward, three forms), its small-launch split form,
// K2 (adjoint gradient) and the stacked output, as templates over the
// operator, window, storage type and position form. Each operator's
// instantiations are compiled in a translation unit of their own
// (semblance_op_*.cu) and reached through pick_kernel / pick_stack.
//
// Work decomposition: (domain, individual) pairs are laid out domain-major;
// a warp owns 64 consecutive pairs, so with NP = 64 it covers one domain,
// and consecutive warps cover adjacent t0 at the same m0. Consecutive
// domains share a group (same m0, same aperture), so every lane of a warp
// walks the same aperture entries in the same order: the geometry-table load
// is a warp-uniform broadcast and the 2w+2 samples each lane reads from a
// trace row sit at nearby addresses for nearby t0 and for a converging
// population, which the L1 cache turns into reuse.
//
// Per aperture trace i (Sec. 2, the W_l x T_a inner loop of eq. order), in
// sample units (A' = A/dt, B' = B/dt^2, C' = C/dt^2, p0 = it0), the position
// u = t/dt of the window centre is found, then
//   j = floor(u), f = u - j, g = 1 - f,
//   a_k = g x[j+k] + f x[j+k+1],  s_k += a_k,  E += a_k^2
// and S = sum_k s_k^2 / (N E) (0 when E = 0).
//
// Two ways to find u, chosen by the record length at launch:
//  * direct (records up to 2048 samples, u <= 2048 + w):
//      q = p0 + A' dm,  U = q^2 + B' dm^2 + C' h^2,  u = sqrt(U)
//    whose FP32 rounding stays within ~1e-4 samples there;
//  * moveout (longer records): u = p0 + du with du the root of
//      du^2 + 2 p0 du - V = 0,  V = x (x + 2 p0) + B' dm^2 + C' h^2,  x = A' dm,
//    taken as du0 = U r - p0 (r ~ U^-1/2 from the hardware, one rounding)
//    refined by one Newton step du = du0 - (du0 (du0 + 2 p0) - V) r / 2.
//    p0 is an exact integer and du is tens of samples for deep events, so
//    the fraction keeps ~1e-5-sample accuracy where u itself (thousands of
//    samples) would round at ~1e-4 samples.
// U < 0 (no real traveltime) gives NaN, which the clamp maps to ns + w: a
// window of padding zeros. The scalar and the packed code run the same
// operations; no product is ever rounded and then added (a pattern a compiler
// may fuse), so they agree bit for bit.
#pragma once

#include "tt_internal.cuh"

namespace tt {
namespace sk {


__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
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

// Per-lane constants of one (domain, individual) pair.
struct Lane {
  int d, e0, e1, p0i;
  float p0, ca, cb, cc, inv_dt;
  float cah, cbh;      // FO-CRS: Ah / dt and Bmh / dt^2
  float two_p0, p0sq;  // 2 p0, p0^2 + 1e-30 (the bias keeps U = 0 finite under rsqrt)
  float lim, neg_p0;   // moveout: du is clamped to [-p0, ns + w - p0]
  float umax;          // direct: u is clamped to ns + w
};

// L.d is the local domain (indexing theta and S); its geometry comes from the
// global domain dom_map[L.d] when a map is given (a subset evaluation).
template <int OP>
__device__ __forceinline__ bool lane_setup(const EvalArgs& a, long long q, Lane& L) {
  if (q >= (long long)a.n_dom * a.P) return false;
  L.d = int(q / a.P);
  const int gd = a.dom_map ? a.dom_map[L.d] : L.d;
  if (gd < 0) return false;
  const int g = a.dom_group[gd];
  L.inv_dt = a.g_inv_dt[g];
  L.e0 = a.ap_ptr[g];
  L.e1 = a.ap_ptr[g + 1];
  L.p0i = a.dom_it0[gd];
  L.p0 = float(L.p0i);
  const float* th = a.theta + q * op_dim(OP);
  const float i2 = L.inv_dt * L.inv_dt;
  L.cah = 0.f;
  L.cbh = 0.f;
  if (OP == TT_OP_CMP) {
    L.ca = 0.f;
    L.cb = 0.f;
    L.cc = th[0] * i2;
  } else if (OP == TT_OP_CRS) {
    L.ca = th[0] * L.inv_dt;
    L.cb = th[1] * i2;
    L.cc = th[2] * i2;
  } else {  // (Am, Ah, Bmm, Bmh, Bhh): ca, cah slopes, cb, cbh, cc curvatures
    L.ca = th[0] * L.inv_dt;
    L.cah = th[1] * L.inv_dt;
    L.cb = th[2] * i2;
    L.cbh = th[3] * i2;
    L.cc = th[4] * i2;
  }
  L.two_p0 = 2.f * L.p0;
  L.p0sq = __fmul_rn(L.p0, L.p0) + 1e-30f;
  L.lim = a.umax - L.p0;
  L.neg_p0 = -L.p0;
  L.umax = a.umax;
  return true;
}

// FO-CRS quadratic part in samples^2: dm (Bmm dm + Bmh dh) + (Bhh dh) dh,
// from the table entry (dm, dh, -, row)
__device__ __forceinline__ float fo_quad(const Lane& L, float4 t4) {
  return fmaf(t4.x, fmaf(L.cb, t4.x, __fmul_rn(L.cbh, t4.y)),
              __fmul_rn(__fmul_rn(L.cc, t4.y), t4.y));
}

// Position of one pair on one trace. Every operation is rounded once, in the
// same order as one lane of the packed path, so both give identical bits.
struct Pos {
  int j;       // window sample k sits at j - W + k
  float f, g;  // interpolation weights
  float u;     // clamped position (samples)
  float q;     // p0 + A' dm (for the gradient)
};

template <int OP, bool MOVEOUT>
__device__ __forceinline__ Pos locate(const Lane& L, float4 t4) {
  Pos P;
  if (!MOVEOUT) {
    float U;
    if (OP == TT_OP_CMP) {
      P.q = L.p0;
      U = fmaf(L.cc, t4.z, __fmul_rn(L.p0, L.p0));
    } else if (OP == TT_OP_CRS) {
      P.q = fmaf(L.ca, t4.x, L.p0);
      U = fmaf(L.cb, t4.y, fmaf(L.cc, t4.z, __fmul_rn(P.q, P.q)));
    } else {
      P.q = fmaf(L.ca, t4.x, fmaf(L.cah, t4.y, L.p0));
      U = fmaf(P.q, P.q, fo_quad(L, t4));
    }
    P.u = fminf(sqrt_approx(U), L.umax);
    const float fl = truncf(P.u);
    P.f = __fsub_rn(P.u, fl);
    P.g = __fsub_rn(1.f, P.f);
    P.j = int(fl);
    return P;
  }
  float V, x;
  if (OP == TT_OP_CMP) {
    x = 0.f;
    V = __fmul_rn(L.cc, t4.z);
  } else if (OP == TT_OP_CRS) {
    x = __fmul_rn(L.ca, t4.x);
    const float w = fmaf(L.cb, t4.y, __fmul_rn(L.cc, t4.z));
    V = fmaf(x, __fadd_rn(x, L.two_p0), w);
  } else {
    x = fmaf(L.ca, t4.x, __fmul_rn(L.cah, t4.y));
    V = fmaf(x, __fadd_rn(x, L.two_p0), fo_quad(L, t4));
  }
  const float U = __fadd_rn(L.p0sq, V);
  const float r = rsqrt_approx(U);
  const float du0 = fmaf(U, r, L.neg_p0);
  const float res = fmaf(du0, __fadd_rn(du0, L.two_p0), __fmul_rn(V, -1.f));
  float du = fmaf(res, __fmul_rn(r, -0.5f), du0);
  du = fmaxf(fminf(du, L.lim), L.neg_p0);
  const float fl = floorf(du);
  P.f = fmaf(fl, -1.f, du);
  P.g = fmaf(P.f, -1.f, 1.f);
  P.j = L.p0i + int(fl);
  P.u = L.p0 + du;
  P.q = L.p0 + x;
  return P;
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

__device__ __forceinline__ void store_S(const EvalArgs& a, long long q, int d, float S) {
  if (a.slots) {
    const int slot = a.slots[q];
    if (slot >= 0) a.S[(size_t)d * a.np_out + slot] = S;
  } else {
    a.S[q] = S;
  }
}

// Accumulate one pair over aperture entries [r0, r1): the stack sums s_k and
// the energy -- one FP32 sum over the range (FP32 storage), or the FP64 sum
// of FP32 sums over 32-entry chunks from r0 (BF16 storage).
template <int OP, int W, typename T, bool MV>
__device__ __forceinline__ void acc_scalar(const EvalArgs& a, const Lane& L, int r0, int r1,
                                           float* s, float& E, double& Ed) {
  constexpr int K = 2 * W + 1;
  const T* __restrict__ tr = static_cast<const T*>(a.traces);
  for (int c0 = r0, c1; c0 < r1; c0 = c1) {
    c1 = (r1 - c0 > Chunk<T>::kTraces) ? c0 + Chunk<T>::kTraces : r1;
    float Ec = 0.f;
    for (int e = c0; e < c1; ++e) {
      const float4 t4 = __ldg(a.ap_tab + e);
      const Pos P = locate<OP, MV>(L, t4);
      const T* x = tr + (__float_as_uint(t4.w) + P.j - W);
      float xv[K + 1];
#pragma unroll
      for (int k = 0; k <= K; ++k) xv[k] = ld_sample<T>(x + k);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float ak = fmaf(P.f, xv[k + 1], __fmul_rn(P.g, xv[k]));
        s[k] = __fadd_rn(s[k], ak);
        Ec = fmaf(ak, ak, Ec);
      }
    }
    if (Chunk<T>::kF64) Ed += double(Ec); else E = Ec;
  }
}

// The same for two pairs sharing an aperture, with packed FP32x2 arithmetic:
// sample k of the two pairs forms one register pair, so every interpolation,
// stack and energy update is one f32x2 instruction for both (same operations
// and bits as two acc_scalar calls).
template <int OP, int W, typename T, bool MV>
__device__ __forceinline__ void acc_packed(const EvalArgs& a, const Lane& L0, const Lane& L1,
                                           int r0, int r1, float2* s, float2& E, double& Ed0,
                                           double& Ed1) {
  constexpr int K = 2 * W + 1;
  const T* __restrict__ tr = static_cast<const T*>(a.traces);
  const float2 ca = make_float2(L0.ca, L1.ca), cb = make_float2(L0.cb, L1.cb),
               cc = make_float2(L0.cc, L1.cc), two_p0 = make_float2(L0.two_p0, L1.two_p0),
               p0sq = make_float2(L0.p0sq, L1.p0sq), neg_p0 = make_float2(L0.neg_p0, L1.neg_p0),
               p0v = make_float2(L0.p0, L1.p0);
  const float2 cah = make_float2(L0.cah, L1.cah), cbh = make_float2(L0.cbh, L1.cbh);
  const float2 p0p0 = __fmul2_rn(p0v, p0v);
  // FO-CRS quadratic part, the packed twin of fo_quad
  auto fo_quad2 = [&](float2 dm, float2 dh) {
    return __ffma2_rn(dm, __ffma2_rn(cb, dm, __fmul2_rn(cbh, dh)),
                      __fmul2_rn(__fmul2_rn(cc, dh), dh));
  };
  const float2 m1 = make_float2(-1.f, -1.f), one = make_float2(1.f, 1.f),
               mhalf = make_float2(-0.5f, -0.5f);
  for (int c0 = r0, c1; c0 < r1; c0 = c1) {
    c1 = (r1 - c0 > Chunk<T>::kTraces) ? c0 + Chunk<T>::kTraces : r1;
    float2 Ec = make_float2(0.f, 0.f);
    for (int e = c0; e < c1; ++e) {
      const float4 t4 = __ldg(a.ap_tab + e);
      float2 f, g;
      int j0, j1;
      if constexpr (!MV) {
        float2 U;
        if (OP == TT_OP_CMP) {
          U = __ffma2_rn(cc, make_float2(t4.z, t4.z), p0p0);
        } else if (OP == TT_OP_CRS) {
          const float2 qv = __ffma2_rn(ca, make_float2(t4.x, t4.x), p0v);
          U = __ffma2_rn(cc, make_float2(t4.z, t4.z), __fmul2_rn(qv, qv));
          U = __ffma2_rn(cb, make_float2(t4.y, t4.y), U);
        } else {
          const float2 dm = make_float2(t4.x, t4.x), dh = make_float2(t4.y, t4.y);
          const float2 qv = __ffma2_rn(ca, dm, __ffma2_rn(cah, dh, p0v));
          U = __ffma2_rn(qv, qv, fo_quad2(dm, dh));
        }
        const float u0 = fminf(sqrt_approx(U.x), L0.umax), u1 = fminf(sqrt_approx(U.y), L1.umax);
        const float fl0 = truncf(u0), fl1 = truncf(u1);
        f = make_float2(__fsub_rn(u0, fl0), __fsub_rn(u1, fl1));
        g = make_float2(__fsub_rn(1.f, f.x), __fsub_rn(1.f, f.y));
        j0 = int(fl0);
        j1 = int(fl1);
      } else {
        float2 V;
        if (OP == TT_OP_CMP) {
          V = __fmul2_rn(cc, make_float2(t4.z, t4.z));
        } else if (OP == TT_OP_CRS) {
          const float2 x = __fmul2_rn(ca, make_float2(t4.x, t4.x));
          const float2 w = __ffma2_rn(cb, make_float2(t4.y, t4.y),
                                      __fmul2_rn(cc, make_float2(t4.z, t4.z)));
          V = __ffma2_rn(x, __fadd2_rn(x, two_p0), w);
        } else {
          const float2 dm = make_float2(t4.x, t4.x), dh = make_float2(t4.y, t4.y);
          const float2 x = __ffma2_rn(ca, dm, __fmul2_rn(cah, dh));
          V = __ffma2_rn(x, __fadd2_rn(x, two_p0), fo_quad2(dm, dh));
        }
        const float2 U = __fadd2_rn(p0sq, V);
        const float2 r = make_float2(rsqrt_approx(U.x), rsqrt_approx(U.y));
        const float2 du0 = __ffma2_rn(U, r, neg_p0);
        const float2 res = __ffma2_rn(du0, __fadd2_rn(du0, two_p0), __fmul2_rn(V, m1));
        float2 du = __ffma2_rn(res, __fmul2_rn(r, mhalf), du0);
        du.x = fmaxf(fminf(du.x, L0.lim), L0.neg_p0);
        du.y = fmaxf(fminf(du.y, L1.lim), L1.neg_p0);
        const float2 fl = make_float2(floorf(du.x), floorf(du.y));
        f = __ffma2_rn(fl, m1, du);
        g = __ffma2_rn(f, m1, one);
        j0 = L0.p0i + int(fl.x);
        j1 = L1.p0i + int(fl.y);
      }
      const unsigned base = __float_as_uint(t4.w) - W;
      const T* x0 = tr + (base + j0);
      const T* x1 = tr + (base + j1);
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
}

// Scalar evaluation of one (domain, individual) pair over its aperture.
template <int OP, int W, typename T, bool MV>
__device__ __forceinline__ float eval_scalar(const EvalArgs& a, const Lane& L) {
  constexpr int K = 2 * W + 1;
  float s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = 0.f;
  float E = 0.f;
  double Ed = 0.0;
  acc_scalar<OP, W, T, MV>(a, L, L.e0, L.e1, s, E, Ed);
  float Q = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) Q = fmaf(s[k], s[k], Q);
  return normalise<T>(Q, L.e1 - L.e0, E, Ed);
}

__device__ __forceinline__ bool same_aperture(const Lane& L0, const Lane& L1) {
  return L1.e0 == L0.e0 && L1.e1 == L0.e1 && L1.inv_dt == L0.inv_dt;
}

// One 64-pair unit: each thread evaluates pairs q and q + 32 (either may be
// absent: past the end, or a domain the map skips). When both lie in one
// group (the common case: same aperture, possibly different t0) the
// aperture is walked once with packed arithmetic; otherwise each pair is
// evaluated on its own (same operations, same bits).
template <int OP, int W, typename T, bool MV>
__device__ __forceinline__ void eval_unit(const EvalArgs& a, long long unit, int lane) {
  constexpr int K = 2 * W + 1;
  const long long q0 = unit * 64 + lane, q1 = q0 + 32;
  Lane L0, L1;
  const bool v0 = lane_setup<OP>(a, q0, L0);
  const bool v1 = lane_setup<OP>(a, q1, L1);
  if (!v0 || !v1 || !same_aperture(L0, L1)) {
    if (v0) store_S(a, q0, L0.d, eval_scalar<OP, W, T, MV>(a, L0));
    if (v1) store_S(a, q1, L1.d, eval_scalar<OP, W, T, MV>(a, L1));
    return;
  }
  float2 s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = make_float2(0.f, 0.f);
  float2 E = make_float2(0.f, 0.f);
  double Ed0 = 0.0, Ed1 = 0.0;
  acc_packed<OP, W, T, MV>(a, L0, L1, L0.e0, L0.e1, s, E, Ed0, Ed1);
  float2 Q = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < K; ++k) Q = __ffma2_rn(s[k], s[k], Q);
  const int N = L0.e1 - L0.e0;
  store_S(a, q0, L0.d, normalise<T>(Q.x, N, E.x, Ed0));
  store_S(a, q1, L1.d, normalise<T>(Q.y, N, E.y, Ed1));
}

// K1 for small launches (few 64-pair units): B blocks of S warps share one
// unit, warp w of block b walking slice b S + w of the B S contiguous slices
// of every pair's aperture. Within a block the slices' partial sums meet in
// shared memory and are added in slice order; with B > 1 each block writes
// its sums to global scratch and the last block of the unit to arrive (an
// atomic ticket, no waiting) adds the B block sums in block order. (S, B)
// is (8, 9) up to half a unit per SM, (8, 7) up to 2 units per SM, (8, 2)
// below 12 per SM and (8, 1) above (76, 304 and 1824 units on a 152-SM
// device), so that the GPU stays busy. The summation order depends on (S, B) and
// differs from the one-warp-per-unit kernel, so all are chosen by launch
// size alone -- every variant of a launch runs the same code -- and results
// stay reproducible.
constexpr int kSplitMaxWarps = 16;

// warps per block of a one-block-per-unit split launch of `units` units on a
// device of n_sm SMs: 8 once that keeps about 32 warps resident per SM, else 16
inline int split_warps(long long units, int n_sm) {
  return units * 8 >= (long long)n_sm * 32 ? 8 : kSplitMaxWarps;
}

// Launches of at most n_sm * kSplitSmallPerSm units run kSplitMultiWarps warps per
// block, kSplitSmallBlocks blocks per unit (56 slices per aperture), or
// kSplitTinyBlocks (72 slices) up to n_sm / 2 units: 256-thread blocks, four
// of which share an SM, so that one block's barrier overlaps the others'
// loads. The best of the (S, B) pairs timed on the ENS 5 x 1 sweep, whose
// launches hold 157 and 63 units (21.7 ms against 23.1 for (16, 4); (8, 5),
// (8, 6), (8, 8), (16, 3), (16, 5) and for the smaller launches (8, 6),
// (16, 4), (16, 8) were slower). Below n_sm * kSplitMultiPerSm units, (8, 2):
// timed 17% faster than (8, 1) on the 938-unit launches of an ENS 30 x 30
// sweep, while from about 2500 units (ENS 80 x 80) one block per unit is
// best.
constexpr int kSplitMultiWarps = 8;

// dynamic shared memory of a split block: FP64 energies [S][64], FP32
// energies [S][64], stack sums [S][64][K]
inline size_t split_smem_bytes(int S, int W) {
  return size_t(S) * 64 * (sizeof(double) + sizeof(float) + sizeof(float) * (2 * W + 1));
}

template <int OP, int W, typename T, bool MV>
__global__ void __launch_bounds__(32 * kSplitMaxWarps, 2) k_semblance_split(const EvalArgs a) {
  constexpr int K = 2 * W + 1;
  extern __shared__ __align__(16) unsigned char split_smem[];
  const int S = blockDim.x >> 5;
  double* part_Ed = reinterpret_cast<double*>(split_smem);   // [S][64]
  float* part_E = reinterpret_cast<float*>(part_Ed + S * 64);  // [S][64]
  float* part_s = part_E + S * 64;                             // [S][64][K]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int B = a.split_blocks;
  const long long unit = blockIdx.x / B;
  const int part = int(blockIdx.x - unit * B);
  const long long q0 = unit * 64 + lane, q1 = q0 + 32;
  Lane L0, L1;
  const bool v0 = lane_setup<OP>(a, q0, L0);
  const bool v1 = lane_setup<OP>(a, q1, L1);
  auto slice = [&](const Lane& L, int& r0, int& r1) {
    const long long n = L.e1 - L.e0, nsl = (long long)S * B, sl = (long long)part * S + w;
    r0 = L.e0 + int(n * sl / nsl);
    r1 = L.e0 + int(n * (sl + 1) / nsl);
  };
  if (v0 && v1 && same_aperture(L0, L1)) {
    int r0, r1;
    slice(L0, r0, r1);
    float2 s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = make_float2(0.f, 0.f);
    float2 E = make_float2(0.f, 0.f);
    double Ed0 = 0.0, Ed1 = 0.0;
    acc_packed<OP, W, T, MV>(a, L0, L1, r0, r1, s, E, Ed0, Ed1);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      part_s[(w * 64 + lane) * K + k] = s[k].x;
      part_s[(w * 64 + lane + 32) * K + k] = s[k].y;
    }
    part_E[w * 64 + lane] = E.x;
    part_E[w * 64 + lane + 32] = E.y;
    part_Ed[w * 64 + lane] = Ed0;
    part_Ed[w * 64 + lane + 32] = Ed1;
  } else {
    for (int h = 0; h < 2; ++h) {
      const Lane& L = h ? L1 : L0;
      if (!(h ? v1 : v0)) continue;
      int r0, r1;
      slice(L, r0, r1);
      float s[K];
#pragma unroll
      for (int k = 0; k < K; ++k) s[k] = 0.f;
      float E = 0.f;
      double Ed = 0.0;
      acc_scalar<OP, W, T, MV>(a, L, r0, r1, s, E, Ed);
      const int p = lane + 32 * h;
#pragma unroll
      for (int k = 0; k < K; ++k) part_s[(w * 64 + p) * K + k] = s[k];
      part_E[w * 64 + p] = E;
      part_Ed[w * 64 + p] = Ed;
    }
  }
  __syncthreads();
  // the block's sums of pair p = threadIdx.x (< 64), slices in order
  const int p = threadIdx.x;
  Lane L;
  const bool valid = p < 64 && lane_setup<OP>(a, unit * 64 + p, L);
  float sk[K];
  float E = 0.f;
  double Ed = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) sk[k] = 0.f;
  if (valid) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      for (int v = 0; v < S; ++v) sk[k] = __fadd_rn(sk[k], part_s[(v * 64 + p) * K + k]);
    for (int v = 0; v < S; ++v) {
      E = __fadd_rn(E, part_E[v * 64 + p]);
      Ed += part_Ed[v * 64 + p];
    }
  }
  if (B > 1) {
    // publish the block's sums; the unit's last block adds them in block order
    const size_t set = size_t(unit) * B + part;
    float* gp = a.split_part + (set * 64 + p) * kSplitPartStride;
    if (valid) {
#pragma unroll
      for (int k = 0; k < K; ++k) gp[k] = sk[k];
      gp[K] = E;
      a.split_part_d[set * 64 + p] = Ed;
    }
    __threadfence();
    __syncthreads();
    __shared__ int last;
    if (threadIdx.x == 0) last = atomicAdd(a.split_ticket + unit, 1u) == unsigned(B - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) a.split_ticket[unit] = 0u;  // ready for the next launch
    if (!valid) return;
#pragma unroll
    for (int k = 0; k < K; ++k) sk[k] = 0.f;
    E = 0.f;
    Ed = 0.0;
    for (int b = 0; b < B; ++b) {
      const size_t sb = size_t(unit) * B + b;
      const float* q = a.split_part + (sb * 64 + p) * kSplitPartStride;
#pragma unroll
      for (int k = 0; k < K; ++k) sk[k] = __fadd_rn(sk[k], __ldcg(q + k));
      E = __fadd_rn(E, __ldcg(q + K));
      Ed += __ldcg(a.split_part_d + sb * 64 + p);
    }
  }
  if (!valid) return;
  float Q = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) Q = fmaf(sk[k], sk[k], Q);
  store_S(a, unit * 64 + p, L.d, normalise<T>(Q, L.e1 - L.e0, E, Ed));
}

// K1, grid-mapped (queue == nullptr: one 64-pair unit per warp, the grid
// covers every unit) or persistent (a grid sized to the GPU; after its first
// unit a warp takes the next one from an atomic counter, so warps whose
// apertures are short take more units).
template <int OP, int W, typename T, bool MV>
__global__ void __launch_bounds__(kBlock) k_semblance(const EvalArgs a) {
  const int lane = threadIdx.x & 31;
  const long long n_units = ((long long)a.n_dom * a.P + 63) / 64;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  long long unit = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  while (unit < n_units) {
    eval_unit<OP, W, T, MV>(a, unit, lane);
    if (!a.queue) break;
    __syncwarp();
    unsigned long long next = 0;
    if (lane == 0) next = atomicAdd(a.queue, 1ull);
    unit = warps + (long long)__shfl_sync(0xffffffffu, next, 0);
  }
}

// K1, one (domain, individual) pair per thread.
template <int OP, int W, typename T, bool MV>
__global__ void __launch_bounds__(kBlock) k_semblance_scalar(const EvalArgs a) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  Lane L;
  if (!lane_setup<OP>(a, q, L)) return;
  store_S(a, q, L.d, eval_scalar<OP, W, T, MV>(a, L));
}

// K2: two passes over the aperture. Pass 1 = K1 (s_k, E, S). With
// alpha = 2/(N E), beta = 2 S / E, dS/da_ik = alpha s_k - beta a_ik, so pass 2
// forms dS/du_i = sum_k (alpha s_k - beta a_ik)(x[j+k+1] - x[j+k]) and
// chains it through du/dtheta (u = p0 + du in samples, q = p0 + A' dm):
//   du/dA = q dm / (u dt),  du/dB = dm^2 / (2 u dt^2),  du/dC = h^2 / (2 u dt^2).
// Positions clamped to the all-zero window and u = 0 contribute nothing.
template <int OP, int W, typename T, bool MV>
__global__ void __launch_bounds__(kBlock) k_semblance_grad(const EvalArgs a) {
  constexpr int K = 2 * W + 1;
  constexpr int D = op_dim(OP);
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  Lane L;
  if (!lane_setup<OP>(a, q, L)) return;
  const T* __restrict__ tr = static_cast<const T*>(a.traces);
  float s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = 0.f;
  float E = 0.f;
  for (int e = L.e0; e < L.e1; ++e) {
    const float4 t4 = __ldg(a.ap_tab + e);
    const Pos P = locate<OP, MV>(L, t4);
    const T* x = tr + (__float_as_uint(t4.w) + P.j - W);
    float xv[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) xv[k] = ld_sample<T>(x + k);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float ak = fmaf(P.f, xv[k + 1], __fmul_rn(P.g, xv[k]));
      s[k] += ak;
      E = fmaf(ak, ak, E);
    }
  }
  float Q = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) Q = fmaf(s[k], s[k], Q);
  const float N = float(L.e1 - L.e0);
  const float S = (E > 0.f) ? Q / (N * E) : 0.f;
  float G0 = 0.f, G1 = 0.f, G2 = 0.f, G3 = 0.f, G4 = 0.f;
  if (E > 0.f) {
    const float alpha = 2.f / (N * E);
    const float beta = 2.f * S / E;
    for (int e = L.e0; e < L.e1; ++e) {
      const float4 t4 = __ldg(a.ap_tab + e);
      const Pos P = locate<OP, MV>(L, t4);
      const T* x = tr + (__float_as_uint(t4.w) + P.j - W);
      float xv[K + 1];
#pragma unroll
      for (int k = 0; k <= K; ++k) xv[k] = ld_sample<T>(x + k);
      float sg = 0.f, ag = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float gk = xv[k + 1] - xv[k];
        const float ak = fmaf(P.f, xv[k + 1], __fmul_rn(P.g, xv[k]));
        sg = fmaf(s[k], gk, sg);
        ag = fmaf(ak, gk, ag);
      }
      const float dSdu = fmaf(alpha, sg, -beta * ag);
      const float inv_u = (P.u > 0.f && P.u < L.umax) ? 1.f / P.u : 0.f;
      const float c = dSdu * inv_u;
      if (OP == TT_OP_FOCRS) {  // dU = 2q dm, 2q dh, dm^2, dm dh, dh^2
        G0 = fmaf(c * P.q, t4.x, G0);
        G1 = fmaf(c * P.q, t4.y, G1);
        G2 = fmaf(0.5f * c, t4.x * t4.x, G2);
        G3 = fmaf(0.5f * c, t4.x * t4.y, G3);
        G4 = fmaf(0.5f * c, t4.y * t4.y, G4);
        continue;
      }
      if (OP == TT_OP_CRS) {
        G0 = fmaf(c * P.q, t4.x, G0);
        G1 = fmaf(0.5f * c, t4.y, G1);
      }
      G2 = fmaf(0.5f * c, t4.z, G2);
    }
  }
  a.S[q] = S;
  float* out = a.dS + q * D;
  const float i2 = L.inv_dt * L.inv_dt;
  if (OP == TT_OP_FOCRS) {
    out[0] = G0 * L.inv_dt;
    out[1] = G1 * L.inv_dt;
    out[2] = G2 * i2;
    out[3] = G3 * i2;
    out[4] = G4 * i2;
  } else if (OP == TT_OP_CRS) {
    out[0] = G0 * L.inv_dt;
    out[1] = G1 * i2;
    out[2] = G2 * i2;
  } else {
    out[0] = G2 * i2;
  }
}

using KFn = void (*)(const EvalArgs);

// Stacked output: one warp per domain (P = 1, theta [n_dom][D]); lane l sums
// the centre amplitudes of aperture entries e0 + l, e0 + l + 32, ... in order,
// the 32 lane sums meet in a butterfly, and the mean is one FP32 division.
// Positions are those of the semblance window's centre sample (same clamp:
// T < 0 or past the record reads the zero padding).
template <int OP, typename T, bool MV>
__global__ void __launch_bounds__(256) k_stack(const EvalArgs a, float* __restrict__ out) {
  const long long d = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  Lane L;
  if (!lane_setup<OP>(a, d, L)) return;  // warp-uniform: the whole warp leaves
  const T* __restrict__ tr = static_cast<const T*>(a.traces);
  float s = 0.f;
  for (int e = L.e0 + lane; e < L.e1; e += 32) {
    const float4 t4 = __ldg(a.ap_tab + e);
    const Pos P = locate<OP, MV>(L, t4);
    const T* x = tr + (__float_as_uint(t4.w) + P.j);
    s = __fadd_rn(s, fmaf(P.f, ld_sample<T>(x + 1), __fmul_rn(P.g, ld_sample<T>(x))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = __fadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
  if (lane == 0) {
    const int N = L.e1 - L.e0;
    out[L.d] = N > 0 ? __fdiv_rn(s, float(N)) : 0.f;
  }
}

// Member order of one population for the evaluation that follows: one warp
// per domain ranks the domain's P members (P <= kOrderMaxP) by the position
// of their window on the domain's middle aperture entry (ties by index; an
// empty aperture keeps the index order), then writes member i's parameters
// to row rank(i) of theta_out and i to slots[d * P + rank(i)]. Evaluating
// theta_out with those slots as the scatter map gives every member its own
// semblance bit for bit (a pair's arithmetic does not depend on its lane),
// while the 32 lanes of a warp read windows that lie close together.
constexpr int kOrderWarps = 8;

template <int OP, bool MV>
__global__ void __launch_bounds__(32 * kOrderWarps) k_member_order(const EvalArgs a,
                                                                   float* __restrict__ theta_out,
                                                                   int* __restrict__ slots) {
  __shared__ float key[kOrderWarps][kOrderMaxP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long d = (long long)blockIdx.x * kOrderWarps + w;
  if (d >= a.n_dom) return;  // warp-uniform
  const int P = a.P;
  for (int i = lane; i < P; i += 32) {
    Lane L;
    float k = 0.f;
    if (lane_setup<OP>(a, d * P + i, L) && L.e1 > L.e0) {
      k = locate<OP, MV>(L, __ldg(a.ap_tab + ((L.e0 + L.e1) >> 1))).u;
      if (!(k == k)) k = 3.0e38f;
    }
    key[w][i] = k;
  }
  __syncwarp();
  constexpr int D = op_dim(OP);
  for (int i = lane; i < P; i += 32) {
    const float ki = key[w][i];
    int rank = 0;
    for (int j = 0; j < P; ++j) {
      const float kj = key[w][j];
      rank += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
    }
    const float* src = a.theta + (d * P + i) * D;
    float* dst = theta_out + (d * P + rank) * D;
#pragma unroll
    for (int k = 0; k < D; ++k) dst[k] = src[k];
    slots[d * P + rank] = i;
  }
}

using OFn = void (*)(const EvalArgs, float*, int*);

template <int OP>
OFn pick_order(bool mv) {
  return mv ? k_member_order<OP, true> : k_member_order<OP, false>;
}

using SFn = void (*)(const EvalArgs, float*);
enum KernelKind { kKindPacked = 0, kKindScalar = 1, kKindSplit = 2, kKindGrad = 3 };

template <int OP, int W, typename T, bool MV>
KFn pick_kind(int kind) {
  switch (kind) {
    case kKindPacked: return k_semblance<OP, W, T, MV>;
    case kKindScalar: return k_semblance_scalar<OP, W, T, MV>;
    case kKindSplit: return k_semblance_split<OP, W, T, MV>;
    case kKindGrad: return k_semblance_grad<OP, W, T, MV>;
  }
  return nullptr;
}

template <int OP, typename T, bool MV>
KFn pick_w(int kind, int W) {
  switch (W) {
    case 0: return pick_kind<OP, 0, T, MV>(kind);
    case 1: return pick_kind<OP, 1, T, MV>(kind);
    case 2: return pick_kind<OP, 2, T, MV>(kind);
    case 3: return pick_kind<OP, 3, T, MV>(kind);
    case 4: return pick_kind<OP, 4, T, MV>(kind);
    case 5: return pick_kind<OP, 5, T, MV>(kind);
    case 6: return pick_kind<OP, 6, T, MV>(kind);
    case 7: return pick_kind<OP, 7, T, MV>(kind);
    case 8: return pick_kind<OP, 8, T, MV>(kind);
  }
  return nullptr;
}

// The kernel of one kind for operator OP, storage type and half window W;
// mv selects the moveout form of the position.
template <int OP>
KFn pick_kernel(int kind, int storage, int W, bool mv) {
  const bool bf = storage == TT_STORE_BF16;
  if (mv) return bf ? pick_w<OP, __nv_bfloat16, true>(kind, W) : pick_w<OP, float, true>(kind, W);
  return bf ? pick_w<OP, __nv_bfloat16, false>(kind, W) : pick_w<OP, float, false>(kind, W);
}

template <int OP>
SFn pick_stack(int storage, bool mv) {
  const bool bf = storage == TT_STORE_BF16;
  if (mv) return bf ? k_stack<OP, __nv_bfloat16, true> : k_stack<OP, float, true>;
  return bf ? k_stack<OP, __nv_bfloat16, false> : k_stack<OP, float, false>;
}

}  // namespace sk
}  // namespace tt
