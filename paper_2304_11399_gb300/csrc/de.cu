// Differential-evolution step (K3), best snapshot, neighbour exchange (K4)
// and the polish update, with a Philox4x32-10 counter-based generator.
//
// One warp per domain: the domain's population is staged in shared memory,
// selection and argmax are warp-local, and every individual draws its random
// words from Philox keyed by the 64-bit seed with counter
// (individual, generation, domain, block), so no generator state exists and
// any step can be recomputed or resumed bit-identically.
#include "tt_internal.cuh"

namespace tt {
namespace {

constexpr int kWarps = 4;  // domains per block

// ---- JADE adaptation (Sec. 2.1.4, the cited JADE with p = 1, c = 0.1) ----
// Draws use only correctly rounded FP32 operations so that they are
// reproducible bit for bit: pairs of Philox words on tagged counter streams
// become points of the unit square (odd multiples of 2^-24 in (-1, 1)); a
// point inside the unit disc gives a normal variate by Marsaglia's polar
// method and a Cauchy variate as the ratio of its coordinates.
constexpr uint32_t kTagArchive = 0x40000000u, kTagNormal = 0x80000000u,
                   kTagCauchy = 0xC0000000u;
constexpr int kNormalTries = 16, kCauchyTries = 32;
constexpr float kAdaptC = 0.1f, kSigma = 0.1f;

__device__ __forceinline__ float signed_unit(uint32_t x) {
  return __fmul_rn(__int2float_rn(int(2u * (x >> 8) + 1u) - (1 << 24)), 5.9604644775390625e-8f);
}

// Natural log of a positive normal float: s = m 2^e with m in [1/sqrt 2,
// sqrt 2), ln s = e ln 2 + 2 atanh(r), r = (m - 1)/(m + 1), and the atanh
// series summed to r^13 (|r| < 0.172, so the next term is below 1e-11).
__device__ float ln_series(float s) {
  const uint32_t b = __float_as_uint(s);
  int e = int((b >> 23) & 0xffu) - 126;
  float m = __uint_as_float((b & 0x007fffffu) | 0x3f000000u);  // [0.5, 1)
  if (m < 0.70710677f) {
    m = __fmul_rn(m, 2.f);
    --e;
  }
  const float r = __fdiv_rn(__fsub_rn(m, 1.f), __fadd_rn(m, 1.f));
  const float r2 = __fmul_rn(r, r);
  float p = __fdiv_rn(1.f, 13.f);
  for (int k = 5; k >= 0; --k) p = __fadd_rn(__fmul_rn(p, r2), __fdiv_rn(1.f, float(2 * k + 1)));
  return __fadd_rn(__fmul_rn(float(e), 0.6931471805599453f), __fmul_rn(__fmul_rn(2.f, r), p));
}

// k-th pair of words of the stream (individual i, tagged generation g,
// domain d): Philox block k/2, words (x, y) or (z, w)
struct PairStream {
  uint32_t k0, k1, d, g, i;
  uint4 blk;
  int cur = -1;
  __device__ PairStream(uint32_t k0_, uint32_t k1_, uint32_t d_, uint32_t g_, uint32_t i_)
      : k0(k0_), k1(k1_), d(d_), g(g_), i(i_) {}
  __device__ float pair(int k, float& v1, float& v2) {
    if ((k >> 1) != cur) {
      cur = k >> 1;
      blk = philox4x32_10(make_uint4(i, g, d, uint32_t(cur)), k0, k1);
    }
    v1 = signed_unit((k & 1) ? blk.z : blk.x);
    v2 = signed_unit((k & 1) ? blk.w : blk.y);
    return __fadd_rn(__fmul_rn(v1, v1), __fmul_rn(v2, v2));  // s
  }
};

// CR_i ~ Normal(mu_CR, 0.1) clipped to [0, 1] (z = 0 if no pair is accepted)
__device__ float jade_cr(const DeArgs& a, uint32_t gd, int i, float mu_cr) {
  PairStream ps(a.key0, a.key1, gd, kTagNormal | uint32_t(a.gen), uint32_t(i));
  float z = 0.f;
  for (int k = 0; k < kNormalTries; ++k) {
    float v1, v2;
    const float s = ps.pair(k, v1, v2);
    if (s < 1.f) {
      const float q = __fdiv_rn(__fmul_rn(-2.f, ln_series(s)), s);
      z = __fmul_rn(v1, __fsqrt_rn(q));
      break;
    }
  }
  return fminf(fmaxf(__fadd_rn(mu_cr, __fmul_rn(kSigma, z)), 0.f), 1.f);
}

// F_i ~ Cauchy(mu_F, 0.1), redrawn while <= 0, capped at 1 (mu_F if every
// try fails)
__device__ float jade_f(const DeArgs& a, uint32_t gd, int i, float mu_f) {
  PairStream ps(a.key0, a.key1, gd, kTagCauchy | uint32_t(a.gen), uint32_t(i));
  for (int k = 0; k < kCauchyTries; ++k) {
    float v1, v2;
    if (ps.pair(k, v1, v2) < 1.f) {
      const float F = __fadd_rn(mu_f, __fmul_rn(kSigma, __fdiv_rn(v1, v2)));
      if (F > 0.f) return fminf(F, 1.f);
    }
  }
  return mu_f;
}

// Selection with the archive and memory updates, one warp per domain, in
// member order: members are visited 32 at a time; the successes (strictly
// better children) of a chunk append their parents to the archive while it
// has room, else overwrite a uniformly drawn entry, the later member winning
// a shared slot; (CR_i, F_i) of the successes are summed in member order.
// mu_cr, mu_f and na are warp-uniform and updated in place.
__device__ void jade_select(const DeArgs& a, int d, uint32_t gd, float* gpop, float* gfit,
                            float* spop, float* sfit, int lane, float& mu_cr, float& mu_f,
                            int& na) {
  const int NP = a.NP, D = a.D;
  float* arc = a.jade_arc + (size_t)d * NP * D;
  float s_cr = 0.f, s_f = 0.f, s_f2 = 0.f;
  int n_succ = 0;
  for (int base = 0; base < NP; base += 32) {
    const int i = base + lane;
    const bool act = i < NP;
    float f = act ? gfit[i] : 0.f;
    const float tf = act ? a.tfit[(size_t)d * NP + i] : 0.f;
    const bool succ = act && rank_key(tf) > rank_key(f);
    const bool take = act && rank_key(tf) >= rank_key(f);
    const unsigned m = __ballot_sync(0xffffffffu, succ);
    float my_cr = 0.f, my_f = 0.f;
    if (succ) {
      my_cr = a.jade_CR[(size_t)d * NP + i];
      my_f = a.jade_F[(size_t)d * NP + i];
      int slot = na + __popc(m & ((1u << lane) - 1u));
      if (slot >= NP) {
        const uint4 w = philox4x32_10(
            make_uint4(uint32_t(i), kTagArchive | uint32_t(a.sel_gen), gd, 0u), a.key0, a.key1);
        slot = int(__umulhi(w.x, uint32_t(NP)));
      }
      const unsigned same = __match_any_sync(m, slot);
      if (31 - __clz(same) == lane)
        for (int q = 0; q < D; ++q) arc[slot * D + q] = gpop[i * D + q];
    }
    for (unsigned mm = m; mm; mm &= mm - 1) {
      const int j = __ffs(mm) - 1;
      const float c = __shfl_sync(0xffffffffu, my_cr, j);
      const float ff = __shfl_sync(0xffffffffu, my_f, j);
      s_cr = __fadd_rn(s_cr, c);
      s_f = __fadd_rn(s_f, ff);
      s_f2 = __fadd_rn(s_f2, __fmul_rn(ff, ff));
    }
    n_succ += __popc(m);
    na = min(NP, na + __popc(m));
    __syncwarp();  // the chunk's parents are archived before they are replaced
    if (act) {
      if (take) {
        f = tf;
        gfit[i] = tf;
      }
      for (int q = 0; q < D; ++q) {
        float v;
        if (take) {
          v = a.trial[((size_t)d * NP + i) * D + q];
          gpop[i * D + q] = v;
        } else {
          v = gpop[i * D + q];
        }
        spop[i * D + q] = v;
      }
      sfit[i] = f;
    }
  }
  if (n_succ) {
    const float omc = __fsub_rn(1.f, kAdaptC);
    const float mean_cr = __fdiv_rn(s_cr, float(n_succ));
    const float lehmer = __fdiv_rn(s_f2, s_f);
    mu_cr = __fadd_rn(__fmul_rn(omc, mu_cr), __fmul_rn(kAdaptC, mean_cr));
    mu_f = __fadd_rn(__fmul_rn(omc, mu_f), __fmul_rn(kAdaptC, lehmer));
  }
  if (lane == 0) {
    a.jade_na[d] = na;
    a.jade_mu[2 * (size_t)d] = mu_cr;
    a.jade_mu[2 * (size_t)d + 1] = mu_f;
  }
}

__global__ void __launch_bounds__(kWarps * 32) k_de_step(const DeArgs a) {
  extern __shared__ float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = blockIdx.x * kWarps + warp;
  if (d >= a.n_dom) return;  // uniform per warp
  const int gd = a.dom_map ? a.dom_map[d] : a.dom_base + d;  // the Philox key's domain
  if (gd < 0) return;
  const int NP = a.NP, D = a.D;
  float* gpop = a.pop + (size_t)d * NP * D;
  float* gfit = a.fit + (size_t)d * NP;
  if (a.gen == 0) {
    for (int i = lane; i < NP; i += 32) {
      Words w(a.key0, a.key1, uint32_t(gd), 0u, uint32_t(i), D);
      for (int k = 0; k < D; ++k) {
        const float u = unit_float(w.w[k]);
        gpop[i * D + k] = __fadd_rn(a.lo[k], __fmul_rn(u, __fsub_rn(a.hi[k], a.lo[k])));
      }
    }
    if (a.adapt && lane == 0) {
      a.jade_mu[2 * (size_t)d] = a.CR0;
      a.jade_mu[2 * (size_t)d + 1] = a.F;
      a.jade_na[d] = 0;
    }
    return;
  }
  float* spop = smem + (size_t)warp * NP * (D + 1);
  float* sfit = spop + NP * D;
  float mu_cr = 0.f, mu_f = 0.f;
  int na = 0;
  if (a.adapt) {
    mu_cr = a.jade_mu[2 * (size_t)d];
    mu_f = a.jade_mu[2 * (size_t)d + 1];
    na = a.jade_na[d];
  }
  // (i) greedy selection of the previous trial
  if (a.adapt && a.trial) {
    jade_select(a, d, uint32_t(gd), gpop, gfit, spop, sfit, lane, mu_cr, mu_f, na);
  } else {
    for (int i = lane; i < NP; i += 32) {
      float f = gfit[i];
      bool take = false;
      if (a.trial) {
        const float tf = a.tfit[(size_t)d * NP + i];
        take = rank_key(tf) >= rank_key(f);
        if (take) {
          f = tf;
          gfit[i] = tf;
        }
      }
      for (int k = 0; k < D; ++k) {
        float v;
        if (take) {
          v = a.trial[((size_t)d * NP + i) * D + k];
          gpop[i * D + k] = v;
        } else {
          v = gpop[i * D + k];
        }
        spop[i * D + k] = v;
      }
      sfit[i] = f;
    }
  }
  __syncwarp();
  // (ii) best = argmax, lowest index on ties
  const int b = warp_argmax(sfit, NP, lane);
  if (lane == 0 && a.best_idx) a.best_idx[d] = b;
  if (a.ens_best_th) {
    if (lane < D) a.ens_best_th[(size_t)gd * D + lane] = spop[b * D + lane];
    if (lane == 0) a.ens_best_S[gd] = sfit[b];
  }
  if (!a.next) return;
  // (iii) DE/current-to-best/1/bin + JADE bound repair, one rounding per op;
  // adaptive: per-member F_i, CR_i and r2 over population + archive
  float* gnext = a.next + (size_t)d * NP * D;
  const float* arc = a.adapt ? a.jade_arc + (size_t)d * NP * D : nullptr;
  __syncwarp();  // archive entries written by other lanes are visible
  for (int i = lane; i < NP; i += 32) {
    Words w(a.key0, a.key1, uint32_t(gd), uint32_t(a.gen), uint32_t(i), 3 + D);
    int r1 = int(__umulhi(w.w[0], uint32_t(NP - 1)));
    if (r1 >= i) ++r1;
    int r2 = int(__umulhi(w.w[1], uint32_t(NP + na - 2)));
    const int lo_i = min(i, r1), hi_i = max(i, r1);
    if (r2 >= lo_i) ++r2;
    if (r2 >= hi_i) ++r2;
    const int jr = int(__umulhi(w.w[2], uint32_t(D)));
    float F = a.F;
    uint32_t thr = a.cr_thr;
    if (a.adapt) {
      const float cr = jade_cr(a, uint32_t(gd), i, mu_cr);
      F = jade_f(a, uint32_t(gd), i, mu_f);
      thr = uint32_t(__fmul_rn(cr, 16777216.f));
      a.jade_CR[(size_t)d * NP + i] = cr;
      a.jade_F[(size_t)d * NP + i] = F;
    }
    for (int k = 0; k < D; ++k) {
      const float xi = spop[i * D + k];
      float v = xi;
      if ((w.w[3 + k] >> 8) < thr || k == jr) {
        const float xb = spop[b * D + k], x1 = spop[r1 * D + k];
        const float x2 = r2 < NP ? spop[r2 * D + k] : arc[(r2 - NP) * D + k];
        v = __fadd_rn(__fadd_rn(xi, __fmul_rn(F, __fsub_rn(xb, xi))),
                      __fmul_rn(F, __fsub_rn(x1, x2)));
      }
      if (v < a.lo[k])
        v = __fmul_rn(__fadd_rn(a.lo[k], xi), 0.5f);
      else if (v > a.hi[k])
        v = __fmul_rn(__fadd_rn(a.hi[k], xi), 0.5f);
      gnext[i * D + k] = v;
    }
  }
}

__global__ void __launch_bounds__(kWarps * 32)
    k_best_snapshot(int n_dom, int NP, int D, const float* pop, const float* fit,
                    float* best_theta, float* best_S) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = blockIdx.x * kWarps + warp;
  if (d >= n_dom) return;
  const int b = warp_argmax(fit + (size_t)d * NP, NP, lane);
  if (lane < D && best_theta) best_theta[(size_t)d * D + lane] = pop[((size_t)d * NP + b) * D + lane];
  if (lane == 0 && best_S) best_S[d] = fit[(size_t)d * NP + b];
}

// K4: the q-th present neighbour (it0-1, it0+1, m0-1, m0+1) replaces the
// q-th worst member by (fitness ascending, index ascending), the domain's
// own best excluded. Reads the best snapshot only; writes pop, imports and
// slots (the imports' fitness is written by the scatter-mode semblance).
// On a slab of a sharded line, the (m0-1) neighbour of the first row and the
// (m0+1) neighbour of the last row are rows of the neighbouring slabs, read
// from halo_prev / halo_next [n_t0][D] when given.
__global__ void __launch_bounds__(kWarps * 32)
    k_exchange_plan(int n_m0, int n_t0, int NP, int D, const float* best_theta, float* pop,
                    const float* fit, float* imports, int* slots, const float* halo_prev,
                    const float* halo_next) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = blockIdx.x * kWarps + warp;
  if (d >= n_m0 * n_t0) return;
  const int im = d / n_t0, it = d - im * n_t0;
  const float* nb[4];  // the neighbours' bests, in the order (t-1, t+1, m-1, m+1)
  int nn = 0;
  if (it > 0) nb[nn++] = best_theta + (size_t)(d - 1) * D;
  if (it < n_t0 - 1) nb[nn++] = best_theta + (size_t)(d + 1) * D;
  if (im > 0) nb[nn++] = best_theta + (size_t)(d - n_t0) * D;
  else if (halo_prev) nb[nn++] = halo_prev + (size_t)it * D;
  if (im < n_m0 - 1) nb[nn++] = best_theta + (size_t)(d + n_t0) * D;
  else if (halo_next) nb[nn++] = halo_next + (size_t)it * D;
  const float* f = fit + (size_t)d * NP;
  const int own = warp_argmax(f, NP, lane);
  int chosen[4] = {-1, -1, -1, -1};
  for (int q = 0; q < nn; ++q) {
    float bk = INFINITY;
    int bi = 0x7fffffff;
    for (int i = lane; i < NP; i += 32) {
      bool skip = i == own;
      for (int r = 0; r < q; ++r) skip |= (i == chosen[r]);
      if (skip) continue;
      const float k = rank_key(f[i]);
      if (bi == 0x7fffffff || k < bk) {
        bk = k;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const float ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ok < bk || (ok == bk && oi < bi)) {
        bk = ok;
        bi = oi;
      }
    }
    chosen[q] = bi < NP ? bi : -1;  // fewer candidates than neighbours: drop the import
  }
  while (nn > 0 && chosen[nn - 1] < 0) --nn;
  for (int t = lane; t < 4 * D; t += 32) {
    const int q = t / D, k = t - q * D;
    float v = 0.f;
    if (q < nn) {
      v = nb[q][k];
      pop[((size_t)d * NP + chosen[q]) * D + k] = v;
    }
    if (imports) imports[((size_t)d * 4 + q) * D + k] = v;
  }
  if (lane < 4) slots[(size_t)d * 4 + lane] = lane < nn ? chosen[lane] : -1;
}

// theta <- clip(theta + lr (hi - lo)^2 g, lo, hi), keeping the best iterate.
__global__ void k_polish_update(int n_dom, int D, float* th, const float* g, const float* S,
                                float* best_th, float* best_S, const float* lo,
                                const float* hi, float lr, int first, int last) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dom) return;
  const float s = S[d];
  if (first || s > best_S[d]) {
    best_S[d] = s;
    for (int k = 0; k < D; ++k) best_th[(size_t)d * D + k] = th[(size_t)d * D + k];
  }
  if (last) return;
  for (int k = 0; k < D; ++k) {
    const float r = hi[k] - lo[k];
    float v = th[(size_t)d * D + k] + lr * r * r * g[(size_t)d * D + k];
    th[(size_t)d * D + k] = fminf(fmaxf(v, lo[k]), hi[k]);
  }
}

}  // namespace

cudaError_t launch_de_step(const DeArgs& a, cudaStream_t s) {
  if (a.n_dom == 0) return cudaSuccess;
  const size_t sm = a.gen == 0 ? 0 : size_t(kWarps) * a.NP * (a.D + 1) * sizeof(float);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_de_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(sm));
    if (e != cudaSuccess) return e;
  }
  k_de_step<<<(a.n_dom + kWarps - 1) / kWarps, kWarps * 32, sm, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_best_snapshot(int n_dom, int NP, int D, const float* pop, const float* fit,
                                 float* best_theta, float* best_S, cudaStream_t s) {
  if (n_dom == 0) return cudaSuccess;
  k_best_snapshot<<<(n_dom + kWarps - 1) / kWarps, kWarps * 32, 0, s>>>(n_dom, NP, D, pop, fit,
                                                                        best_theta, best_S);
  return cudaGetLastError();
}

cudaError_t launch_exchange_plan(int n_m0, int n_t0, int NP, int D, const float* best_theta,
                                 float* pop, const float* fit, float* imports, int* slots,
                                 cudaStream_t s, const float* halo_prev,
                                 const float* halo_next) {
  const int n = n_m0 * n_t0;
  if (n == 0) return cudaSuccess;
  k_exchange_plan<<<(n + kWarps - 1) / kWarps, kWarps * 32, 0, s>>>(
      n_m0, n_t0, NP, D, best_theta, pop, fit, imports, slots, halo_prev, halo_next);
  return cudaGetLastError();
}

cudaError_t launch_polish_update(int n_dom, int D, float* th, const float* g, const float* S,
                                 float* best_th, float* best_S, const float* lo, const float* hi,
                                 float lr, int first, int last, cudaStream_t s) {
  if (n_dom == 0) return cudaSuccess;
  k_polish_update<<<(n_dom + 255) / 256, 256, 0, s>>>(n_dom, D, th, g, S, best_th, best_S, lo,
                                                      hi, lr, first, last);
  return cudaGetLastError();
}

}  // namespace tt

namespace {

tt_status need_cfg(tt_ctx* c) {
  if (!c) return tt_fail(nullptr, TT_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->has_cfg) return tt_fail(c, TT_ERR_INVALID_ARG, "context was created without a cfg");
  return TT_OK;
}

}  // namespace

tt::DeArgs tt_make_de_args(const tt_ctx* c, int gen) {
  tt::DeArgs a{};
  a.n_dom = c->n_dom;
  a.NP = c->cfg.np;
  a.D = c->D;
  a.gen = gen;
  a.key0 = uint32_t(c->cfg.seed & 0xffffffffull);
  a.key1 = uint32_t(c->cfg.seed >> 32);
  a.F = c->cfg.F;
  a.cr_thr = uint32_t(double(c->cfg.CR) * 16777216.0);
  for (int k = 0; k < TT_MAX_DIM; ++k) {
    a.lo[k] = c->cfg.lo[k];
    a.hi[k] = c->cfg.hi[k];
  }
  a.sel_gen = gen - 1;
  if (c->cfg.adapt) {
    a.adapt = 1;
    a.CR0 = c->cfg.CR;
    a.jade_mu = c->jade_mu;
    a.jade_na = c->jade_na;
    a.jade_arc = c->jade_arc;
    a.jade_F = c->jade_F;
    a.jade_CR = c->jade_CR;
  }
  return a;
}

extern "C" tt_status tt_de_step(tt_ctx* c, int32_t gen, float* pop, float* fit,
                                const float* trial, const float* trial_fit, float* next_trial,
                                int32_t* best_idx, void* stream) {
  tt_status st = need_cfg(c);
  if (st != TT_OK) return st;
  if (gen < 0) return tt_fail(c, TT_ERR_INVALID_ARG, "gen < 0");
  if (c->cfg.adapt && gen >= (1 << 30))
    return tt_fail(c, TT_ERR_INVALID_ARG, "adaptive search: gen must be below 2^30");
  if (c->n_dom > 0) {
    if (!pop) return tt_fail(c, TT_ERR_INVALID_ARG, "pop is NULL");
    if (gen > 0 && !fit) return tt_fail(c, TT_ERR_INVALID_ARG, "fit is NULL");
    if (gen > 0 && trial && !trial_fit)
      return tt_fail(c, TT_ERR_INVALID_ARG, "trial given without trial_fit");
  }
  tt::DeArgs a = tt_make_de_args(c, gen);
  a.pop = pop;
  a.fit = fit;
  a.trial = gen > 0 ? trial : nullptr;
  a.tfit = gen > 0 ? trial_fit : nullptr;
  a.next = gen > 0 ? next_trial : nullptr;
  a.best_idx = gen > 0 ? best_idx : nullptr;
  a.sel_gen = next_trial ? gen - 1 : gen;
  return tt_cuda_check(c, c->counted(tt::launch_de_step(a, static_cast<cudaStream_t>(stream))),
                       "de_step launch");
}

extern "C" tt_status tt_jade_state(tt_ctx* c, int32_t save, float* mu, int32_t* n_arc,
                                   float* archive, float* F, float* CR, void* stream) {
  tt_status st = need_cfg(c);
  if (st != TT_OK) return st;
  if (!c->cfg.adapt) return tt_fail(c, TT_ERR_INVALID_ARG, "context was created without adapt");
  if (c->n_dom == 0) return TT_OK;
  if (!mu || !n_arc || !archive || !F || !CR) return tt_fail(c, TT_ERR_INVALID_ARG, "NULL array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nd = size_t(c->n_dom), np = size_t(c->cfg.np), D = size_t(c->D);
  struct {
    void* ctx;
    void* user;
    size_t bytes;
  } parts[] = {{c->jade_mu, mu, nd * 2 * 4},
               {c->jade_na, n_arc, nd * 4},
               {c->jade_arc, archive, nd * np * D * 4},
               {c->jade_F, F, nd * np * 4},
               {c->jade_CR, CR, nd * np * 4}};
  for (auto& p : parts) {
    cudaError_t e = save ? cudaMemcpyAsync(p.user, p.ctx, p.bytes, cudaMemcpyDeviceToDevice, s)
                         : cudaMemcpyAsync(p.ctx, p.user, p.bytes, cudaMemcpyDeviceToDevice, s);
    st = tt_cuda_check(c, e, "copy adaptation state");
    if (st != TT_OK) return st;
  }
  return TT_OK;
}

extern "C" tt_status tt_best_snapshot(tt_ctx* c, const float* pop, const float* fit,
                                      float* best_theta, float* best_S, void* stream) {
  tt_status st = need_cfg(c);
  if (st != TT_OK) return st;
  if (c->n_dom > 0 && (!pop || !fit)) return tt_fail(c, TT_ERR_INVALID_ARG, "NULL array");
  return tt_cuda_check(c,
                       c->counted(tt::launch_best_snapshot(c->n_dom, c->cfg.np, c->D, pop, fit,
                                                           best_theta, best_S,
                                                           static_cast<cudaStream_t>(stream))),
                       "snapshot launch");
}

extern "C" tt_status tt_neighbor_exchange(tt_ctx* c, int32_t n_m0, int32_t n_t0,
                                          const float* best_theta, float* pop, float* fit,
                                          float* imports, int32_t* slots, void* stream) {
  tt_status st = need_cfg(c);
  if (st != TT_OK) return st;
  if (n_m0 < 0 || n_t0 < 0 || (long long)n_m0 * n_t0 != c->n_dom)
    return tt_fail(c, TT_ERR_INVALID_ARG, "n_m0 * n_t0 must equal n_dom");
  if (c->n_dom == 0) return TT_OK;
  if (!best_theta || !pop || !fit) return tt_fail(c, TT_ERR_INVALID_ARG, "NULL array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* sl = slots ? slots : c->slots;
  if (!sl) return tt_fail(c, TT_ERR_INVALID_ARG, "no slots buffer");
  float* imp = imports ? imports : c->imports;
  st = tt_cuda_check(c, c->counted(tt::launch_exchange_plan(n_m0, n_t0, c->cfg.np, c->D,
                                                            best_theta, pop, fit, imp, sl, s)),
                     "exchange launch");
  if (st != TT_OK) return st;
  tt::EvalArgs a = c->eval_args(imp, 4, fit);
  a.slots = sl;
  a.np_out = c->cfg.np;
  return tt_cuda_check(c, c->semblance(a, s, false), "import evaluation");
}
