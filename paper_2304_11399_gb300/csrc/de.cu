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

__global__ void __launch_bounds__(kWarps * 32) k_de_step(const DeArgs a) {
  extern __shared__ float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = blockIdx.x * kWarps + warp;
  if (d >= a.n_dom) return;  // uniform per warp
  const int gd = a.dom_map ? a.dom_map[d] : d;  // global id: the Philox key's domain
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
    return;
  }
  float* spop = smem + (size_t)warp * NP * (D + 1);
  float* sfit = spop + NP * D;
  // (i) greedy selection of the previous trial
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
  __syncwarp();
  // (ii) best = argmax, lowest index on ties
  const int b = warp_argmax(sfit, NP, lane);
  if (lane == 0 && a.best_idx) a.best_idx[d] = b;
  if (!a.next) return;
  // (iii) DE/current-to-best/1/bin + JADE bound repair, one rounding per op
  float* gnext = a.next + (size_t)d * NP * D;
  for (int i = lane; i < NP; i += 32) {
    Words w(a.key0, a.key1, uint32_t(gd), uint32_t(a.gen), uint32_t(i), 3 + D);
    int r1 = int(__umulhi(w.w[0], uint32_t(NP - 1)));
    if (r1 >= i) ++r1;
    int r2 = int(__umulhi(w.w[1], uint32_t(NP - 2)));
    const int lo_i = min(i, r1), hi_i = max(i, r1);
    if (r2 >= lo_i) ++r2;
    if (r2 >= hi_i) ++r2;
    const int jr = int(__umulhi(w.w[2], uint32_t(D)));
    for (int k = 0; k < D; ++k) {
      const float xi = spop[i * D + k];
      float v = xi;
      if ((w.w[3 + k] >> 8) < a.cr_thr || k == jr) {
        const float xb = spop[b * D + k], x1 = spop[r1 * D + k], x2 = spop[r2 * D + k];
        v = __fadd_rn(__fadd_rn(xi, __fmul_rn(a.F, __fsub_rn(xb, xi))),
                      __fmul_rn(a.F, __fsub_rn(x1, x2)));
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
__global__ void __launch_bounds__(kWarps * 32)
    k_exchange_plan(int n_m0, int n_t0, int NP, int D, const float* best_theta, float* pop,
                    const float* fit, float* imports, int* slots) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = blockIdx.x * kWarps + warp;
  if (d >= n_m0 * n_t0) return;
  const int im = d / n_t0, it = d - im * n_t0;
  int nb[4];
  int nn = 0;
  if (it > 0) nb[nn++] = d - 1;
  if (it < n_t0 - 1) nb[nn++] = d + 1;
  if (im > 0) nb[nn++] = d - n_t0;
  if (im < n_m0 - 1) nb[nn++] = d + n_t0;
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
      v = best_theta[(size_t)nb[q] * D + k];
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
                                 cudaStream_t s) {
  const int n = n_m0 * n_t0;
  if (n == 0) return cudaSuccess;
  k_exchange_plan<<<(n + kWarps - 1) / kWarps, kWarps * 32, 0, s>>>(n_m0, n_t0, NP, D,
                                                                    best_theta, pop, fit,
                                                                    imports, slots);
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
  return a;
}

extern "C" tt_status tt_de_step(tt_ctx* c, int32_t gen, float* pop, float* fit,
                                const float* trial, const float* trial_fit, float* next_trial,
                                int32_t* best_idx, void* stream) {
  tt_status st = need_cfg(c);
  if (st != TT_OK) return st;
  if (gen < 0) return tt_fail(c, TT_ERR_INVALID_ARG, "gen < 0");
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
  return tt_cuda_check(c, c->counted(tt::launch_de_step(a, static_cast<cudaStream_t>(stream))),
                       "de_step launch");
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
