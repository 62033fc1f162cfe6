// Internal declarations shared by the libtt translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "tt.h"

namespace tt {

// parameters per operator: CMP (C), CRS (A, B, C), FO-CRS (Am, Ah, Bmm, Bmh, Bhh)
constexpr int op_dim(int op) { return op == TT_OP_CMP ? 1 : op == TT_OP_CRS ? 3 : 5; }

// Small-launch split thresholds, in 64-pair units per SM of the device
// (the SM count is queried when a context is created): a forward launch of
// fewer than n_sm * kSplitUnitsPerSm units (one warp per unit then leaves
// SMs short of their 32 resident warps) splits each unit's aperture over
// the warps of a block; up to n_sm * kSplitSmallPerSm units a unit spreads
// over kSplitSmallBlocks blocks (kSplitTinyBlocks up to n_sm / 2 units),
// below n_sm * kSplitMultiPerSm over two. The multi-block launches combine
// partial sums in context scratch: one set per (unit, block), so the scratch
// holds the largest units x blocks of any launch, at most
// max(2 kSplitMultiPerSm, kSplitSmallPerSm kSplitSmallBlocks,
// kSplitTinyBlocks / 2) n_sm sets.
constexpr int kSplitUnitsPerSm = 32;
constexpr int kSplitSmallPerSm = 2;
constexpr int kSplitMultiPerSm = 12;
constexpr int kSplitSmallBlocks = 7;
constexpr int kSplitTinyBlocks = 9;
static_assert(kSplitSmallPerSm * kSplitSmallBlocks <= 2 * kSplitMultiPerSm &&
                  kSplitTinyBlocks <= 4 * kSplitMultiPerSm,
              "every split shape fits the 2 kSplitMultiPerSm n_sm part sets");
// scratch sets (one per block of a multi-block split launch) and tickets
// (one per unit) for a device of n_sm SMs
inline long long split_part_sets(int n_sm) { return 2ll * kSplitMultiPerSm * n_sm; }
inline long long split_tickets(int n_sm) { return (long long)kSplitMultiPerSm * n_sm; }
constexpr int kSplitPartStride = 2 * 8 + 2;  // floats per pair: K + 1 for the widest window

// Padded trace layout: sample n of trace r lives at r * pitch + kPadFront + n.
// kPadFront >= max half window; kPadBack >= 2 * max half window + 2 so that a
// window whose position is clamped to ns + w reads only padding zeros.
constexpr int kPadFront = 8;
constexpr int kPadBack = 24;
constexpr int kBlock = 256;
constexpr int kOrderMaxP = 256;  // largest population the member order handles
// automatic member order: on when the mean aperture holds at least this many traces
constexpr double kOrderMinMeanAperture = 768.0;

inline int padded_pitch(int ns) { return ((kPadFront + ns + kPadBack) + 15) / 16 * 16; }

// Everything a semblance launch needs (passed by value to the kernels).
struct EvalArgs {
  const void* traces;       // padded traces, float or bf16
  const float4* ap_tab;     // per aperture entry: dm, dm^2, h^2, row offset (bits)
  const int* ap_ptr;        // [G+1]
  const float* g_inv_dt;    // [G]
  const int* dom_it0;       // [n_dom]
  const int* dom_group;     // [n_dom]
  int n_dom, P, D, op, W, storage;
  float umax;               // ns + W: positions are clamped here (window all zero)
  const float* theta;       // [n_dom][P][D]
  float* S;                 // [n_dom][P], or fit [n_dom][np_out] in scatter mode
  float* dS;                // [n_dom][P][D] (gradient launches)
  const int* slots;         // scatter mode: result (d, p) -> S[d*np_out + slots[d*P+p]]
  int np_out;
  const int* dom_map;       // optional: local domain r -> global domain (-1: skip r)
  int kernel;               // TT_KERNEL_PACKED / _PERSISTENT / _SCALAR (forward launches)
  int block;                // threads per block: 128 or 256
  int split;                // 1: small forward launches split the aperture over warps
  int split_blocks;         // blocks per unit of a split launch (set by the launcher)
  int n_sm;                 // SMs of the device (split thresholds, persistent grid)
  float* split_part;        // [split_part_sets][64][K + 1] block partial sums (s_k, E)
  double* split_part_d;     // [split_part_sets][64] block partial FP64 energies
  unsigned* split_ticket;   // [split_tickets] arrivals per unit, zero between launches
  unsigned long long* queue;  // persistent mode: work-unit counter, zero at launch
};

cudaError_t launch_semblance(const EvalArgs& a, cudaStream_t s);
cudaError_t launch_semblance_grad(const EvalArgs& a, cudaStream_t s);
// Members of each domain of theta (a.theta, a.P <= 256, no domain map) sorted
// by window position: parameters to theta_out, original slots to slots
// ([n_dom][P]); evaluate theta_out with slots as the scatter map.
cudaError_t launch_member_order(const EvalArgs& a, float* theta_out, int* slots,
                                cudaStream_t s);
cudaError_t launch_stack(const EvalArgs& a, float* out, cudaStream_t s);
cudaError_t launch_l1_probe(const float* buf, float* out, int n_sm, int iters, double* bytes,
                            cudaStream_t s);

struct DeArgs {
  int n_dom, NP, D, gen;
  const int* dom_map;       // optional: local domain -> global id keying Philox (-1: skip)
  int dom_base;             // without a map: global id = dom_base + local domain
  float* pop;
  float* fit;
  const float* trial;
  const float* tfit;
  float* next;
  int* best_idx;
  uint32_t key0, key1;
  float F;
  uint32_t cr_thr;          // floor(CR * 2^24)
  float lo[TT_MAX_DIM], hi[TT_MAX_DIM];
  // JADE adaptation (adapt == 1): per-domain state indexed like pop
  int adapt;
  int sel_gen;              // generation of the trial being selected
  float CR0;                // initial mu_CR (the initial mu_F is F)
  float* jade_mu;           // [n_dom][2]: mu_CR, mu_F
  int* jade_na;             // [n_dom] archive fill
  float* jade_arc;          // [n_dom][NP][D] archived parents
  float* jade_F;            // [n_dom][NP] F_i of the pending trial
  float* jade_CR;           // [n_dom][NP] CR_i of the pending trial
  // ENS (optional): after the selection the population's best theta and S
  // go to [global id][D] / [global id] of the sweep's best panel
  float* ens_best_th;
  float* ens_best_S;
};

cudaError_t launch_de_step(const DeArgs& a, cudaStream_t s);

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
// (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)), key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Word n of the stream of (domain d, generation g, individual i).
struct Words {
  uint32_t w[8];
  __device__ Words(uint32_t k0, uint32_t k1, uint32_t d, uint32_t g, uint32_t i, int n) {
    const uint4 a = philox4x32_10(make_uint4(i, g, d, 0u), k0, k1);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    if (n > 4) {
      const uint4 b = philox4x32_10(make_uint4(i, g, d, 1u), k0, k1);
      w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    }
  }
};

// Uniform in [0, 1) from a 32-bit word, exact in FP32: (w >> 8) 2^-24.
__device__ __forceinline__ float unit_float(uint32_t w) {
  return __uint2float_rn(w >> 8) * 5.9604644775390625e-8f;
}

__device__ __forceinline__ float rank_key(float v) { return isnan(v) ? -INFINITY : v; }

// Warp argmax of fit[0..NP) with the lowest index on ties (NaN lowest).
__device__ inline int warp_argmax(const float* fit, int NP, int lane) {
  float bk = -INFINITY;
  int bi = 0x7fffffff;
  for (int i = lane; i < NP; i += 32) {
    const float k = rank_key(fit[i]);
    if (bi == 0x7fffffff || k > bk) {
      bk = k;
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float ok = __shfl_xor_sync(0xffffffffu, bk, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ok > bk || (ok == bk && oi < bi)) {
      bk = ok;
      bi = oi;
    }
  }
  return bi;
}
cudaError_t launch_best_snapshot(int n_dom, int NP, int D, const float* pop, const float* fit,
                                 float* best_theta, float* best_S, cudaStream_t s);
// halo_prev / halo_next [n_t0][D] (may be NULL): bests of the m0 rows just
// before / after the grid, held by the neighbouring slabs of a sharded line
cudaError_t launch_exchange_plan(int n_m0, int n_t0, int NP, int D, const float* best_theta,
                                 float* pop, const float* fit, float* imports, int* slots,
                                 cudaStream_t s, const float* halo_prev = nullptr,
                                 const float* halo_next = nullptr);
cudaError_t launch_polish_update(int n_dom, int D, float* th, const float* g, const float* S,
                                 float* best_th, float* best_S, const float* lo, const float* hi,
                                 float lr, int first, int last, cudaStream_t s);

}  // namespace tt

struct tt_ctx {
  int device = 0;
  int n_sm = 1;             // multiprocessors of the device (queried at creation)
  // gathers (padded device copy)
  int n_traces = 0, ns = 0, storage = TT_STORE_F32, pitch = 0;
  void* traces = nullptr;
  float* mid = nullptr;     // copies kept to rebuild nothing; used by reloads
  float* off = nullptr;
  float* stage = nullptr;   // f32 staging rows for bf16 reloads (n_traces*ns), lazily
  // problem
  int op = 0, W = 0, D = 1, n_groups = 0, n_dom = 0, n_m0 = 0, n_t0 = 0;
  long long nnz = 0;
  float* g_inv_dt = nullptr;
  int* ap_ptr = nullptr;
  float4* ap_tab = nullptr;
  int* dom_it0 = nullptr;
  int* dom_group = nullptr;
  // search settings and scratch
  bool has_cfg = false;
  tt_de_cfg cfg{};
  float* bounds = nullptr;  // [2][D] lo, hi on the device
  float *pop = nullptr, *fit = nullptr, *trial[2] = {nullptr, nullptr};
  float* tfit[2] = {nullptr, nullptr};
  float *snap = nullptr, *imports = nullptr;
  int *slots = nullptr, *best_idx = nullptr;
  float *jade_mu = nullptr, *jade_arc = nullptr, *jade_F = nullptr, *jade_CR = nullptr;
  int* jade_na = nullptr;
  float *pol_th = nullptr, *pol_g = nullptr, *pol_S = nullptr, *pol_bth = nullptr,
        *pol_bS = nullptr;
  int* d_err = nullptr;     // device-side validation flag
  unsigned long long* queue = nullptr;  // persistent-kernel work counter
  float* split_part = nullptr;          // multi-block split scratch (tt::split_part_sets sets)
  double* split_part_d = nullptr;
  unsigned* split_ticket = nullptr;
  // a second split scratch and a side stream: the ENS sweep evaluates each
  // step's interpolated samples concurrently with the next step
  float* split_part2 = nullptr;
  double* split_part_d2 = nullptr;
  unsigned* split_ticket2 = nullptr;
  cudaStream_t side_stream = nullptr;
  cudaEvent_t side_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // launch configuration (tt_ctx_set_option / tt_ctx_autotune)
  int kernel = TT_KERNEL_PACKED, block = 256;
  bool split = true;  // TT_OPT_SPLIT
  int member_order = 2;  // TT_OPT_MEMBER_ORDER: 0 index order, 1 member order, 2 automatic
  bool use_graph = true;
  // CUDA graph of the whole search, captured on first use
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  float *out_th = nullptr, *out_S = nullptr;
  unsigned long long g_evals = 0, g_launch = 0, g_sem = 0;
  double g_trace_evals = 0;
  // CUDA graph of the ENS sweep (tt_ens_search), for the settings in ens_cfg
  cudaGraphExec_t ens_exec = nullptr;
  tt_ens_cfg ens_cfg{};
  unsigned long long ens_calls = 0, ens_launch = 0, ens_sem = 0;
  double ens_trace_evals = 0;
  std::string err;
  // counters and optional event timing of semblance launches
  double sum_N = 0;         // sum over domains of the aperture size
  unsigned long long n_launch = 0, n_sem = 0, n_timed = 0;
  double trace_evals = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev;   // pairs (start, end)
  size_t ev_used = 0;

  tt::EvalArgs eval_args(const float* theta, int P, float* S) const;
  // every semblance / gradient launch of the library goes through here
  cudaError_t semblance(const tt::EvalArgs& a, cudaStream_t s, bool grad);
  cudaError_t counted(cudaError_t e) {
    ++n_launch;
    return e;
  }
};

tt_status tt_fail(tt_ctx* ctx, tt_status code, const char* fmt, ...);
void tt_ctx_drop_graph(tt_ctx* ctx);
tt_status tt_cuda_check(tt_ctx* ctx, cudaError_t e, const char* what);
