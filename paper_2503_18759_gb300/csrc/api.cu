// C ABI of the CP-ALS-QR library: context, sweep driver (Alg. 3 with the
// schedules of Section 3.1) and the operation-level entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <stdexcept>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/cpqr.h"
#include "common.cuh"
#include "schedule.h"

using namespace cpqr;

// NVTX ranges on the host timeline of a sweep (cpqr:sweep, cpqr:ttm, cpqr:krp_qr, cpqr:update,
// cpqr:residual): a profiler selects the kernels launched inside one, e.g. ncu --nvtx
// --nvtx-include "cpqr:sweep/".  Without a tool attached they cost a call into a no-op.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

namespace {

// Section 4.2: alpha = 1/10; beta picked by fit level once the change in fit drops below 0.03.
constexpr double kAlphaDefault = 0.1;
constexpr double kActivateDfit = 0.03;
double beta_band(double fit) {
  if (fit > 0.95) return 1.0 / 20000.0;
  if (fit > 0.90) return 1.0 / 2000.0;
  if (fit > 0.70) return 1.0 / 500.0;
  return 1.0 / 250.0;
}

struct DeviceBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Caching pool for tree nodes: blocks are kept by size and reused; at release they go back to
// the process-wide cache.
class Pool {
 public:
  ~Pool() { release(); }
  cudaError_t get(size_t bytes, void** out) {
    auto it = free_.find(bytes);
    if (it != free_.end()) {
      *out = it->second;
      free_.erase(it);
      return cudaSuccess;
    }
    cudaError_t e = cache_malloc(out, bytes);
    if (e == cudaSuccess) all_.emplace_back(*out, bytes);
    return e;
  }
  void put(size_t bytes, void* p) { free_.emplace(bytes, p); }
  void release() {
    for (auto& b : all_) cache_free(b.first, b.second);
    all_.clear();
    free_.clear();
  }

 private:
  std::multimap<size_t, void*> free_;
  std::vector<std::pair<void*, size_t>> all_;
};

struct NodeBuf {
  void* p;
  size_t bytes;
  uint32_t free_mask;
  bool is_x;
  // split path: which copies the node holds, back to back in p: FP32, then bf16 hi, lo
  bool has_f32 = true;
  bool has_split = false;
  SplitLayout lay;  // the split copy's rows (last dimension padded to a multiple of 8, or dense)
};

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct Checkpoint {
  bool valid = false;
  void* arena = nullptr;  // device copy of the state arena
  std::unique_ptr<Schedule> sched;
  std::map<int, NodeBuf> nodes;
  std::vector<double> fits, betas;
  double beta_active = 0.0;
  bool activated = false;
  double last_beta = 0.0;
  int64_t sweeps = 0;
  bool has_prev[CPQR_MAXN] = {};
  double* Q0prev[CPQR_MAXN] = {};
  double* Q0 = nullptr;
  float* Q0fprev[CPQR_MAXN] = {};
  float* Q0f = nullptr;
  int next_class = -1;
};

struct cpqr_ctx {
  int N = 0, R = 0;
  std::vector<int64_t> dims;
  int tree = 2, prec = 0, extrap = 1;
  bool gram = true;  // Gram QR route (cpqr_qr_route)
  // wide-rank path (32 < R <= 192): Cholesky QRs, CUDA-core TTMs and V / finish kernels that tile the
  // columns; workspaces of the factor QR (main stream) and of the Khatri-Rao QR (side stream)
  bool wide = false;
  double* wq_main = nullptr;
  double* wq_side = nullptr;
  double* wrows = nullptr;  // I x (R + 2): rows of A^ and per-row fit terms
  double alpha = kAlphaDefault, beta_fixed = 0.0;
  cudaStream_t st = nullptr;
  cudaStream_t st2 = nullptr;      // side stream: Khatri-Rao QR overlapped with the TTM chain
  cudaEvent_t ev_ready = nullptr;  // main stream: triangles R_k of the previous update ready
  cudaEvent_t ev_z = nullptr;      // side stream: Q0, R0 of the upcoming update ready
  // Lagged fit (split path, once nothing in the next sweep depends on the fit): the explicit
  // residual of sweep k runs on st3 after the first factor QR of sweep k + 1, beside that sweep's
  // next TTM chain, and is read one sweep later.
  cudaStream_t st3 = nullptr;
  cudaEvent_t ev_prep = nullptr;   // main stream: the point after which the lagged residual runs
  cudaEvent_t ev_fit = nullptr;    // st3: lagged residual read back
  bool lag_ok = false;             // set by the sweep loops that need no fit before the next sweep
  bool resid_pending = false;      // snapshot of the factors taken, residual not launched yet
  bool resid_inflight = false;     // residual launched, fit not read yet
  // the sweep behind the pending / in-flight residual: its beta (the learned proposer's history)
  // and whether it ran inside an approval window (its fit drop is checked when the fit arrives)
  double pending_beta = 0.0, inflight_beta = 0.0;
  bool pending_check = false, inflight_check = false;
  bool sweep_check = false;        // the sweep being run is inside an approval window
  int64_t lagged_fits = 0;
  bool z_pending = false;
  int z_mode = -1;
  const void* X = nullptr;
  bool x64 = false;
  int64_t nX = 0;
  cpqr_status err = CPQR_OK;

  std::vector<std::pair<void*, size_t>> owned;  // from the block cache, returned at destroy
  void* arena = nullptr;     // every per-mode state array (factors, QRs, Q0 history, staging)
  size_t arena_bytes = 0;
  Checkpoint ckpt[3];        // 0: caller's slot, 1 and 2: the two branches of a judged proposal
  std::map<int, NodeBuf> orphans;  // nodes freed while a checkpoint still references them
  // learned proposer: FP32 parameters, their bf16 transposed copy, and the device state (fit /
  // beta history, rule state, proposal) in the state arena
  float* mlp_params = nullptr;
  __nv_bfloat16* mlp_wt = nullptr;
  MlpState* mlp_state = nullptr;
  int next_class = -1;        // proposal for the next sweep, read with the last sweep's fit
  // judging: a proposal that beat the rule's sweep from the same checkpoint stays approved for
  // approve_left more sweeps while the fit does not drop; each win doubles the window (<= kWindowCap)
  int approved_class = -1, approve_window = 1, approve_left = 0;
  // after a loss the rule runs unjudged for hold_left sweeps; consecutive losses double the hold
  int hold_window = 1, hold_left = 0;
  int64_t judged = 0, preapproved = 0, deferred = 0;
  double* A[CPQR_MAXN] = {};
  double* Q[CPQR_MAXN] = {};
  double* Rf[CPQR_MAXN] = {};
  float* Qf[CPQR_MAXN] = {};
  double* Q0prev[CPQR_MAXN] = {};
  bool has_prev[CPQR_MAXN] = {};
  __nv_bfloat16* Qt[CPQR_MAXN] = {};
  int Rp = 0;
  int64_t Kp[CPQR_MAXN] = {};
  __nv_bfloat16 *Xhi = nullptr, *Xlo = nullptr;
  SplitLayout xlay;  // the split X's rows padded to a multiple of 8 when the last side is not
  double* lambda = nullptr;
  double* Q0 = nullptr;
  float* Q0f = nullptr;                // split path: FP32 copy of Q0 for V = Y_(n) Q0
  float* Q0fprev[CPQR_MAXN] = {};      // split path: FP32 copies of Q0^{k-1}
  double* R0 = nullptr;
  double* V = nullptr;                 // rows of A^ = V^ R0^{-T}
  double* fitpart = nullptr;           // per-block partial fit terms of the finish preparation
  double* qr_work = nullptr;
  double* zq_work = nullptr;
  double* zg_work = nullptr;       // Gram-route Khatri-Rao QR workspace
  // per mode (state arena): equilibrated Gram of the factor (float-float, 32 x 32 upper) and
  // its column norms, from which the Gram route's Khatri-Rao Cholesky is formed
  float2* Gf[CPQR_MAXN] = {};
  double* cn[CPQR_MAXN] = {};
  int zchol_mode = -1;               // mode whose Khatri-Rao Cholesky is already issued on st2
  bool zchol_split = false;          // ... and it is the split route's (all m Grams, W's guard)
  // Split Khatri-Rao QR (Gram route, N - 1 >= 3 triangles): right behind the QR for mode n, st2
  // forms the QR of W, the product of the triangles of every mode but n and the update after n
  // (they are final by then); that next update's QR then waits for its last level only, the one
  // with R_n.  Stream order on st2 keeps W's buffers apart from their previous reader.
  double* wg_work = nullptr;
  double* wq_work = nullptr;
  double* WQ = nullptr;  // Q_W, R^(N-2) x R
  double* WS = nullptr;  // S_W, R x R
  bool w_ok = false;     // the buffers above exist (N - 1 >= 3)
  int wpf_mode = -1;     // the update whose W is formed; -1: none
  int wpf_excl = -1;     // the update before it, left out of W
  int last_updated = -1;  // mode of the last update enqueued
  int next_first = -1;    // first update of the sweep after the current one (-1: unknown)
  int64_t n_split = 0;    // Khatri-Rao QRs issued on the split route
  cudaEvent_t ev_gram = nullptr;     // main stream: the last factor's Gram stored
  double* fg_work = nullptr;       // Gram-route factor QR workspace
  double* hpart = nullptr;         // per-block folded Gram partials of A^ (finish prep)
  double* v_work = nullptr;
  double* res_work = nullptr;
  double* fit_terms = nullptr;
  double* d_scalar = nullptr;
  unsigned int* dstatus = nullptr;
  double* h_pinned = nullptr;  // 4 doubles: fit terms, status
  int32_t* d_perm = nullptr;
  ZPlan zplan{};   // Khatri-Rao row plan of the N-1 triangles
  int32_t* d_perm2 = nullptr;
  ZPlan zplan2{};  // plan of a two-triangle product (nested QR for N - 1 >= 3)

  std::unique_ptr<Schedule> sched;
  std::vector<Op> ops;
  std::map<int, NodeBuf> nodes;
  Pool pool;

  // per-launch timing (CUDA events on st), buckets of cpqr.h
  bool timing = false;
  std::vector<cudaEvent_t> evpool;
  std::vector<std::pair<int, int>> evused;  // (bucket, index of start event; end = +1)
  int evnext = 0;                           // next free pair in evpool (groups may nest)
  double ms_bucket[CPQR_NBUCKETS] = {};
  int64_t n_bucket[CPQR_NBUCKETS] = {};
  int64_t launches = 0;

  double normX2 = 0.0;
  std::vector<double> betas;
  std::vector<double> fits;
  double beta_active = 0.0;
  bool activated = false;
  double last_beta = 0.0;
  int64_t sweeps = 0;
  int64_t proposals = 0, accepted = 0;
  // failure-detection test hook (cp_als_qr_test_wait_timeout): the next tensor-core TTM issues no
  // tile loads and its pipeline waits give up after test_wait_ns
  bool test_skip_next_ttm = false;
  unsigned long long test_wait_ns = 0;

  ~cpqr_ctx() {
    if (st) cudaStreamSynchronize(st);
    if (st2) cudaStreamSynchronize(st2);
    if (st3) cudaStreamSynchronize(st3);
    for (cudaEvent_t e : evpool) cudaEventDestroy(e);
    if (ev_prep) cudaEventDestroy(ev_prep);
    if (ev_fit) cudaEventDestroy(ev_fit);
    if (st3) cudaStreamDestroy(st3);
    for (Checkpoint& c : ckpt)
      if (c.arena) cache_free(c.arena, arena_bytes);
    if (ev_ready) cudaEventDestroy(ev_ready);
    if (ev_z) cudaEventDestroy(ev_z);
    if (ev_gram) cudaEventDestroy(ev_gram);
    if (st2) cudaStreamDestroy(st2);
    pool.release();
    for (auto& b : owned) cache_free(b.first, b.second);
    if (h_pinned) cache_free_host(h_pinned, 8 * sizeof(double));
  }

  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cache_malloc(&q, bytes);
    if (e == cudaSuccess) {
      owned.emplace_back(q, bytes);
      *p = static_cast<T*>(q);
    }
    return e;
  }
};

#define CK(...)                                                           \
  do {                                                                    \
    cudaError_t e_ = (__VA_ARGS__);                                            \
    if (e_ != cudaSuccess) {                                              \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? CPQR_ENOMEM : CPQR_ECUDA); \
    }                                                                     \
  } while (0)

namespace {

cpqr_status fail(cpqr_ctx* ctx, cpqr_status s) {
  if (ctx && ctx->err == CPQR_OK) ctx->err = s;
  return s;
}

// Brackets one launch group with CUDA events when timing is on.
struct Timed {
  cpqr_ctx* ctx;
  int bucket;
  int idx = -1;
  cudaStream_t s;
  Timed(cpqr_ctx* c, int b, int nlaunch, cudaStream_t stream = nullptr) : ctx(c), bucket(b) {
    s = stream ? stream : ctx->st;
    ctx->launches += nlaunch;
    if (!ctx->timing) return;
    idx = ctx->evnext;
    ctx->evnext += 2;
    while ((int)ctx->evpool.size() < idx + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        idx = -1;
        return;
      }
      ctx->evpool.push_back(e);
    }
    cudaEventRecord(ctx->evpool[idx], s);
  }
  ~Timed() {
    if (idx < 0) return;
    cudaEventRecord(ctx->evpool[idx + 1], s);
    ctx->evused.push_back({bucket, idx});
  }
};

void collect_timing(cpqr_ctx* ctx) {
  for (auto& u : ctx->evused) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->evpool[u.second], ctx->evpool[u.second + 1]) == cudaSuccess) {
      ctx->ms_bucket[u.first] += ms;
      ctx->n_bucket[u.first] += 1;
    }
  }
  ctx->evused.clear();
  ctx->evnext = 0;
}

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Khatri-Rao row order for the staircase QR: rows sorted by their largest digit.
std::vector<int32_t> krp_perm(int m, int R) {
  int64_t M = ipow(R, m);
  std::vector<std::vector<int32_t>> buckets(R);
  for (int64_t idx = 0; idx < M; ++idx) {
    int64_t x = idx;
    int mx = 0;
    for (int k = 0; k < m; ++k) {
      mx = std::max<int>(mx, (int)(x % R));
      x /= R;
    }
    buckets[mx].push_back((int32_t)idx);
  }
  std::vector<int32_t> perm;
  perm.reserve(M);
  for (auto& b : buckets) perm.insert(perm.end(), b.begin(), b.end());
  return perm;
}

std::vector<int64_t> node_dims(const cpqr_ctx* ctx, uint32_t mask) {
  std::vector<int64_t> d(ctx->N);
  for (int k = 0; k < ctx->N; ++k) d[k] = (mask & (1u << k)) ? ctx->dims[k] : ctx->R;
  return d;
}

size_t elem_size_of_nodes(const cpqr_ctx* ctx) { return ctx->prec == CPQR_PREC_FP64 ? 8 : 4; }

size_t align16(size_t b) { return (b + 15) / 16 * 16; }

// Split-path tree nodes hold what their consumers read: the bf16 hi / lo split (the operand
// of the tensor-core TTMs) for a node with two or more uncontracted modes, the FP32 tensor for
// a leaf (V = Y_(n) Q0) and for a node that a CUDA-core TTM will read.
// The split copy of a node whose last dimension is `last`: rows padded to a multiple of 8 (so that
// every TTM over it can take the tensor cores) unless already one.
SplitLayout node_split_layout(int64_t last) {
  SplitLayout l;
  if (last % 8 != 0) {
    l.last = last;
    l.ld = (last + 7) / 8 * 8;
  }
  return l;
}
int64_t split_elems(int64_t n, SplitLayout lay) { return lay.ld ? n / lay.last * lay.ld : n; }
size_t split_node_bytes(int64_t n, bool f32, bool split, SplitLayout lay) {
  return (f32 ? align16((size_t)n * 4) : 0) + (split ? 2 * align16((size_t)split_elems(n, lay) * 2) : 0);
}
void split_views(void* base, int64_t n, bool f32, SplitLayout lay, __nv_bfloat16** hi, __nv_bfloat16** lo) {
  char* b = static_cast<char*>(base) + (f32 ? align16((size_t)n * 4) : 0);
  *hi = reinterpret_cast<__nv_bfloat16*>(b);
  *lo = reinterpret_cast<__nv_bfloat16*>(b + align16((size_t)split_elems(n, lay) * 2));
}

cpqr_status run_ttm(cpqr_ctx* ctx, const Op& op) {
  NvtxRange nvtx_range("cpqr:ttm");
  const int dst = op.a, src = op.b, k = op.c;
  auto it = ctx->nodes.find(src);
  if (it == ctx->nodes.end()) return fail(ctx, CPQR_EINVAL);
  const NodeBuf sb = it->second;
  std::vector<int64_t> d = node_dims(ctx, sb.free_mask);
  int64_t P = 1, S = 1;
  for (int j = 0; j < k; ++j) P *= d[j];
  for (int j = k + 1; j < ctx->N; ++j) S *= d[j];
  const int64_t K = d[k];
  const int R = ctx->R;
  const size_t es = elem_size_of_nodes(ctx);
  const bool split = ctx->prec == CPQR_PREC_SPLIT_BF16;
  const int64_t n_out = P * R * S;
  const uint32_t out_mask = sb.free_mask & ~(1u << k);
  // split path: which copies the output needs (see split_node_bytes)
  bool need_f32 = true, need_split = false;
  SplitLayout olay;
  if (split) {
    const std::vector<int64_t> od = node_dims(ctx, out_mask);
    olay = node_split_layout(od[ctx->N - 1]);
    int nfree = 0;
    bool cuda_core_consumer = false;
    for (int j = 0; j < ctx->N; ++j) {
      if (!(out_mask & (1u << j))) continue;
      ++nfree;
      int64_t Pj = 1, Sj = 1;
      for (int q = 0; q < j; ++q) Pj *= od[q];
      for (int q = j + 1; q < ctx->N; ++q) Sj *= od[q];
      if (!(ctx->wide ? ttm_tc_wide_supported(Pj, od[j], Sj, R, olay) : ttm_tc_supported(Pj, od[j], Sj, R, olay)))
        cuda_core_consumer = true;
    }
    need_split = nfree >= 2;
    need_f32 = nfree < 2 || cuda_core_consumer;
    if (!need_split) olay = SplitLayout{};
  }
  const size_t bytes = split ? split_node_bytes(n_out, need_f32, need_split, olay) : (size_t)n_out * es;
  void* out = nullptr;
  CK(ctx->pool.get(bytes, &out));
  cudaStream_t st = ctx->st;
  Timed tm(ctx, sb.is_x ? CPQR_BUCKET_TTM_FULL : CPQR_BUCKET_TTM_DEEP, 1);
  if (!split && ctx->wide) {
    if (sb.is_x && !ctx->x64)
      CK((launch_ttm_wide<float, double, double, double>((const float*)sb.p, ctx->Q[k], (double*)out, P, K, S, R,
                                                         st)));
    else
      CK((launch_ttm_wide<double, double, double, double>((const double*)sb.p, ctx->Q[k], (double*)out, P, K, S, R,
                                                          st)));
  } else if (!split) {
    if (sb.is_x && !ctx->x64)
      CK(launch_ttm<float, double, double>((const float*)sb.p, ctx->Q[k], (double*)out, P, K, S, R, st));
    else
      CK(launch_ttm<double, double, double>((const double*)sb.p, ctx->Q[k], (double*)out, P, K, S, R, st));
  } else if (ctx->wide) {
    __nv_bfloat16 *ohi = nullptr, *olo = nullptr;
    if (need_split) split_views(out, n_out, need_f32, olay, &ohi, &olo);
    float* of = need_f32 ? static_cast<float*>(out) : nullptr;
    const SplitLayout lay = sb.is_x ? ctx->xlay : sb.lay;
    if (ttm_tc_wide_supported(P, K, S, R, lay) && (sb.is_x || sb.has_split)) {
      const __nv_bfloat16 *shi = ctx->Xhi, *slo = ctx->Xlo;
      if (!sb.is_x) {
        __nv_bfloat16 *h, *l;
        split_views(sb.p, P * K * S, sb.has_f32, sb.lay, &h, &l);
        shi = h;
        slo = l;
      }
      CK(launch_ttm_tc_wide(shi, slo, ctx->Qt[k], ctx->Rp, ctx->Kp[k], of, P, K, S, R, ctx->dstatus, st, ohi, olo,
                            lay, olay));
    } else {
      // the CUDA-core FP32 TTM from the node's FP32 copy (kept for every CUDA-core consumer)
      if (!sb.has_f32) return fail(ctx, CPQR_EINVAL);
      float* o32 = of;
      if (!o32) {
        void* tmp = nullptr;
        CK(ctx->pool.get((size_t)n_out * 4, &tmp));
        o32 = static_cast<float*>(tmp);
      }
      CK((launch_ttm_wide<float, float, float, float>((const float*)sb.p, ctx->Qf[k], o32, P, K, S, R, st)));
      if (need_split) {
        if (olay.ld)
          CK(launch_split_x_padded(o32, ohi, olo, n_out / olay.last, olay.last, olay.ld, st));
        else
          CK(launch_split_x(o32, ohi, olo, n_out, st));
        ctx->launches += 1;
      }
      if (!of) ctx->pool.put((size_t)n_out * 4, o32);
    }
  } else {
    __nv_bfloat16 *ohi = nullptr, *olo = nullptr;
    if (need_split) split_views(out, n_out, need_f32, olay, &ohi, &olo);
    float* of = need_f32 ? static_cast<float*>(out) : nullptr;
    const SplitLayout lay = sb.is_x ? ctx->xlay : sb.lay;
    if (ttm_tc_supported(P, K, S, R, lay) && (sb.is_x || sb.has_split)) {
      const __nv_bfloat16 *shi = ctx->Xhi, *slo = ctx->Xlo;
      if (!sb.is_x) {
        __nv_bfloat16 *h, *l;
        split_views(sb.p, P * K * S, sb.has_f32, sb.lay, &h, &l);
        shi = h;
        slo = l;
      }
      // a Householder Khatri-Rao QR running on the side stream holds one 16-CTA cluster: the
      // persistent grid then leaves a GPC free so that the two overlap instead of queueing behind
      // each other.  That costs the TTM a third of the SMs (one 16-CTA cluster per GPC), so the
      // Gram route, whose side-stream work is row kernels plus a fallback that returns at once,
      // gives the TTM the whole GPU.
      const int reserve = (ctx->z_pending && !ctx->gram) ? qr_cluster_sms() : 0;
      const bool skip = ctx->test_skip_next_ttm;
      ctx->test_skip_next_ttm = false;
      CK(launch_ttm_tc(shi, slo, ctx->Qt[k], ctx->Rp, ctx->Kp[k], of, P, K, S, R, ctx->dstatus, st, reserve, ohi,
                       olo, skip ? ctx->test_wait_ns : 0, skip ? 1 : 0, lay, olay));
    } else {
      if (!sb.has_f32) return fail(ctx, CPQR_EINVAL);  // not produced for a CUDA-core consumer
      float* o32 = of;
      if (!o32) {  // scratch FP32 output from the pool, split below
        void* tmp = nullptr;
        CK(ctx->pool.get((size_t)n_out * 4, &tmp));
        o32 = static_cast<float*>(tmp);
      }
      cudaError_t e = launch_ttm_f32_tiled((const float*)sb.p, ctx->Qf[k], o32, P, K, S, R, st);
      if (e == cudaErrorNotSupported) e = launch_ttm<float, float, float>((const float*)sb.p, ctx->Qf[k], o32, P, K,
                                                                           S, R, st);
      CK(e);
      if (need_split) {
        if (olay.ld)
          CK(launch_split_x_padded(o32, ohi, olo, n_out / olay.last, olay.last, olay.ld, st));
        else
          CK(launch_split_x(o32, ohi, olo, n_out, st));
        ctx->launches += 1;
      }
      if (!of) ctx->pool.put((size_t)n_out * 4, o32);  // stream order protects it until the split ran
    }
  }
  NodeBuf nb{out, bytes, out_mask, false};
  nb.has_f32 = need_f32;
  nb.has_split = need_split;
  nb.lay = olay;
  ctx->nodes[dst] = nb;
  return CPQR_OK;
}

bool pinned(const cpqr_ctx* ctx, int id) {
  for (const Checkpoint& c : ctx->ckpt)
    if (c.valid && c.nodes.count(id)) return true;
  return false;
}

void free_node(cpqr_ctx* ctx, int id) {
  auto it = ctx->nodes.find(id);
  if (it == ctx->nodes.end() || it->second.is_x) return;
  if (pinned(ctx, id)) ctx->orphans[id] = it->second;  // a checkpoint still needs its contents
  else ctx->pool.put(it->second.bytes, it->second.p);
  ctx->nodes.erase(it);
}

// Returns orphaned node buffers that no checkpoint and no live node references to the pool.
void sweep_orphans(cpqr_ctx* ctx) {
  for (auto it = ctx->orphans.begin(); it != ctx->orphans.end();) {
    if (!pinned(ctx, it->first) && !ctx->nodes.count(it->first)) {
      ctx->pool.put(it->second.bytes, it->second.p);
      it = ctx->orphans.erase(it);
    } else {
      ++it;
    }
  }
}

cpqr_status checkpoint_save(cpqr_ctx* ctx, int slot) {
  Checkpoint& c = ctx->ckpt[slot];
  if (!c.arena) CK(cache_malloc(&c.arena, ctx->arena_bytes));
  CK(cudaMemcpyAsync(c.arena, ctx->arena, ctx->arena_bytes, cudaMemcpyDeviceToDevice, ctx->st));
  if (c.valid) {  // re-saving: previously pinned nodes may become free
    c.valid = false;
    sweep_orphans(ctx);
  }
  c.sched.reset(new Schedule(*ctx->sched));
  c.nodes = ctx->nodes;
  c.fits = ctx->fits;
  c.betas = ctx->betas;
  c.beta_active = ctx->beta_active;
  c.activated = ctx->activated;
  c.last_beta = ctx->last_beta;
  c.sweeps = ctx->sweeps;
  for (int n = 0; n < CPQR_MAXN; ++n) {
    c.has_prev[n] = ctx->has_prev[n];
    c.Q0prev[n] = ctx->Q0prev[n];
    c.Q0fprev[n] = ctx->Q0fprev[n];
  }
  c.Q0 = ctx->Q0;
  c.Q0f = ctx->Q0f;
  c.next_class = ctx->next_class;
  c.valid = true;
  return CPQR_OK;
}

cpqr_status checkpoint_restore(cpqr_ctx* ctx, int slot) {
  Checkpoint& c = ctx->ckpt[slot];
  if (!c.valid) return CPQR_EINVAL;
  CK(cudaMemcpyAsync(ctx->arena, c.arena, ctx->arena_bytes, cudaMemcpyDeviceToDevice, ctx->st));
  for (auto& kv : ctx->nodes) {
    if (kv.second.is_x || c.nodes.count(kv.first)) continue;
    if (pinned(ctx, kv.first)) ctx->orphans[kv.first] = kv.second;
    else ctx->pool.put(kv.second.bytes, kv.second.p);
  }
  ctx->nodes = c.nodes;
  for (auto& kv : ctx->nodes) ctx->orphans.erase(kv.first);
  ctx->sched.reset(new Schedule(*c.sched));
  ctx->fits = c.fits;
  ctx->betas = c.betas;
  ctx->beta_active = c.beta_active;
  ctx->activated = c.activated;
  ctx->last_beta = c.last_beta;
  ctx->sweeps = c.sweeps;
  for (int n = 0; n < CPQR_MAXN; ++n) {
    ctx->has_prev[n] = c.has_prev[n];
    ctx->Q0prev[n] = c.Q0prev[n];
    ctx->Q0fprev[n] = c.Q0fprev[n];
  }
  ctx->Q0 = c.Q0;
  ctx->Q0f = c.Q0f;
  ctx->next_class = c.next_class;
  ctx->z_pending = false;
  ctx->zchol_mode = -1;
  ctx->wpf_mode = -1;
  ctx->last_updated = -1;
  return CPQR_OK;
}

void checkpoint_drop(cpqr_ctx* ctx, int slot) {
  Checkpoint& c = ctx->ckpt[slot];
  if (!c.valid) return;
  c.valid = false;
  c.nodes.clear();
  c.sched.reset();
  sweep_orphans(ctx);
}

cpqr_status stage_q(cpqr_ctx* ctx, int n) {
  if (ctx->prec != CPQR_PREC_SPLIT_BF16) return CPQR_OK;
  Timed tm(ctx, CPQR_BUCKET_OTHER, 1);
  CK(launch_split_q(ctx->Q[n], ctx->dims[n], ctx->R, ctx->Qt[n], ctx->Rp, ctx->Kp[n], ctx->st));
  return CPQR_OK;
}

// The stored Grams and column norms of the modes other than n (ascending, as the triangles of Z_n).
GramPtrs z_grams(const cpqr_ctx* ctx, int n) {
  GramPtrs gp{};
  int m = 0;
  for (int k = 0; k < ctx->N; ++k)
    if (k != n) {
      gp.g[m] = ctx->Gf[k];
      gp.s[m] = ctx->cn[k];
      ++m;
    }
  return gp;
}

// The Grams of the first Cholesky of Z_n's Gram-route QR: the last two triangles (level 2 of the
// nested QR; all of Z_n for an order-3 tensor).
GramPtrs z_grams_level2(const cpqr_ctx* ctx, int n) {
  const GramPtrs all = z_grams(ctx, n);
  const int m = ctx->N - 1;
  GramPtrs g2{};
  g2.g[0] = all.g[m - 2];
  g2.s[0] = all.s[m - 2];
  g2.g[1] = all.g[m - 1];
  g2.s[1] = all.s[m - 1];
  return g2;
}

// The QR of W for the update `after` (the one that follows n): the triangles of every mode but n
// and `after`, final once the update before n has run.  On st2 behind the QR for mode n: beside
// it on a stream of its own, W's kernels shared the SMs with the TTM chain's persistent grid and
// held it back by about what they saved (48^5, R = 16: 1.945 against 1.928 ms per sweep).
cpqr_status launch_w(cpqr_ctx* ctx, int n, int after) {
  TriPtrs tw{};
  GramPtrs gw{};
  int mw = 0;
  for (int k = 0; k < ctx->N; ++k)
    if (k != n && k != after) {
      tw.p[mw] = ctx->Rf[k];
      gw.g[mw] = ctx->Gf[k];
      gw.s[mw] = ctx->cn[k];
      ++mw;
    }
  GramPtrs g2{};
  g2.g[0] = gw.g[mw - 2];
  g2.s[0] = gw.s[mw - 2];
  g2.g[1] = gw.g[mw - 1];
  g2.s[1] = gw.s[mw - 1];
  {
    Timed tm(ctx, CPQR_BUCKET_Q0, 1, ctx->st2);
    CK(launch_krp_chol(g2, 2, ctx->R, ctx->wg_work, ctx->st2));
    int nl = 0;
    CK(launch_krp_rows(ctx->zplan2, tw, mw, gw, ctx->WQ, ctx->WS, ctx->wg_work, ctx->wq_work, ctx->dstatus, ctx->st2,
                       nullptr, &nl, false));
    ctx->launches += nl;
  }
  ctx->wpf_mode = after;
  ctx->wpf_excl = n;
  return CPQR_OK;
}

// Whether the split route serves the QR for mode n: W formed for n, leaving out the last update.
bool split_ready(const cpqr_ctx* ctx, int n) {
  return ctx->gram && ctx->w_ok && ctx->wpf_mode == n && ctx->last_updated >= 0 &&
         ctx->wpf_excl == ctx->last_updated && ctx->last_updated != n;
}

// Alg. 3 lines 3-4 for mode n: QR of the Khatri-Rao product of the other triangles,
// issued on the side stream as soon as the previous update has produced its R_k so
// that it runs under the TTM chain of mode n.  On the Gram route its Cholesky may already be
// on the side stream (issued by the previous update once its factor's Gram existed); with a W
// formed for n, only the level with the last update's triangle is left (split route), and the W
// of the update after n (`after`, -1 if none in this sweep) is started.
cpqr_status launch_z(cpqr_ctx* ctx, int n, int after) {
  NvtxRange nvtx_range("cpqr:krp_qr");
  TriPtrs tri{};
  int m = 0, s = -1;
  for (int k = 0; k < ctx->N; ++k)
    if (k != n) {
      if (k == ctx->last_updated) s = m;
      tri.p[m++] = ctx->Rf[k];
    }
  const bool split = split_ready(ctx, n) && s >= 0;
  CK(cudaEventRecord(ctx->ev_ready, ctx->st));
  CK(cudaStreamWaitEvent(ctx->st2, ctx->ev_ready, 0));
  {
    Timed tm(ctx, CPQR_BUCKET_Q0, 1, ctx->st2);
    if (ctx->wide) {
      CK(launch_wide_qr(nullptr, ipow(ctx->R, m), ctx->R, tri.p, m, ctx->Q0, ctx->Q0f, ctx->R0, ctx->wq_side,
                        ctx->dstatus, ctx->st2));
    } else if (split) {
      if (!(ctx->zchol_mode == n && ctx->zchol_split)) {
        CK(launch_krp_chol(z_grams(ctx, n), m, ctx->R, ctx->zg_work, ctx->st2, 0, gram_flag(ctx->wg_work)));
        ctx->launches += 1;
      }
      int nl = 0;
      CK(launch_krp_rows_split(ctx->zplan2, tri, m, s, ctx->WQ, ctx->WS, ctx->Q0, ctx->R0, ctx->zg_work, ctx->zq_work,
                               ctx->dstatus, ctx->st2, ctx->Q0f, &nl));
      ctx->launches += nl - 1;
      ctx->n_split += 1;
    } else if (ctx->gram) {
      if (!(ctx->zchol_mode == n && !ctx->zchol_split)) {
        CK(launch_krp_chol(z_grams_level2(ctx, n), 2, ctx->R, ctx->zg_work, ctx->st2));
        ctx->launches += 1;
      }
      int nl = 0;
      CK(launch_krp_rows(ctx->zplan2, tri, m, z_grams(ctx, n), ctx->Q0, ctx->R0, ctx->zg_work, ctx->zq_work,
                         ctx->dstatus, ctx->st2, ctx->Q0f, &nl));
      ctx->launches += nl - 1;
    } else if (m >= 3) {
      int nl = 0;
      CK(launch_krp_qr_nested(ctx->zplan2, tri, m, ctx->Q0, ctx->R0, ctx->zq_work, ctx->dstatus, ctx->st2, ctx->Q0f,
                              &nl));
      ctx->launches += nl - 1;
    } else {
      CK(launch_krp_qr(ctx->zplan, tri, ctx->Q0, ctx->R0, ctx->zq_work, ctx->dstatus, ctx->st2, ctx->Q0f));
    }
  }
  ctx->zchol_mode = -1;
  ctx->wpf_mode = -1;
  CK(cudaEventRecord(ctx->ev_z, ctx->st2));
  ctx->z_pending = true;
  ctx->z_mode = n;
  if (ctx->gram && ctx->w_ok && m >= 3 && after >= 0 && after != n) {
    cpqr_status st = launch_w(ctx, n, after);
    if (st != CPQR_OK) return st;
  }
  return CPQR_OK;
}

cpqr_status launch_lagged_residual(cpqr_ctx* ctx);

cpqr_status run_update(cpqr_ctx* ctx, int n, int leaf, double beta, int next_mode) {
  NvtxRange nvtx_range("cpqr:update");
  auto it = ctx->nodes.find(leaf);
  if (it == ctx->nodes.end()) return fail(ctx, CPQR_EINVAL);
  const NodeBuf lb = it->second;
  const int N = ctx->N, R = ctx->R;
  cudaStream_t st = ctx->st;
  if (!ctx->z_pending || ctx->z_mode != n) {
    cpqr_status s = launch_z(ctx, n, next_mode);
    if (s != CPQR_OK) return s;
  }
  CK(cudaStreamWaitEvent(st, ctx->ev_z, 0));
  ctx->z_pending = false;
  // Lines 5 and 7: V = Y_(n) [Q0 | Q0^{k-1}] as split-K slices.
  int64_t P = ipow(R, n), S = ipow(R, N - 1 - n);
  const int64_t I = ctx->dims[n];
  const bool ext = (beta != 0.0) && ctx->has_prev[n];
  const int C = ext ? 2 * R : R;
  const bool fp64 = ctx->prec == CPQR_PREC_FP64;
  int nparts = 0;
  {
    Timed tm(ctx, CPQR_BUCKET_APPLY_Q0, 1);
    if (fp64)
      CK(launch_leaf_v<double, double>((const double*)lb.p, P, I, S, ctx->Q0, ctx->Q0prev[n], R, C, ctx->v_work,
                                       &nparts, st));
    else
      CK(launch_leaf_v<float, float>((const float*)lb.p, P, I, S, ctx->Q0f, ctx->Q0fprev[n], R, C,
                                     (float*)ctx->v_work, &nparts, st));
  }
  if (ctx->wide) {
    // Lines 8-10 on the wide path: eq. 19, the R0^{-T} solve, lambda, then the factor's Cholesky QR
    Timed tm(ctx, CPQR_BUCKET_QR, 12);
    const double b = ext ? beta : 0.0;
    if (fp64)
      CK(launch_wide_finish<double>(ctx->v_work, nparts, I, C, R, ctx->R0, b, ctx->alpha, ctx->A[n], ctx->lambda,
                                    ctx->fit_terms, ctx->wrows, ctx->dstatus, st));
    else
      CK(launch_wide_finish<float>((const float*)ctx->v_work, nparts, I, C, R, ctx->R0, b, ctx->alpha, ctx->A[n],
                                   ctx->lambda, ctx->fit_terms, ctx->wrows, ctx->dstatus, st));
    CK(launch_wide_qr(ctx->A[n], I, R, nullptr, 0, ctx->Q[n], ctx->Qf[n], ctx->Rf[n], ctx->wq_main, ctx->dstatus,
                      st));
    if (!fp64) {  // the tensor cores' operand: bf16 hi / lo of the new Q_n^T
      cpqr_status sq = stage_q(ctx, n);
      if (sq != CPQR_OK) return sq;
    }
    if (ctx->resid_pending) {  // the previous sweep's residual, beside the rest of this sweep
      CK(cudaEventRecord(ctx->ev_prep, st));
      cpqr_status sr = launch_lagged_residual(ctx);
      if (sr != CPQR_OK) return sr;
    }
    std::swap(ctx->Q0, ctx->Q0prev[n]);
    std::swap(ctx->Q0f, ctx->Q0fprev[n]);
    ctx->has_prev[n] = true;
    ctx->last_updated = n;
    return CPQR_OK;
  }
  // Lines 8-10: eq. 19 and the R0^{-T} solve over all SMs, then normalisation and the factor QR.
  FinishOut fo{ctx->A[n], ctx->lambda, ctx->Q[n], ctx->Rf[n], ctx->Qf[n], ctx->fit_terms};
  if (!fp64) {  // the finish kernel also stages Q_n^T for the tensor cores
    fo.Qt = ctx->Qt[n];
    fo.Rp = ctx->Rp;
    fo.Kp = ctx->Kp[n];
  }
  {
    // finish prep, then the factor QR: by the guarded Gram route, 4 kernels and the Householder
    // finish, which runs only when the guard trips; else the Householder finish alone
    Timed tm(ctx, CPQR_BUCKET_QR, ctx->gram ? 6 : 2);
    const double b = ext ? beta : 0.0;
    double* hpart = ctx->gram ? ctx->hpart : nullptr;
    if (fp64)
      CK(launch_finish_prep<double>(ctx->v_work, nparts, I, C, R, ctx->R0, b, ctx->alpha, ctx->V, ctx->fitpart,
                                    hpart, ctx->dstatus, st));
    else
      CK(launch_finish_prep<float>((const float*)ctx->v_work, nparts, I, C, R, ctx->R0, b, ctx->alpha, ctx->V,
                                   ctx->fitpart, hpart, ctx->dstatus, st));
    if (ctx->gram) {
      const int nblk = finish_prep_blocks(I);
      CK(launch_finish_gram_chol(ctx->hpart, ctx->fitpart, nblk, I, R, fo, ctx->fg_work, ctx->Gf[n], ctx->cn[n], st));
      if (next_mode >= 0 && next_mode != n && !ctx->z_pending) {
        // the next mode's Khatri-Rao Cholesky needs only the factors' Grams: it runs on the
        // side stream beside the rest of this factor QR (on the split route, the Cholesky of its
        // last level, which also takes W's guard)
        const bool split = ctx->gram && ctx->w_ok && ctx->wpf_mode == next_mode && ctx->wpf_excl == n;
        CK(cudaEventRecord(ctx->ev_gram, st));
        CK(cudaStreamWaitEvent(ctx->st2, ctx->ev_gram, 0));
        Timed tz(ctx, CPQR_BUCKET_Q0, 1, ctx->st2);
        if (split)
          CK(launch_krp_chol(z_grams(ctx, next_mode), N - 1, R, ctx->zg_work, ctx->st2, 0, gram_flag(ctx->wg_work)));
        else
          CK(launch_krp_chol(z_grams_level2(ctx, next_mode), 2, R, ctx->zg_work, ctx->st2));
        ctx->zchol_mode = next_mode;
        ctx->zchol_split = split;
      }
      CK(launch_finish_gram_rows(ctx->V, ctx->fitpart, nblk, I, R, fo, ctx->fg_work, ctx->qr_work, ctx->dstatus, st));
    } else
      CK(launch_mode_finish(ctx->V, ctx->fitpart, finish_prep_blocks(I), I, R, fo, ctx->qr_work, ctx->dstatus, st));
  }
  if (ctx->resid_pending) {
    // the previous sweep's residual runs after this factor QR, beside the next mode's TTM chain
    // and Khatri-Rao QR: launched beside the factor QR, it raced the factor Cholesky's cluster for
    // a free GPC and sometimes held it back for the whole residual
    CK(cudaEventRecord(ctx->ev_prep, st));
    cpqr_status s = launch_lagged_residual(ctx);
    if (s != CPQR_OK) return s;
  }
  std::swap(ctx->Q0, ctx->Q0prev[n]);
  std::swap(ctx->Q0f, ctx->Q0fprev[n]);
  ctx->has_prev[n] = true;
  ctx->last_updated = n;
  return CPQR_OK;
}

double fit_from_r2(const cpqr_ctx* ctx, double r2) {
  return 1.0 - std::sqrt(std::max(r2, 0.0)) / std::sqrt(ctx->normX2);
}

// Whether the fit of the current sweep may be read one sweep late: split path with the tensor-
// core residual or on the wide path, and a beta for the following sweeps that no longer depends on
// the fit.
bool can_lag(const cpqr_ctx* ctx) {
  if (!ctx->lag_ok || ctx->prec != CPQR_PREC_SPLIT_BF16 || ctx->x64) return false;
  // the tensor-core residual (R <= 32), which leaves a GPC free for the chain's cluster kernels, or
  // the wide path's CUDA-core residual, beside QRs that launch no clusters (its FP32 work shares
  // the SMs with their FP64 work)
  if (!ctx->wide && !residual_tc_supported(ctx->N, ctx->dims.data(), ctx->R, ctx->X)) return false;
  // the rule's beta depends on the fit until it has activated (the learned proposer's fallback)
  if ((ctx->extrap == CPQR_EXTRAP_PAPER || ctx->extrap == CPQR_EXTRAP_LEARNED) && !ctx->activated) return false;
  return true;
}

// The residual of the snapshot in res_work on st3, after ev_prep (recorded on st after the
// snapshot), leaving one GPC free for the cluster kernels of the chain; its value goes to
// h_pinned[4].
cpqr_status launch_lagged_residual(cpqr_ctx* ctx) {
  NvtxRange nvtx_range("cpqr:residual");
  CK(cudaStreamWaitEvent(ctx->st3, ctx->ev_prep, 0));
  {
    Timed tm(ctx, CPQR_BUCKET_FIT, 1, ctx->st3);
    const double* A[CPQR_MAXN];
    for (int n = 0; n < ctx->N; ++n) A[n] = ctx->A[n];
    CK(launch_residual2<float>((const float*)ctx->X, ctx->N, ctx->dims.data(), A, ctx->lambda, ctx->R,
                               ctx->d_scalar + 1, ctx->res_work, ctx->dstatus, ctx->st3, RESIDUAL_EVALUATE,
                               qr_cluster_sms()));
  }
  if (ctx->mlp_state) {
    // the learned proposer's next proposal from this fit, beside the sweep that follows it
    Timed tm(ctx, CPQR_BUCKET_OTHER, 1, ctx->st3);
    MlpFitSource src{ctx->d_scalar + 1, ctx->fit_terms, ctx->normX2};
    CK(mlp_propose(ctx->mlp_wt, ctx->mlp_params, ctx->mlp_state, src, ctx->pending_beta, ctx->st3));
    CK(cudaMemcpyAsync(ctx->h_pinned + 5, &ctx->mlp_state->cls, sizeof(int32_t), cudaMemcpyDeviceToHost,
                       ctx->st3));
  }
  CK(cudaMemcpyAsync(ctx->h_pinned + 4, ctx->d_scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, ctx->st3));
  CK(cudaEventRecord(ctx->ev_fit, ctx->st3));
  ctx->resid_pending = false;
  ctx->resid_inflight = true;
  ctx->inflight_beta = ctx->pending_beta;
  ctx->inflight_check = ctx->pending_check;
  return CPQR_OK;
}

void observe_fit(cpqr_ctx* ctx, double fit);

// Reads the lagged fit once its residual has finished and records it.
cpqr_status collect_lagged_fit(cpqr_ctx* ctx) {
  if (!ctx->resid_inflight) return CPQR_OK;
  CK(cudaEventSynchronize(ctx->ev_fit));
  ctx->resid_inflight = false;
  const double f = fit_from_r2(ctx, ctx->h_pinned[4]);
  if (!std::isfinite(f)) return fail(ctx, CPQR_ENONFINITE);
  const double prev = ctx->fits.empty() ? NAN : ctx->fits.back();
  observe_fit(ctx, f);
  if (ctx->mlp_state) {
    int32_t c;
    std::memcpy(&c, ctx->h_pinned + 5, sizeof(c));
    ctx->next_class = (c >= 0 && c < CPQR_MLP_CLASSES) ? c : -1;
  }
  // a sweep run inside an approval window: a drop beyond the fit's rounding ends the approval
  if (ctx->inflight_check && !(f >= prev - 1e-7)) {
    ctx->approved_class = -1;
    ctx->approve_window = 1;
    ctx->approve_left = 0;
  }
  ctx->inflight_check = false;
  return CPQR_OK;
}

// Completes every lagged fit, checks the device status and collects the timing events.
cpqr_status flush_lag(cpqr_ctx* ctx) {
  if (!ctx->resid_pending && !ctx->resid_inflight) return CPQR_OK;
  if (ctx->resid_pending) {
    CK(cudaEventRecord(ctx->ev_prep, ctx->st));
    cpqr_status s = launch_lagged_residual(ctx);
    if (s != CPQR_OK) return s;
  }
  cpqr_status s = collect_lagged_fit(ctx);
  if (s != CPQR_OK) return s;
  CK(cudaMemcpyAsync(ctx->h_pinned + 2, ctx->dstatus, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaStreamSynchronize(ctx->st2));
  if (ctx->timing) collect_timing(ctx);
  unsigned int ds;
  std::memcpy(&ds, ctx->h_pinned + 2, sizeof(ds));
  if (ds & CPQR_DEV_TIMEOUT) return fail(ctx, CPQR_ETIMEOUT);
  if (ds & CPQR_DEV_SINGULAR) return fail(ctx, CPQR_ESINGULAR);
  return CPQR_OK;
}

// Fit after a sweep.  FP64 path: Section 4.1's reduced form from the last mode's V0, V^.
// Split path: the reduced form cancels ||X||^2 against terms that carry the split operands'
// ~2^-16 relative error, which can exceed a 1e-6 change in fit, so the fit comes from an
// explicit residual pass over X with the current factors instead (one read of X).
cpqr_status read_fit(cpqr_ctx* ctx, double* fit, double beta) {
  const bool explicit_fit = (ctx->prec == CPQR_PREC_SPLIT_BF16);
  if (explicit_fit) {
    Timed tm(ctx, CPQR_BUCKET_FIT, 1);
    const double* A[CPQR_MAXN];
    for (int n = 0; n < ctx->N; ++n) A[n] = ctx->A[n];
    CK(launch_residual2<float>((const float*)ctx->X, ctx->N, ctx->dims.data(), A, ctx->lambda, ctx->R,
                               ctx->d_scalar, ctx->res_work, ctx->dstatus, ctx->st));
  }
  const bool propose = ctx->mlp_state != nullptr;
  if (propose) {
    // the learned proposer's next proposal, from this sweep's fit, on the device
    Timed tm(ctx, CPQR_BUCKET_OTHER, 1);
    MlpFitSource src{explicit_fit ? ctx->d_scalar : nullptr, ctx->fit_terms, ctx->normX2};
    CK(mlp_propose(ctx->mlp_wt, ctx->mlp_params, ctx->mlp_state, src, beta, ctx->st));
  }
  {
    Timed tm(ctx, CPQR_BUCKET_OTHER, 0);
    if (explicit_fit)
      CK(cudaMemcpyAsync(ctx->h_pinned + 3, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(ctx->h_pinned, ctx->fit_terms, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(ctx->h_pinned + 2, ctx->dstatus, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->st));
    if (propose)
      CK(cudaMemcpyAsync(ctx->h_pinned + 5, &ctx->mlp_state->cls, sizeof(int32_t), cudaMemcpyDeviceToHost,
                         ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  if (propose) {
    int32_t c;
    std::memcpy(&c, ctx->h_pinned + 5, sizeof(c));
    ctx->next_class = (c >= 0 && c < CPQR_MLP_CLASSES) ? c : -1;
  }
  if (ctx->timing) {
    CK(cudaStreamSynchronize(ctx->st2));  // the next sweep's W may still be running there
    collect_timing(ctx);
  }
  unsigned int ds;
  std::memcpy(&ds, ctx->h_pinned + 2, sizeof(ds));
  if (ds & CPQR_DEV_TIMEOUT) return fail(ctx, CPQR_ETIMEOUT);
  if (ds & CPQR_DEV_SINGULAR) return fail(ctx, CPQR_ESINGULAR);
  double in = ctx->h_pinned[0], nn = ctx->h_pinned[1];
  double r2 = explicit_fit ? ctx->h_pinned[3] : ctx->normX2 - 2.0 * in + nn;
  double f = fit_from_r2(ctx, r2);
  if (!std::isfinite(f)) return fail(ctx, CPQR_ENONFINITE);
  *fit = f;
  return CPQR_OK;
}

double beta_for_sweep(cpqr_ctx* ctx) {
  switch (ctx->extrap) {
    case CPQR_EXTRAP_NONE: return 0.0;
    case CPQR_EXTRAP_FIXED: return ctx->sweeps >= 1 ? ctx->beta_fixed : 0.0;
    case CPQR_EXTRAP_LEARNED:
    default: return ctx->beta_active;
  }
}

void observe_fit(cpqr_ctx* ctx, double fit) {
  ctx->fits.push_back(fit);
  size_t k = ctx->fits.size();
  if (!ctx->activated && k >= 2 && std::fabs(ctx->fits[k - 1] - ctx->fits[k - 2]) < kActivateDfit) {
    ctx->beta_active = beta_band(fit);
    ctx->activated = true;
  }
}

// allow_lag: a forced beta that may still have its fit read one sweep late (the learned
// proposer's unjudged sweeps)
cpqr_status one_sweep(cpqr_ctx* ctx, double* fit_out, const double* forced_beta = nullptr, bool allow_lag = false) {
  NvtxRange nvtx_range("cpqr:sweep");
  const double beta = forced_beta ? *forced_beta : beta_for_sweep(ctx);
  const bool lag = (!forced_beta || allow_lag) && can_lag(ctx);
  if (!lag) {
    cpqr_status s = flush_lag(ctx);
    if (s != CPQR_OK) return s;
  }
  ctx->ops.clear();
  try {
    ctx->sched->next_sweep(ctx->ops);
  } catch (const std::exception&) {
    return fail(ctx, CPQR_EINVAL);
  }
  // The schedule is deterministic, so a copy tells the first update of the following sweep: the
  // last update of this one forms the W of that update.  Between sweeps only a rollback changes the
  // factors, and it drops that W (wpf_mode); a W is otherwise used only for the update and the
  // last-updated mode it was formed for.
  ctx->next_first = -1;
  try {
    Schedule peek(*ctx->sched);
    std::vector<Op> nxt;
    peek.next_sweep(nxt);
    for (const Op& q : nxt)
      if (q.kind == OP_UPDATE) {
        ctx->next_first = q.a;
        break;
      }
  } catch (const std::exception&) {
    ctx->next_first = -1;
  }
  // the update after ops[k]: the next one in this sweep, else the first of the next sweep
  auto update_after = [ctx](size_t k) {
    for (size_t q = k + 1; q < ctx->ops.size(); ++q)
      if (ctx->ops[q].kind == OP_UPDATE) return ctx->ops[q].a;
    return ctx->next_first;
  };
  for (size_t i = 0; i < ctx->ops.size(); ++i) {
    const Op& op = ctx->ops[i];
    cpqr_status s = CPQR_OK;
    if (op.kind == OP_TTM && !ctx->z_pending) {
      // first TTM of the next mode's chain: start its Khatri-Rao QR alongside
      for (size_t k = i + 1; k < ctx->ops.size(); ++k)
        if (ctx->ops[k].kind == OP_UPDATE) {
          s = launch_z(ctx, ctx->ops[k].a, update_after(k));
          break;
        }
      if (s != CPQR_OK) return s;
    }
    if (op.kind == OP_TTM) s = run_ttm(ctx, op);
    else if (op.kind == OP_UPDATE) {
      s = run_update(ctx, op.a, op.b, beta, update_after(i));
    }
    else free_node(ctx, op.a);
    if (s != CPQR_OK) return s;
  }
  if (lag) {
    // snapshot of this sweep's factors for its residual (launched during the next sweep); the
    // previous residual reads the same buffer, so the snapshot waits for it (and a residual still
    // pending, had no update launched it, goes first)
    if (ctx->resid_pending) {
      CK(cudaEventRecord(ctx->ev_prep, ctx->st));
      cpqr_status sp = launch_lagged_residual(ctx);
      if (sp != CPQR_OK) return sp;
    }
    if (ctx->resid_inflight) CK(cudaStreamWaitEvent(ctx->st, ctx->ev_fit, 0));
    {
      Timed tm(ctx, CPQR_BUCKET_OTHER, 1);
      const double* A[CPQR_MAXN];
      for (int n = 0; n < ctx->N; ++n) A[n] = ctx->A[n];
      CK(launch_residual2<float>((const float*)ctx->X, ctx->N, ctx->dims.data(), A, ctx->lambda, ctx->R,
                                 ctx->d_scalar + 1, ctx->res_work, ctx->dstatus, ctx->st, RESIDUAL_SNAPSHOT));
    }
    ctx->last_beta = beta;
    ++ctx->sweeps;
    ctx->betas.push_back(beta);
    cpqr_status s = collect_lagged_fit(ctx);  // the previous sweep's
    if (s != CPQR_OK) return s;
    ctx->resid_pending = true;
    ++ctx->lagged_fits;
    ctx->pending_beta = beta;
    ctx->pending_check = ctx->sweep_check;
    if (fit_out) *fit_out = NAN;
    return CPQR_OK;
  }
  double fit = 0.0;
  cpqr_status s = read_fit(ctx, &fit, beta);
  if (s != CPQR_OK) return s;
  ctx->last_beta = beta;
  ++ctx->sweeps;
  ctx->betas.push_back(beta);
  observe_fit(ctx, fit);
  if (fit_out) *fit_out = fit;
  return CPQR_OK;
}

// Section 4.2 rule's beta for the next sweep (what CPQR_EXTRAP_PAPER would use).
double rule_beta_next(const cpqr_ctx* ctx) { return ctx->beta_active; }

const double kMlpBetas[CPQR_MLP_CLASSES] = {0.0, 5e-5, 2e-4, 5e-4, 2e-3, 4e-3, 1e-2, 3e-2};

void mlp_features(const double* fits, const double* betas, int n, double rule_beta, int activated, float* f) {
  for (int i = 0; i < CPQR_MLP_FEATURES; ++i) f[i] = 0.f;
  for (int j = 0; j < 8; ++j) {
    const int k = n - 1 - j;  // sweep index (0-based) j sweeps back
    if (k < 0) break;
    const double fit = fits[k];
    f[3 * j] = (float)(std::log10(std::max(1.0 - fit, 1e-12)) / 12.0);
    if (k >= 1) {
      const double d = fits[k] - fits[k - 1];
      const double m = (std::log10(std::max(std::fabs(d), 1e-14)) + 14.0) / 14.0;
      f[3 * j + 1] = (float)(d >= 0 ? m : -m);
    }
    f[3 * j + 2] = (float)(std::log10(betas[k] + 1e-8) / 8.0);
  }
  f[24] = (float)(std::log10((double)n + 1.0) / 3.0);
  f[25] = (float)(std::log10(rule_beta + 1e-8) / 8.0);
  f[26] = activated ? 1.f : 0.f;
}

// CPQR_EXTRAP_LEARNED.  After every sweep the device proposes the next sweep's beta (features and
// network in one kernel, read back with the fit).  A proposal equal to the Section 4.2 rule's beta
// runs as is.  Any other proposal, beta = 0 included, is judged: from one checkpoint the proposal's
// sweep and the rule's sweep both run, and the proposal is kept only if its fit is higher, else the
// rule's sweep stands (the rule is the fallback).  A proposal that won stays approved for the next
// approve_window sweeps (2, 4, ... 128 after consecutive wins) as long as the fit does not drop by
// more than 1e-7; such a drop ends the approval.  After a loss the rule runs for hold_window sweeps
// (1, 2, ... 128 after consecutive losses) with the proposals deferred unjudged; then the next
// differing proposal is judged again.  A judge costs a flush of the lagged fit, three checkpoint
// copies and two sweeps with synchronous fits (~1.2 ms against a 0.33 ms sweep at 400^3), so the
// windows keep it to about one sweep in a hundred once either side keeps winning.
constexpr int kWindowCap = 128;
cpqr_status learned_sweep(cpqr_ctx* ctx, double* fit_out) {
  const double rule = rule_beta_next(ctx);
  const int cls = ctx->next_class;
  // Sweeps that are not judged may read their fit one sweep late (inside a multi-sweep call, once
  // the rule has activated): the proposal then comes from the fits up to the sweep before, and an
  // approved sweep's fit drop is checked when its fit arrives.
  if (!ctx->mlp_state || ctx->fits.size() < 2 || cls < 0) return one_sweep(ctx, fit_out, &rule, true);
  const double prop = kMlpBetas[cls];
  if (prop == rule) return one_sweep(ctx, fit_out, &rule, true);
  ++ctx->proposals;
  if (ctx->hold_left > 0) {  // a recent loss: the rule runs, the proposal is deferred unjudged
    --ctx->hold_left;
    ++ctx->deferred;
    return one_sweep(ctx, fit_out, &rule, true);
  }
  double f = 0.0;
  if (cls == ctx->approved_class && ctx->approve_left > 0) {
    --ctx->approve_left;
    const double prev = ctx->fits.back();
    ctx->sweep_check = true;
    cpqr_status s = one_sweep(ctx, &f, &prop, true);
    ctx->sweep_check = false;
    if (s != CPQR_OK) return s;
    ++ctx->accepted;
    ++ctx->preapproved;
    // a drop beyond the per-sweep fit's rounding (a sweep's explicit residual moves by ~1e-12 between
    // nearly equal models) ends the approval; a lagged fit (NaN here) is checked when it arrives
    if (!std::isnan(f) && !(f >= prev - 1e-7)) {
      ctx->approved_class = -1;
      ctx->approve_window = 1;
      ctx->approve_left = 0;
    }
    if (fit_out) *fit_out = f;
    return CPQR_OK;
  }
  ++ctx->judged;
  // both branches start from one checkpoint with every fit read
  cpqr_status s = flush_lag(ctx);
  if (s != CPQR_OK) return s;
  s = checkpoint_save(ctx, 1);
  if (s != CPQR_OK) return s;
  double fp = 0.0, fr = 0.0;
  s = one_sweep(ctx, &fp, &prop);
  if (s == CPQR_OK) s = checkpoint_save(ctx, 2);  // the proposal's branch
  if (s == CPQR_OK) s = checkpoint_restore(ctx, 1);
  if (s == CPQR_OK) s = one_sweep(ctx, &fr, &rule);
  if (s != CPQR_OK) return s;
  if (fp > fr) {
    s = checkpoint_restore(ctx, 2);
    if (s != CPQR_OK) return s;
    ++ctx->accepted;
    ctx->approved_class = cls;
    ctx->approve_window = std::min(2 * ctx->approve_window, kWindowCap);
    ctx->approve_left = ctx->approve_window;
    ctx->hold_window = 1;
    f = fp;
  } else {
    ctx->approved_class = -1;
    ctx->approve_window = 1;
    ctx->approve_left = 0;
    ctx->hold_left = ctx->hold_window;
    ctx->hold_window = std::min(2 * ctx->hold_window, kWindowCap);
    f = fr;
  }
  checkpoint_drop(ctx, 1);
  checkpoint_drop(ctx, 2);
  if (fit_out) *fit_out = f;
  return CPQR_OK;
}

cpqr_status next_sweep(cpqr_ctx* ctx, double* fit_out) {
  if (ctx->extrap == CPQR_EXTRAP_LEARNED) return learned_sweep(ctx, fit_out);
  return one_sweep(ctx, fit_out);
}

bool valid_enum(int v, int lo, int hi) { return v >= lo && v <= hi; }

}  // namespace

extern "C" {

void cp_als_qr_default_options(cpqr_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->tree = CPQR_TREE_RESTRUCTURED;
  opt->prec = CPQR_PREC_FP64;
  opt->extrap = CPQR_EXTRAP_PAPER;
  opt->qr_route = CPQR_QR_GRAM;
  opt->alpha = kAlphaDefault;
  opt->beta_fixed = 0.0;
  opt->seed = 0;
  opt->mlp_weights = nullptr;
}

const char* cp_als_qr_strerror(int32_t s) {
  switch (s) {
    case CPQR_OK: return "ok";
    case CPQR_EINVAL: return "invalid argument";
    case CPQR_ENOMEM: return "out of device memory";
    case CPQR_ECUDA: return "CUDA error";
    case CPQR_ESINGULAR: return "singular factor (zero column norm or zero R diagonal)";
    case CPQR_ENONFINITE: return "non-finite fit";
    case CPQR_ETIMEOUT: return "device wait timed out";
    case CPQR_ENOTCONV: return "max_sweeps reached before tol";
    case CPQR_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

cpqr_status cp_als_qr_init(cpqr_ctx** out, int32_t N, const int64_t* dims, int32_t R, const void* X_dev,
                           int32_t x_is_fp64, const double* const* A0_host, const cpqr_options* opt_in,
                           void* stream) {
  if (!out) return CPQR_EINVAL;
  *out = nullptr;
  if (N < 3 || N > CPQR_MAXN || !dims || R < 1 || R > CPQR_MAXR_WIDE || !X_dev) return CPQR_EINVAL;
  cpqr_options opt;
  if (opt_in) opt = *opt_in;
  else cp_als_qr_default_options(&opt);
  if (!valid_enum(opt.tree, 0, 2) || !valid_enum(opt.prec, 0, 1) || !valid_enum(opt.extrap, 0, 3) ||
      !valid_enum(opt.qr_route, 0, 1))
    return CPQR_EINVAL;
  int64_t nX = 1;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < R || dims[n] > (1 << 30)) return CPQR_EINVAL;
    nX *= dims[n];
    if (nX > (int64_t(1) << 40)) return CPQR_EINVAL;
  }
  if (opt.prec == CPQR_PREC_SPLIT_BF16 && x_is_fp64) return CPQR_EUNSUPPORTED;
  if (ipow(R, N - 1) > (int64_t(1) << 30)) return CPQR_EINVAL;

  std::unique_ptr<cpqr_ctx> c;
  try {
    c.reset(new cpqr_ctx());
  } catch (...) {
    return CPQR_ENOMEM;
  }
  cpqr_ctx* ctx = c.get();
  ctx->N = N;
  ctx->R = R;
  ctx->dims.assign(dims, dims + N);
  ctx->tree = opt.tree;
  ctx->prec = opt.prec;
  ctx->extrap = opt.extrap;
  ctx->gram = opt.qr_route == CPQR_QR_GRAM;
  ctx->wide = R > CPQR_MAXR;
  if (ctx->wide) ctx->gram = false;  // the wide path has its own (Cholesky) QRs
  ctx->alpha = opt.alpha > 0 ? opt.alpha : kAlphaDefault;
  ctx->beta_fixed = opt.beta_fixed;
  ctx->st = (cudaStream_t)stream;
  ctx->X = X_dev;
  ctx->x64 = x_is_fp64 != 0;
  ctx->nX = nX;
  cudaStream_t st = ctx->st;

  const int64_t M0 = ipow(R, N - 1);
  int64_t Imax = 0;
  for (int n = 0; n < N; ++n) Imax = std::max(Imax, dims[n]);
  CK(cache_malloc_host((void**)&ctx->h_pinned, 8 * sizeof(double)));
  // Per-mode state lives in one arena so that a checkpoint is a single copy.
  const bool split = opt.prec == CPQR_PREC_SPLIT_BF16;
  ctx->Rp = ((R + 15) / 16) * 16;
  {
    size_t off = 0;
    auto take = [&](size_t bytes) {
      size_t o = off;
      off += (bytes + 255) / 256 * 256;
      return o;
    };
    size_t oA[CPQR_MAXN], oQ[CPQR_MAXN], oR[CPQR_MAXN], oQf[CPQR_MAXN], oP[CPQR_MAXN], oT[CPQR_MAXN], oPf[CPQR_MAXN];
    size_t oG[CPQR_MAXN], oC[CPQR_MAXN];
    for (int n = 0; n < N; ++n) {
      ctx->Kp[n] = ((dims[n] + 63) / 64) * 64;
      oA[n] = take(dims[n] * R * 8);
      oQ[n] = take(dims[n] * R * 8);
      oR[n] = take((size_t)R * R * 8);
      oQf[n] = take(dims[n] * R * 4);
      oP[n] = take(M0 * R * 8);
      oT[n] = split ? take((size_t)2 * ctx->Rp * ctx->Kp[n] * 2) : 0;
      oPf[n] = split ? take(M0 * R * 4) : 0;
      oG[n] = take((size_t)CPQR_MAXR * CPQR_MAXR * sizeof(float2));
      oC[n] = take((size_t)CPQR_MAXR * 8);
    }
    size_t oQ0 = take(M0 * R * 8), oL = take(R * 8), oQ0f = split ? take(M0 * R * 4) : 0;
    const bool learned = opt.extrap == CPQR_EXTRAP_LEARNED && opt.mlp_weights;
    size_t oM = learned ? take(sizeof(MlpState)) : 0;
    ctx->arena_bytes = off;
    CK(cache_malloc(&ctx->arena, off));
    ctx->owned.emplace_back(ctx->arena, off);
    CK(cudaMemsetAsync(ctx->arena, 0, off, st));
    char* a = static_cast<char*>(ctx->arena);
    for (int n = 0; n < N; ++n) {
      ctx->A[n] = (double*)(a + oA[n]);
      ctx->Q[n] = (double*)(a + oQ[n]);
      ctx->Rf[n] = (double*)(a + oR[n]);
      ctx->Qf[n] = (float*)(a + oQf[n]);
      ctx->Q0prev[n] = (double*)(a + oP[n]);
      if (split) ctx->Qt[n] = (__nv_bfloat16*)(a + oT[n]);
      if (split) ctx->Q0fprev[n] = (float*)(a + oPf[n]);
      ctx->Gf[n] = (float2*)(a + oG[n]);
      ctx->cn[n] = (double*)(a + oC[n]);
    }
    ctx->Q0 = (double*)(a + oQ0);
    if (split) ctx->Q0f = (float*)(a + oQ0f);
    ctx->lambda = (double*)(a + oL);
    if (learned) ctx->mlp_state = (MlpState*)(a + oM);  // zeroed with the arena
  }
  CK(ctx->alloc(&ctx->R0, (size_t)R * R));
  CK(ctx->alloc(&ctx->V, Imax * 2 * R));
  CK(ctx->alloc(&ctx->fitpart, 2 * (size_t)finish_prep_blocks(Imax)));
  CK(ctx->alloc(&ctx->qr_work, std::max<int64_t>(M0, Imax) * R));
  CK(ctx->alloc(&ctx->zq_work, std::max<size_t>((size_t)(M0 * R), krp_nested_work_doubles(N - 1, R))));
  CK(ctx->alloc(&ctx->zg_work, krp_gram_work_doubles(R)));
  if (ctx->wide) {
    CK(ctx->alloc(&ctx->wq_main, wide_work_doubles(R)));
    CK(ctx->alloc(&ctx->wq_side, wide_work_doubles(R)));
    CK(ctx->alloc(&ctx->wrows, (size_t)Imax * (R + 2)));
  }
  CK(ctx->alloc(&ctx->fg_work, factor_gram_work_doubles(Imax, R)));
  CK(ctx->alloc(&ctx->hpart, (size_t)finish_prep_blocks(Imax) * 17 * 32));
  CK(cudaMemsetAsync(ctx->zg_work, 0, krp_gram_work_doubles(R) * sizeof(double), st));
  CK(cudaMemsetAsync(ctx->fg_work, 0, factor_gram_work_doubles(Imax, R) * sizeof(double), st));
  CK(ctx->alloc((char**)&ctx->res_work, residual2_work_bytes(N, dims, R)));
  {
    int64_t vw = 0;
    for (int n = 0; n < N; ++n) vw = std::max<int64_t>(vw, (int64_t)leaf_v_splits(dims[n], M0) * dims[n] * 2 * R);
    CK(ctx->alloc(&ctx->v_work, vw));
  }
  {
    // The Khatri-Rao QR needs one 16-CTA cluster (16 free SMs in one GPC) while a persistent TTM
    // grid is about to fill the GPU: its stream gets the highest priority so that the cluster is
    // placed first when both become ready together.
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&ctx->st2, cudaStreamNonBlocking, greatest));
    CK(cudaStreamCreateWithPriority(&ctx->st3, cudaStreamNonBlocking, least));
  }
  if (N - 1 >= 3) {
    // the split Khatri-Rao QR's W (a few hundred KB at most)
    size_t mwq = (size_t)R;
    for (int k = 0; k < N - 2; ++k) mwq *= (size_t)R;
    CK(ctx->alloc(&ctx->wg_work, krp_gram_work_doubles(R)));
    CK(cudaMemsetAsync(ctx->wg_work, 0, krp_gram_work_doubles(R) * sizeof(double), st));
    CK(ctx->alloc(&ctx->wq_work, std::max<size_t>(krp_nested_work_doubles(N - 2, R), 1)));
    CK(ctx->alloc(&ctx->WQ, mwq));
    CK(ctx->alloc(&ctx->WS, (size_t)R * R));
    ctx->w_ok = true;
  }
  CK(cudaEventCreateWithFlags(&ctx->ev_prep, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ctx->ev_fit, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ctx->ev_ready, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ctx->ev_z, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ctx->ev_gram, cudaEventDisableTiming));
  CK(ctx->alloc(&ctx->fit_terms, 2));
  CK(ctx->alloc(&ctx->d_scalar, 2));
  CK(ctx->alloc(&ctx->dstatus, 1));
  CK(cudaMemsetAsync(ctx->dstatus, 0, sizeof(unsigned int), st));
  CK(cudaMemsetAsync(ctx->fit_terms, 0, 2 * sizeof(double), st));
  CK(cudaMemsetAsync(ctx->lambda, 0, R * sizeof(double), st));

  // Khatri-Rao row plans: of the N-1 triangles (identical for every mode; only an order-3 tensor's
  // two-triangle product uses it directly, higher orders go through two-triangle levels) and of a
  // two-triangle product.
  {
    std::vector<int32_t> perm = krp_perm(N == 3 ? N - 1 : 1, R);
    CK(ctx->alloc(&ctx->d_perm, perm.size()));
    CK(cudaMemcpyAsync(ctx->d_perm, perm.data(), perm.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    ctx->zplan.m = N - 1;
    ctx->zplan.R = R;
    ctx->zplan.M = M0;
    ctx->zplan.perm = ctx->d_perm;
    for (int j = 0; j < CPQR_MAXR; ++j) ctx->zplan.act[j] = (int32_t)std::min<int64_t>(M0, ipow(j + 1, N - 1));
    std::vector<int32_t> perm2 = krp_perm(2, R);
    CK(ctx->alloc(&ctx->d_perm2, perm2.size()));
    CK(cudaMemcpyAsync(ctx->d_perm2, perm2.data(), perm2.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    ctx->zplan2.m = 2;
    ctx->zplan2.R = R;
    ctx->zplan2.M = (int64_t)R * R;
    ctx->zplan2.perm = ctx->d_perm2;
    for (int j = 0; j < CPQR_MAXR; ++j) ctx->zplan2.act[j] = (int32_t)std::min<int64_t>((int64_t)R * R, ipow(j + 1, 2));
    CK(cudaStreamSynchronize(st));  // the perm vectors go out of scope
  }

  // Starting factors (Alg. 2 "Initialize") and their QRs, issued back to back (one host copy of
  // each factor, alive until the synchronisation after the loop).
  std::vector<std::vector<double>> hosts(N);
  uint64_t seed = opt.seed;
  for (int n = 0; n < N; ++n) {
    std::vector<double>& host = hosts[n];
    host.resize(dims[n] * R);
    if (A0_host && A0_host[n]) {
      std::memcpy(host.data(), A0_host[n], host.size() * sizeof(double));
      for (double v : host)
        if (!std::isfinite(v)) return CPQR_ENONFINITE;
    } else {
      for (size_t i = 0; i < host.size(); ++i) {  // Box-Muller on SplitMix64
        double u1 = ((splitmix64(seed) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        double u2 = ((splitmix64(seed) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        host[i] = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
      }
    }
  }
  // The narrow path's QRs are independent 16-CTA cluster kernels: the modes go round-robin over
  // the three streams, each stream with Householder scratch of its own.
  cudaStream_t qs[3] = {st, ctx->st2, ctx->st3};
  double* qw[3] = {ctx->qr_work, nullptr, nullptr};
  if (!ctx->wide) {
    for (int k = 1; k < 3 && k < N; ++k) CK(ctx->alloc(&qw[k], (size_t)std::max<int64_t>(M0, Imax) * R));
    // after everything already queued on st (the arena's and the status word's clearing)
    CK(cudaEventRecord(ctx->ev_ready, st));
    CK(cudaStreamWaitEvent(ctx->st2, ctx->ev_ready, 0));
    CK(cudaStreamWaitEvent(ctx->st3, ctx->ev_ready, 0));
  }
  for (int n = 0; n < N; ++n) {
    const std::vector<double>& host = hosts[n];
    if (ctx->wide) {
      CK(cudaMemcpyAsync(ctx->A[n], host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      CK(launch_wide_qr(ctx->A[n], dims[n], R, nullptr, 0, ctx->Q[n], ctx->Qf[n], ctx->Rf[n], ctx->wq_main,
                        ctx->dstatus, st));
    } else {
      cudaStream_t s = qs[n % 3];
      CK(cudaMemcpyAsync(ctx->A[n], host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(launch_house_qr(ctx->A[n], dims[n], R, ctx->Q[n], ctx->Rf[n], qw[n % 3], ctx->dstatus, s));
      CK(launch_to_f32(ctx->Q[n], ctx->Qf[n], dims[n] * R, s));
      CK(launch_tri_gram(ctx->Rf[n], R, ctx->Gf[n], ctx->cn[n], s));
    }
  }
  CK(cudaStreamSynchronize(ctx->st2));
  CK(cudaStreamSynchronize(ctx->st3));
  CK(cudaStreamSynchronize(st));
  // Split-precision staging.
  if (ctx->prec == CPQR_PREC_SPLIT_BF16) {
    for (int n = 0; n < N; ++n) {
      cpqr_status s = stage_q(ctx, n);
      if (s != CPQR_OK) return s;
    }
    const int64_t last = dims[N - 1];
    if (last % 8 == 0) {
      CK(ctx->alloc(&ctx->Xhi, nX));
      CK(ctx->alloc(&ctx->Xlo, nX));
      CK(launch_split_x((const float*)X_dev, ctx->Xhi, ctx->Xlo, nX, st));
    } else {
      // TMA rows must be multiples of 16 bytes: pad the last dimension of the split copy so that
      // every TTM over X can take the tensor cores
      const int64_t ld = (last + 7) / 8 * 8, rows = nX / last;
      CK(ctx->alloc(&ctx->Xhi, rows * ld));
      CK(ctx->alloc(&ctx->Xlo, rows * ld));
      CK(launch_split_x_padded((const float*)X_dev, ctx->Xhi, ctx->Xlo, rows, last, ld, st));
      ctx->xlay.last = last;
      ctx->xlay.ld = ld;
    }
  }
  // ||X||^2 (precomputed once, Section 4.1).
  {
    double* nwork = nullptr;
    CK(ctx->alloc(&nwork, norm2_work_doubles()));
    if (ctx->x64) CK(launch_norm2<double>((const double*)X_dev, nX, ctx->d_scalar, nwork, st));
    else CK(launch_norm2<float>((const float*)X_dev, nX, ctx->d_scalar, nwork, st));
  }
  CK(cudaMemcpyAsync(ctx->h_pinned, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->h_pinned + 2, ctx->dstatus, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->normX2 = ctx->h_pinned[0];
  {
    unsigned int ds;
    std::memcpy(&ds, ctx->h_pinned + 2, sizeof(ds));
    if (ds & CPQR_DEV_SINGULAR) return CPQR_ESINGULAR;
  }
  if (!std::isfinite(ctx->normX2)) return CPQR_ENONFINITE;
  if (!(ctx->normX2 > 0.0)) return CPQR_EINVAL;

  if (ctx->extrap == CPQR_EXTRAP_LEARNED && opt.mlp_weights) {
    CK(ctx->alloc(&ctx->mlp_params, CPQR_MLP_NPARAMS));
    CK(cudaMemcpyAsync(ctx->mlp_params, opt.mlp_weights, CPQR_MLP_NPARAMS * sizeof(float), cudaMemcpyHostToDevice,
                       st));
    CK(ctx->alloc(&ctx->mlp_wt, CPQR_MLP_NPARAMS));
    CK(mlp_prepare_weights(ctx->mlp_params, ctx->mlp_wt, st));
    CK(cudaStreamSynchronize(st));
  }
  try {
    ctx->sched.reset(new Schedule(ctx->dims, R, ctx->tree));
  } catch (...) {
    return CPQR_ENOMEM;
  }
  ctx->nodes[0] = NodeBuf{const_cast<void*>(X_dev), 0, (1u << N) - 1u, true};
  *out = c.release();
  return CPQR_OK;
}

cpqr_status cp_als_qr_sweep(cpqr_ctx* ctx, int32_t nsweeps, double* fits_host) {
  if (!ctx) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  if (nsweeps < 0) return CPQR_EINVAL;
  // no decision between these sweeps needs a fit once beta is fixed: fits may come one sweep late
  ctx->lag_ok = true;
  cpqr_status s = CPQR_OK;
  for (int i = 0; i < nsweeps && s == CPQR_OK; ++i) s = next_sweep(ctx, nullptr);
  ctx->lag_ok = false;
  if (s != CPQR_OK) return s;
  s = flush_lag(ctx);
  if (s != CPQR_OK) return s;
  if ((int64_t)ctx->fits.size() < nsweeps) return fail(ctx, CPQR_EINVAL);  // every fit is read by now
  if (fits_host)
    for (int i = 0; i < nsweeps; ++i) fits_host[i] = ctx->fits[ctx->fits.size() - nsweeps + i];
  return CPQR_OK;
}

cpqr_status cp_als_qr_fit(cpqr_ctx* ctx, double tol, int32_t max_sweeps, double* final_fit, int32_t* sweeps_done) {
  if (!ctx) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  if (max_sweeps < 0) return CPQR_EINVAL;
  if (!(tol > 0.0)) {  // no stopping test: every sweep runs, fits may come one sweep late
    cpqr_status s = cp_als_qr_sweep(ctx, max_sweeps, nullptr);
    if (s != CPQR_OK) return s;
    if (final_fit) *final_fit = ctx->fits.empty() ? NAN : ctx->fits.back();
    if (sweeps_done) *sweeps_done = max_sweeps;
    return max_sweeps == 0 ? CPQR_OK : CPQR_ENOTCONV;
  }
  {
    cpqr_status s = flush_lag(ctx);
    if (s != CPQR_OK) return s;
  }
  double prev = NAN, f = NAN;
  int done = 0;
  bool conv = false;
  for (int i = 0; i < max_sweeps; ++i) {
    cpqr_status s = next_sweep(ctx, &f);
    if (s != CPQR_OK) return s;
    ++done;
    if (i >= 1 && std::fabs(f - prev) < tol) {
      conv = true;
      break;
    }
    prev = f;
  }
  if (final_fit) *final_fit = f;
  if (sweeps_done) *sweeps_done = done;
  return (conv || max_sweeps == 0) ? CPQR_OK : CPQR_ENOTCONV;
}

cpqr_status cp_als_qr_get(cpqr_ctx* ctx, int32_t n, double* A_host, double* lambda_host, double* Q_host,
                          double* R_host) {
  if (!ctx) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  if (n < 0 || n >= ctx->N) return CPQR_EINVAL;
  const size_t I = ctx->dims[n], R = ctx->R;
  cudaStream_t st = ctx->st;
  if (A_host) CK(cudaMemcpyAsync(A_host, ctx->A[n], I * R * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (lambda_host) CK(cudaMemcpyAsync(lambda_host, ctx->lambda, R * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (Q_host) CK(cudaMemcpyAsync(Q_host, ctx->Q[n], I * R * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (R_host) CK(cudaMemcpyAsync(R_host, ctx->Rf[n], R * R * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return CPQR_OK;
}

cpqr_status cp_als_qr_stats(cpqr_ctx* ctx, cpqr_stats* out) {
  if (!ctx || !out) return CPQR_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->sweeps = ctx->sweeps;
  out->ttm_flops = ctx->sched ? ctx->sched->flops() : 0;
  out->full_ttms = ctx->sched ? ctx->sched->full_ttms() : 0;
  out->last_fit = ctx->fits.empty() ? 0.0 : ctx->fits.back();
  out->beta = ctx->last_beta;
  out->proposals = ctx->proposals;
  out->accepted = ctx->accepted;
  out->judged = ctx->judged;
  out->preapproved = ctx->preapproved;
  out->deferred = ctx->deferred;
  out->launches = ctx->launches;
  out->krp_split = ctx->n_split;
  out->lagged_fits = ctx->lagged_fits;
  for (int b = 0; b < CPQR_NBUCKETS; ++b) {
    out->ms_bucket[b] = ctx->ms_bucket[b];
    out->n_bucket[b] = ctx->n_bucket[b];
  }
  if (ctx->zg_work && ctx->fg_work) {
    int cnt[4] = {0, 0, 0, 0};
    if (cudaStreamSynchronize(ctx->st) != cudaSuccess || cudaStreamSynchronize(ctx->st2) != cudaSuccess ||
        cudaMemcpy(&cnt[0], gram_fallback_counter(ctx->zg_work), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&cnt[1], gram_fallback_counter(ctx->fg_work), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&cnt[2], gram_second_pass_counter(ctx->zg_work), sizeof(int), cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(&cnt[3], gram_second_pass_counter(ctx->fg_work), sizeof(int), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
      return fail(ctx, CPQR_ECUDA);
    out->qr_fallbacks = (int64_t)cnt[0] + cnt[1];
    out->qr_second_pass = (int64_t)cnt[2] + cnt[3];
  }
  return ctx->err;
}

cpqr_status cp_als_qr_set_timing(cpqr_ctx* ctx, int32_t on) {
  if (!ctx) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  CK(cudaStreamSynchronize(ctx->st));
  ctx->evused.clear();
  ctx->evnext = 0;
  ctx->timing = on != 0;
  for (int b = 0; b < CPQR_NBUCKETS; ++b) {
    ctx->ms_bucket[b] = 0.0;
    ctx->n_bucket[b] = 0;
  }
  return CPQR_OK;
}

cpqr_status cp_als_qr_fit_exact(cpqr_ctx* ctx, double* fit) {
  if (!ctx || !fit) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  const double* A[CPQR_MAXN];
  for (int n = 0; n < ctx->N; ++n) A[n] = ctx->A[n];
  if (ctx->x64)
    CK(launch_residual2<double>((const double*)ctx->X, ctx->N, ctx->dims.data(), A, ctx->lambda, ctx->R,
                                ctx->d_scalar, ctx->res_work, ctx->dstatus, ctx->st));
  else
    CK(launch_residual2<float>((const float*)ctx->X, ctx->N, ctx->dims.data(), A, ctx->lambda, ctx->R,
                               ctx->d_scalar, ctx->res_work, ctx->dstatus, ctx->st));
  CK(cudaMemcpyAsync(ctx->h_pinned, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(ctx->h_pinned + 2, ctx->dstatus, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  unsigned int ds;
  std::memcpy(&ds, ctx->h_pinned + 2, sizeof(ds));
  if (ds & CPQR_DEV_TIMEOUT) return fail(ctx, CPQR_ETIMEOUT);
  *fit = 1.0 - std::sqrt(std::max(ctx->h_pinned[0], 0.0)) / std::sqrt(ctx->normX2);
  return CPQR_OK;
}

void cp_als_qr_destroy(cpqr_ctx* ctx) { delete ctx; }

cpqr_status cp_als_qr_checkpoint(cpqr_ctx* ctx) {
  if (!ctx) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  return checkpoint_save(ctx, 0);
}

cpqr_status cp_als_qr_rollback(cpqr_ctx* ctx) {
  if (!ctx) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  return checkpoint_restore(ctx, 0);
}

cpqr_status cp_als_qr_commit(cpqr_ctx* ctx) {
  if (!ctx) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  checkpoint_drop(ctx, 0);
  return CPQR_OK;
}

cpqr_status cp_als_qr_test_wait_timeout(cpqr_ctx* ctx, uint64_t limit_ns) {
  if (!ctx || limit_ns == 0) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  if (ctx->prec != CPQR_PREC_SPLIT_BF16) return CPQR_EUNSUPPORTED;
  ctx->test_skip_next_ttm = true;
  ctx->test_wait_ns = limit_ns;
  return CPQR_OK;
}

cpqr_status cp_als_qr_sweep_beta(cpqr_ctx* ctx, double beta, double* fit_host) {
  if (!ctx || !(beta >= 0.0) || !std::isfinite(beta)) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  return one_sweep(ctx, fit_host, &beta);
}

cpqr_status cp_als_qr_history(cpqr_ctx* ctx, double* fits_host, double* betas_host, int32_t cap, int32_t* n,
                              double* rule_beta, int32_t* activated) {
  if (!ctx) return CPQR_EINVAL;
  const int m = (int)ctx->fits.size();
  for (int i = 0; i < m && i < cap; ++i) {
    if (fits_host) fits_host[i] = ctx->fits[i];
    if (betas_host) betas_host[i] = ctx->betas[i];
  }
  if (n) *n = m;
  if (rule_beta) *rule_beta = rule_beta_next(ctx);
  if (activated) *activated = ctx->activated ? 1 : 0;
  return ctx->err;
}

cpqr_status cp_als_qr_mlp_state(cpqr_ctx* ctx, float* features_host, float* logits_host, int32_t* cls) {
  if (!ctx) return CPQR_EINVAL;
  if (ctx->err != CPQR_OK) return ctx->err;
  if (!ctx->mlp_state) return CPQR_EUNSUPPORTED;
  MlpState h;
  CK(cudaMemcpyAsync(&h, ctx->mlp_state, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (features_host) std::memcpy(features_host, h.feat, sizeof(h.feat));
  if (logits_host) std::memcpy(logits_host, h.logits, sizeof(h.logits));
  if (cls) *cls = h.cls;
  return CPQR_OK;
}

double cp_als_qr_mlp_beta(int32_t c) {
  if (c < 0 || c >= CPQR_MLP_CLASSES) return NAN;
  return kMlpBetas[c];
}

cpqr_status cpqr_mlp_features(const double* fits, const double* betas, int32_t n, double rule_beta,
                              int32_t activated, float* out_host) {
  if (!out_host || n < 0 || (n > 0 && (!fits || !betas))) return CPQR_EINVAL;
  mlp_features(fits, betas, n, rule_beta, activated, out_host);
  return CPQR_OK;
}

int64_t cpqr_mlp_work_bytes(int32_t B) { return B < 1 ? 0 : (int64_t)mlp_work_bytes(B); }

cpqr_status cpqr_mlp_forward(const float* params_dev, const float* X_dev, int32_t B, float* logits_dev,
                             void* work_dev, void* stream) {
  if (!params_dev || !X_dev || !logits_dev || !work_dev || B < 1 || B > 65535) return CPQR_EINVAL;
  return mlp_forward(params_dev, X_dev, B, logits_dev, work_dev, (cudaStream_t)stream) == cudaSuccess ? CPQR_OK
                                                                                                     : CPQR_ECUDA;
}

cpqr_status cpqr_mlp_grad(const float* params_dev, const float* X_dev, const int32_t* y_dev, int32_t B,
                          float* grad_dev, float* loss_dev, void* work_dev, void* stream) {
  if (!params_dev || !X_dev || !y_dev || !grad_dev || !loss_dev || !work_dev || B < 1 || B > 65535)
    return CPQR_EINVAL;
  return mlp_grad(params_dev, X_dev, y_dev, B, grad_dev, loss_dev, work_dev, (cudaStream_t)stream) == cudaSuccess
             ? CPQR_OK
             : CPQR_ECUDA;
}

cpqr_status cpqr_mlp_adam(float* params_dev, float* m_dev, float* v_dev, const float* grad_dev, float lr,
                          int32_t step, void* stream) {
  if (!params_dev || !m_dev || !v_dev || !grad_dev || step < 1 || !(lr > 0.f)) return CPQR_EINVAL;
  return mlp_adam(params_dev, m_dev, v_dev, grad_dev, lr, step, (cudaStream_t)stream) == cudaSuccess ? CPQR_OK
                                                                                                   : CPQR_ECUDA;
}

cpqr_status cp_als_qr_run_host(int32_t N, const int64_t* dims, int32_t R, const void* X_host, int32_t x_is_fp64,
                               const double* const* A0_host, const cpqr_options* opt, double tol,
                               int32_t max_sweeps, double* const* A_out_host, double* lambda_out_host,
                               double* final_fit, int32_t* sweeps_done, void* stream) {
  if (N < 3 || N > CPQR_MAXN || !dims || !X_host || !A_out_host) return CPQR_EINVAL;
  int64_t n = 1;
  for (int k = 0; k < N; ++k) {
    if (dims[k] < 1) return CPQR_EINVAL;
    n *= dims[k];
  }
  const size_t bytes = (size_t)n * (x_is_fp64 ? 8 : 4);
  cudaStream_t st = (cudaStream_t)stream;
  void* X = nullptr;
  if (cache_malloc(&X, bytes) != cudaSuccess) return CPQR_ENOMEM;
  cpqr_status s = CPQR_OK;
  if (cudaMemcpyAsync(X, X_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) s = CPQR_ECUDA;
  cpqr_ctx* ctx = nullptr;
  if (s == CPQR_OK) s = cp_als_qr_init(&ctx, N, dims, R, X, x_is_fp64, A0_host, opt, stream);
  if (s == CPQR_OK) {
    cpqr_status fs = cp_als_qr_fit(ctx, tol, max_sweeps, final_fit, sweeps_done);
    if (fs != CPQR_OK && fs != CPQR_ENOTCONV) s = fs;
    for (int k = 0; k < N && s == CPQR_OK; ++k)
      s = cp_als_qr_get(ctx, k, A_out_host[k], k == N - 1 ? lambda_out_host : nullptr, nullptr, nullptr);
    if (s == CPQR_OK) s = fs;
  }
  cp_als_qr_destroy(ctx);
  cudaStreamSynchronize(st);  // a failed set-up may leave the copy running
  cache_free(X, bytes);
  return s;
}

cpqr_status cp_als_qr_schedule(int32_t N, const int64_t* dims, int32_t R, int32_t tree, int32_t nsweeps,
                               int32_t* ops, int64_t cap, int64_t* count, int64_t* flops) {
  if (N < 3 || N > CPQR_MAXN || !dims || R < 1 || tree < 0 || tree > 2 || nsweeps < 0) return CPQR_EINVAL;
  try {
    std::vector<int64_t> d(dims, dims + N);
    Schedule s(d, R, tree);
    std::vector<Op> all;
    for (int i = 0; i < nsweeps; ++i) s.next_sweep(all);
    if (count) *count = (int64_t)all.size();
    if (flops) *flops = s.flops();
    if (ops) {
      int64_t n = std::min<int64_t>(cap, (int64_t)all.size());
      for (int64_t i = 0; i < n; ++i) {
        ops[4 * i] = all[i].kind;
        ops[4 * i + 1] = all[i].a;
        ops[4 * i + 2] = all[i].b;
        ops[4 * i + 3] = all[i].c;
      }
    }
  } catch (...) {
    return CPQR_EINVAL;
  }
  return CPQR_OK;
}

cpqr_status cpqr_ttm(const void* T_dev, int32_t nd, const int64_t* tdims, int32_t k, const void* Q_dev, int32_t R,
                     void* out_dev, int32_t dtype, void* stream) {
  if (!T_dev || !Q_dev || !out_dev || !tdims || nd < 1 || nd > 8 || k < 0 || k >= nd || R < 1 || R > CPQR_MAXR_WIDE)
    return CPQR_EINVAL;
  int64_t P = 1, S = 1;
  for (int j = 0; j < k; ++j) P *= tdims[j];
  for (int j = k + 1; j < nd; ++j) S *= tdims[j];
  const int64_t K = tdims[k];
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (dtype) {
    case 0: e = launch_ttm<double, double, double>((const double*)T_dev, (const double*)Q_dev, (double*)out_dev, P, K, S, R, st); break;
    case 1:
      e = launch_ttm_f32_tiled((const float*)T_dev, (const float*)Q_dev, (float*)out_dev, P, K, S, R, st);
      if (e == cudaErrorNotSupported)
        e = launch_ttm<float, float, float>((const float*)T_dev, (const float*)Q_dev, (float*)out_dev, P, K, S, R, st);
      break;
    case 2: e = launch_ttm<float, double, double>((const float*)T_dev, (const double*)Q_dev, (double*)out_dev, P, K, S, R, st); break;
    case 3: {
      const bool wide_tc = R > CPQR_MAXR;
      if (!(wide_tc ? ttm_tc_wide_supported(P, K, S, R) : ttm_tc_supported(P, K, S, R))) return CPQR_EUNSUPPORTED;
      const int Rp = ((R + 15) / 16) * 16;
      const int64_t Kp = ((K + 63) / 64) * 64;
      const int64_t n = P * K * S;
      __nv_bfloat16 *xh = nullptr, *xl = nullptr, *qt = nullptr;
      unsigned int* ds = nullptr;
      if (cudaMalloc(&xh, n * 2) != cudaSuccess || cudaMalloc(&xl, n * 2) != cudaSuccess ||
          cudaMalloc(&qt, (size_t)2 * Rp * Kp * 2) != cudaSuccess || cudaMalloc(&ds, 4) != cudaSuccess) {
        cudaFree(xh); cudaFree(xl); cudaFree(qt); cudaFree(ds);
        return CPQR_ENOMEM;
      }
      e = cudaMemsetAsync(ds, 0, 4, st);
      if (e == cudaSuccess) e = launch_split_x((const float*)T_dev, xh, xl, n, st);
      if (e == cudaSuccess) e = launch_split_q((const double*)Q_dev, K, R, qt, Rp, Kp, st);
      if (e == cudaSuccess)
        e = wide_tc ? launch_ttm_tc_wide(xh, xl, qt, Rp, Kp, (float*)out_dev, P, K, S, R, ds, st)
                    : launch_ttm_tc(xh, xl, qt, Rp, Kp, (float*)out_dev, P, K, S, R, ds, st);
      unsigned int hs = 0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, ds, 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      cudaFree(xh); cudaFree(xl); cudaFree(qt); cudaFree(ds);
      if (e == cudaSuccess && hs) return status_of_device_word(hs);
      break;
    }
    default: return CPQR_EINVAL;
  }
  return e == cudaSuccess ? CPQR_OK : CPQR_ECUDA;
}

// The wide-rank Cholesky QR behind cpqr_house_qr / cpqr_krp_qr for 32 < R <= CPQR_MAXR_WIDE.
static cpqr_status wide_entry_qr(const double* Y, int64_t M, int R, const double* const* tri, int m, double* Q,
                                 double* Rout, cudaStream_t st) {
  double* work = nullptr;
  unsigned int* ds = nullptr;
  if (cudaMalloc(&work, wide_work_doubles(R) * sizeof(double)) != cudaSuccess || cudaMalloc(&ds, 4) != cudaSuccess) {
    cudaFree(work); cudaFree(ds);
    return CPQR_ENOMEM;
  }
  unsigned int hs = 0;
  cudaError_t e = cudaMemsetAsync(ds, 0, 4, st);
  if (e == cudaSuccess) e = launch_wide_qr(Y, M, R, tri, m, Q, nullptr, Rout, work, ds, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, ds, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(work);
  cudaFree(ds);
  return e == cudaSuccess ? status_of_device_word(hs) : CPQR_ECUDA;
}

cpqr_status cpqr_house_qr(const double* A_dev, int64_t M, int32_t R, double* Q_dev, double* R_dev, void* stream) {
  if (!A_dev || !Q_dev || !R_dev || R < 1 || R > CPQR_MAXR_WIDE || M < R) return CPQR_EINVAL;
  if (R > CPQR_MAXR) return wide_entry_qr(A_dev, M, R, nullptr, 0, Q_dev, R_dev, (cudaStream_t)stream);
  cudaStream_t st = (cudaStream_t)stream;
  double* work = nullptr;
  unsigned int* ds = nullptr;
  if (cudaMalloc(&work, (size_t)M * R * sizeof(double)) != cudaSuccess || cudaMalloc(&ds, 4) != cudaSuccess) {
    cudaFree(work); cudaFree(ds);
    return CPQR_ENOMEM;
  }
  cudaError_t e = cudaMemsetAsync(ds, 0, 4, st);
  if (e == cudaSuccess) e = launch_house_qr(A_dev, M, R, Q_dev, R_dev, work, ds, st);
  unsigned int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, ds, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(work);
  cudaFree(ds);
  return e == cudaSuccess ? status_of_device_word(hs) : CPQR_ECUDA;
}

cpqr_status cpqr_krp_qr(const double* Rs_dev, int32_t m, int32_t R, double* Q0_dev, double* R0_dev, void* stream) {
  if (!Rs_dev || !Q0_dev || !R0_dev || m < 1 || m > CPQR_MAXN - 1 || R < 1 || R > CPQR_MAXR_WIDE) return CPQR_EINVAL;
  int64_t M = ipow(R, m);
  if (M < R || M > (int64_t(1) << 34)) return CPQR_EINVAL;
  if (R > CPQR_MAXR) {
    const double* tri[CPQR_MAXN];
    for (int k = 0; k < m; ++k) tri[k] = Rs_dev + (size_t)k * R * R;
    return wide_entry_qr(nullptr, M, R, tri, m, Q0_dev, R0_dev, (cudaStream_t)stream);
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int mp = (m >= 3) ? 2 : m;  // m >= 3 goes through the nested QR of two-triangle products
  std::vector<int32_t> perm = krp_perm(mp, R);
  const int64_t Mp = ipow(R, mp);
  const size_t wd = std::max<size_t>((size_t)(M * R), m >= 3 ? krp_nested_work_doubles(m, R) : 0);
  int32_t* dperm = nullptr;
  double* work = nullptr;
  unsigned int* ds = nullptr;
  if (cudaMalloc(&dperm, perm.size() * 4) != cudaSuccess || cudaMalloc(&work, wd * 8) != cudaSuccess ||
      cudaMalloc(&ds, 4) != cudaSuccess) {
    cudaFree(dperm); cudaFree(work); cudaFree(ds);
    return CPQR_ENOMEM;
  }
  ZPlan plan{};
  plan.m = mp;
  plan.R = R;
  plan.M = Mp;
  plan.perm = dperm;
  for (int j = 0; j < CPQR_MAXR; ++j) plan.act[j] = (int32_t)std::min<int64_t>(Mp, ipow(j + 1, mp));
  TriPtrs tri{};
  for (int k = 0; k < m; ++k) tri.p[k] = Rs_dev + (size_t)k * R * R;
  cudaError_t e = cudaMemcpyAsync(dperm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ds, 0, 4, st);
  double* gwork = nullptr;
  if (e == cudaSuccess && m >= 2 && cudaMalloc(&gwork, krp_gram_work_doubles(R) * 8) != cudaSuccess)
    e = cudaErrorMemoryAllocation;
  // the workspace's guard flag and fallback count start at zero
  if (e == cudaSuccess && gwork) e = cudaMemsetAsync(gwork, 0, krp_gram_work_doubles(R) * 8, st);
  if (e == cudaSuccess) {
    if (m >= 2) e = launch_krp_qr_gram(plan, tri, m, Q0_dev, R0_dev, gwork, work, ds, st);
    else e = launch_krp_qr(plan, tri, Q0_dev, R0_dev, work, ds, st);
  }
  unsigned int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, ds, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dperm); cudaFree(work); cudaFree(ds); cudaFree(gwork);
  return e == cudaSuccess ? status_of_device_word(hs) : CPQR_ECUDA;
}

}  // extern "C"
