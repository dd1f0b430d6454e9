/*
 * cpqr.h - C ABI of the GB300 (sm_103a) CP-ALS-QR library.
 *
 * Method: CP-ALS-QR (Alg. 2) with the restructured dimension tree (Section
 * 3.1) and the customised extrapolation on Q0 (eq. 19, Alg. 3), i.e. the
 * ALS-QR-BRE algorithm.  A dense N-way tensor X (C order: last index fastest)
 * is approximated by [[lambda; A^(1), ..., A^(N)]] of rank R.
 *
 * Conventions for every entry point below:
 *  - Matrices are row-major.  A factor A^(n) is I_n x R with element (i, r)
 *    at [i * R + r]; an R x R triangle likewise.
 *  - "device" pointers must come from cudaMalloc / a CUDA caching allocator on
 *    the current device; "host" pointers are ordinary host memory.
 *  - All GPU work is issued on the cudaStream_t given at init (passed as
 *    void*; NULL = legacy default stream).  Calls that return host results
 *    synchronise that stream before returning.
 *  - No entry point aborts or exits.  Errors are returned as cpqr_status and
 *    are sticky in a context: after the first failure every later call on the
 *    same context returns the same status.  cp_als_qr_strerror() names them.
 *  - The library owns all of its workspaces; the caller owns X and every
 *    buffer it passes.  X is borrowed read-only and must outlive the context.
 *  - Limits: 3 <= N <= 6, 1 <= R <= 192, R <= I_n for every n (compact QR of
 *    each factor), prod(I_n) < 2^40.  Ranks up to 32 run the warp-per-factor kernels;
 *    ranks 33..192 (the high-rank regime) run the wide-rank path: Cholesky QRs
 *    (float-float Cholesky of the Gram, FP64 substitution, a second pass when the first
 *    leaves |Q^T Q - I| > 1e-8, a first-order correction) and column-tiled kernels.
 */
#ifndef CPQR_H
#define CPQR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cpqr_ctx cpqr_ctx; /* opaque, owned by the library */

typedef enum {
  CPQR_OK = 0,
  CPQR_EINVAL = 1,      /* bad argument (sizes, pointers, enum values) */
  CPQR_ENOMEM = 2,      /* device allocation failed */
  CPQR_ECUDA = 3,       /* a CUDA call failed (launch, copy, device fault) */
  CPQR_ESINGULAR = 4,   /* a column norm lambda_r or a diagonal of R0 became 0 */
  CPQR_ENONFINITE = 5,  /* NaN or Inf in the fit */
  CPQR_ETIMEOUT = 6,    /* a bounded device wait gave up */
  CPQR_ENOTCONV = 7,    /* cp_als_qr_fit hit max_sweeps before tol */
  CPQR_EUNSUPPORTED = 8 /* valid request this build does not implement */
} cpqr_status;

/* TTM schedule of line 6 of Alg. 3 (Section 3.1; costs in Tables 1-6). */
typedef enum {
  CPQR_TREE_NONE = 0,        /* every mode update contracts X directly */
  CPQR_TREE_STANDARD = 1,    /* dimension tree, 2 full-tensor TTMs per sweep */
  CPQR_TREE_RESTRUCTURED = 2 /* restructured tree, 1 full TTM per sweep after the first */
} cpqr_tree;

/* Arithmetic of the TTM chains.  Z_n = Q0 R0, the R0^{-T} solve and the
 * factor QRs are FP64 in both modes.  Inside a sweep, the Khatri-Rao QR and each factor QR take
 * a guarded Gram route (Cholesky of the Gram matrix, one orthogonality correction); a pivot that
 * is not positive or a correction above 1e-8 hands that QR to the Householder QR, so the result is
 * the Householder-quality QR either way. */
typedef enum {
  CPQR_PREC_FP64 = 0,      /* every TTM in FP64 (X promoted exactly) */
  CPQR_PREC_SPLIT_BF16 = 1 /* TTMs at every tree level on tcgen05 tensor cores with the
                              operands split into bf16 hi + lo (all four products, FP32
                              accumulate; shapes outside the kernel's range on FP32 CUDA
                              cores); V = Y_(n) Q0 in FP32; fit from an explicit residual */
} cpqr_prec;

/* Extrapolation on Q0 (eq. 19). */
typedef enum {
  CPQR_EXTRAP_NONE = 0,   /* beta = 0: ALS-QR-BR */
  CPQR_EXTRAP_PAPER = 1,  /* Section 4.2 rule: alpha = 1/10, beta chosen by fit level once
                             |fit_k - fit_{k-1}| < 0.03, then fixed */
  CPQR_EXTRAP_FIXED = 2,  /* beta = beta_fixed from the second sweep on */
  CPQR_EXTRAP_LEARNED = 3 /* beta proposed by the learned model after every sweep (features and
                             network on the device).  A proposal other than the Section 4.2
                             rule's beta (beta = 0 included) is judged: from one checkpoint both
                             the proposal's and the rule's sweep run and the proposal is kept only
                             if its fit is higher; the rule is the fallback.  A winning proposal
                             stays approved for 2, 4, ... 128 further sweeps (doubling on
                             consecutive wins) while the fit does not drop by more than 1e-7;
                             after a losing one the
                             rule runs unjudged for 1, 2, ... 128 sweeps (doubling on consecutive
                             losses) */
} cpqr_extrap;

/* How a sweep computes the QR of a two-triangle Khatri-Rao product and the factor QRs. */
typedef enum {
  CPQR_QR_GRAM = 0,       /* guarded Gram route (default; see cpqr_prec) */
  CPQR_QR_HOUSEHOLDER = 1 /* Householder QR only */
} cpqr_qr_route;

typedef struct {
  int32_t tree;       /* cpqr_tree */
  int32_t prec;       /* cpqr_prec */
  int32_t extrap;     /* cpqr_extrap */
  int32_t qr_route;   /* cpqr_qr_route */
  double alpha;       /* eq. 19 alpha; <= 0 selects 1/10 */
  double beta_fixed;  /* beta for CPQR_EXTRAP_FIXED */
  uint64_t seed;      /* seed of the N(0,1) starting factors when A0 is NULL */
  const float* mlp_weights; /* host, CPQR_MLP_NPARAMS floats, for CPQR_EXTRAP_LEARNED (NULL =
                               the rule alone); copied at init */
} cpqr_options;

/* Time buckets of a sweep (the per-iteration breakdown of Section 4.3 plus the
 * split of TTM time by tree level). */
enum {
  CPQR_BUCKET_TTM_FULL = 0,  /* TTMs that read all of X */
  CPQR_BUCKET_TTM_DEEP = 1,  /* TTMs on cached intermediates */
  CPQR_BUCKET_Q0 = 2,        /* Khatri-Rao product and its QR (computation of Q0) */
  CPQR_BUCKET_APPLY_Q0 = 3,  /* V = Y_(n) [Q0 | Q0^{k-1}] (application of Q0) */
  CPQR_BUCKET_QR = 4,        /* extrapolation, R0^{-T} solve, normalisation, factor QR */
  CPQR_BUCKET_OTHER = 5,     /* operand staging, fit read-back, learned proposal */
  CPQR_BUCKET_FIT = 6,       /* explicit residual ||X - K||^2 of the split-precision path */
  CPQR_NBUCKETS = 7
};

/* Per-context counters. */
typedef struct {
  int64_t sweeps;          /* sweeps done */
  int64_t ttm_flops;       /* 2 * R * prod(source dims) summed over every TTM issued */
  int64_t full_ttms;       /* TTMs that read all of X */
  double last_fit;         /* fit after the last sweep */
  double beta;             /* beta used by the last sweep */
  int64_t proposals;       /* learned proposals that differed from the rule's beta */
  int64_t accepted;        /* ... of which ran (won the judge, or within an approval window) */
  int64_t launches;        /* kernels this context launched */
  double ms_bucket[CPQR_NBUCKETS];   /* device time per bucket (only while timing is on) */
  int64_t n_bucket[CPQR_NBUCKETS];   /* launches per bucket (only while timing is on) */
  int64_t qr_fallbacks;    /* Gram-route QRs (Khatri-Rao and factor) whose guard handed them to
                              the Householder QR; reading it synchronises the context's streams */
  int64_t krp_split;       /* Khatri-Rao QRs (order >= 4, Gram route) that took the split route:
                              the QR of the other triangles formed one update ahead, only the level
                              with the last-updated triangle after that update */
  int64_t judged;          /* learned proposals judged against the rule's sweep (two sweeps each) */
  int64_t preapproved;     /* learned proposals run within an approval window */
  int64_t deferred;        /* learned proposals set aside (the rule ran) within a hold after a loss */
  int64_t qr_second_pass;  /* Gram-route QRs (R <= 32) whose first Cholesky pass left 1e-8 < max |E| <=
                              1e-3 and that a second Cholesky pass finished (CholeskyQR2) instead
                              of the Householder QR; reading it synchronises the context's streams */
  int64_t lagged_fits;     /* sweeps whose fit was read one sweep late (split path, inside one
                              multi-sweep call, once beta no longer depends on that fit) */
} cpqr_stats;

/* Turn per-launch CUDA-event timing on (1) or off (0); resets the bucket times. */
cpqr_status cp_als_qr_set_timing(cpqr_ctx* ctx, int32_t on);

/* Fill *opt with the defaults: restructured tree, FP64, paper extrapolation, Gram QR route,
 * alpha = 0.1, beta_fixed = 0, seed = 0, no learned model. */
void cp_als_qr_default_options(cpqr_options* opt);

/* Create a context for X (device, C order, dims[0..N-1], float32 if x_is_fp64 = 0 else
 * float64) and rank R, and run Alg. 2's "Initialize": starting factors A0 (host array of
 * N host pointers to I_n x R FP64 row-major; NULL draws N(0,1) from opt->seed), their QRs
 * with positive diagonal, ||X||^2, and, for CPQR_PREC_SPLIT_BF16, the bf16 hi/lo split of X
 * (one pass over X).  opt NULL = defaults.  stream: cudaStream_t or NULL.
 * A non-finite entry in A0 or in X returns CPQR_ENONFINITE, a zero column of A0 (no QR)
 * CPQR_ESINGULAR, X = 0 CPQR_EINVAL.  On failure *out is NULL and nothing is leaked. */
cpqr_status cp_als_qr_init(cpqr_ctx** out, int32_t N, const int64_t* dims, int32_t R,
                           const void* X_dev, int32_t x_is_fp64, const double* const* A0_host,
                           const cpqr_options* opt, void* stream);

/* Run nsweeps sweeps (outer iterations of Alg. 3: every mode updated once, TTMs per the
 * schedule, customised extrapolation per the options).  fits_host (nsweeps doubles, may be
 * NULL) receives the fit after each sweep.  FP64 contexts compute it as in Section 4.1 from the
 * last mode of the sweep: 1 - sqrt(max(||X||^2 - 2<V0, V^> + ||V^||^2, 0)) / ||X||; split-
 * precision contexts from an explicit residual pass (see cp_als_qr_fit_exact), because the
 * reduced form's cancellation would expose the split operands' error. */
cpqr_status cp_als_qr_sweep(cpqr_ctx* ctx, int32_t nsweeps, double* fits_host);

/* Sweep until |fit_k - fit_{k-1}| < tol (the stopping test of Alg. 2/3, read as a change in
 * fit) or max_sweeps; returns CPQR_ENOTCONV (not sticky) if max_sweeps was reached first.
 * final_fit / sweeps_done may be NULL. */
cpqr_status cp_als_qr_fit(cpqr_ctx* ctx, double tol, int32_t max_sweeps, double* final_fit,
                          int32_t* sweeps_done);

/* Copy factor n (I_n x R, unit columns) and, if lambda_host != NULL, the weights (R) to the
 * host.  Q_host / R_host (may be NULL) receive Q_n (I_n x R) and R_n (R x R, upper, positive
 * diagonal) of the current factor. */
cpqr_status cp_als_qr_get(cpqr_ctx* ctx, int32_t n, double* A_host, double* lambda_host,
                          double* Q_host, double* R_host);

/* Counters since init. */
cpqr_status cp_als_qr_stats(cpqr_ctx* ctx, cpqr_stats* out);

/* Fit of the current model from an explicit pass over X: 1 - ||X - [[lambda; A]]|| / ||X||.  The
 * model entries are formed in FP32 from the FP64 factors and the squared residual is summed in
 * FP64, so the result does not suffer the cancellation of ||X||^2 - 2<X,K> + ||K||^2 (relative
 * error ~1e-7 in ||X - K||).  One read of X plus R FMAs per element; rows of X (product of all
 * but the last dimension) < 2^31. */
cpqr_status cp_als_qr_fit_exact(cpqr_ctx* ctx, double* fit);

/* End-to-end decomposition of a HOST tensor: copies X_host (C order, float32 or float64; pinned
 * memory gives an asynchronous copy) to the device, runs cp_als_qr_init and cp_als_qr_fit(tol,
 * max_sweeps), copies every factor to A_out_host[n] (I_n x R, host) and the weights to
 * lambda_out_host (R, host), and releases everything.  final_fit / sweeps_done may be NULL.
 * Returns CPQR_ENOTCONV if max_sweeps was reached before tol (results are still written). */
cpqr_status cp_als_qr_run_host(int32_t N, const int64_t* dims, int32_t R, const void* X_host,
                               int32_t x_is_fp64, const double* const* A0_host,
                               const cpqr_options* opt, double tol, int32_t max_sweeps,
                               double* const* A_out_host, double* lambda_out_host,
                               double* final_fit, int32_t* sweeps_done, void* stream);

/* Release every device allocation of ctx (NULL is ignored).  The blocks go to a process-wide
 * cache, keyed by device and size, from which the next context of the same shape takes them
 * without cudaMalloc; at most a quarter of a device's memory stays cached (see
 * cpqr_release_cached_memory). */
void cp_als_qr_destroy(cpqr_ctx* ctx);

/* Not from the paper: runtime memory management.  Frees every device and pinned host block that
 * destroyed contexts left in the library's cache (cp_als_qr_destroy, cp_als_qr_run_host).  Call
 * it when the memory is wanted elsewhere, and before cudaDeviceReset (blocks that a reset made
 * invalid are otherwise detected and dropped when next requested).  Thread-safe; no context may
 * be in use on another thread while it runs.  Returns CPQR_ECUDA if a free failed. */
cpqr_status cpqr_release_cached_memory(void);

/* Static string for a status code. */
const char* cp_als_qr_strerror(int32_t status);

/* The TTM schedule the library runs (Section 3.1), host only, no GPU needed.  Writes up to
 * cap operations of nsweeps sweeps as 4 int32 each into ops (may be NULL to count):
 *   {0, dst, src, k}  TTM: node dst = node src x_k Q_k^T (node 0 is X, modes 0-based)
 *   {1, n, leaf, 0}   mode-n update from node leaf
 *   {2, id, 0, 0}     node id released
 * *count = number of operations, *flops = sum of 2 * R * prod(source dims). */
cpqr_status cp_als_qr_schedule(int32_t N, const int64_t* dims, int32_t R, int32_t tree,
                               int32_t nsweeps, int32_t* ops, int64_t cap, int64_t* count,
                               int64_t* flops);

/* ---- Operation-level entry points (the steps of one mode update, on device buffers) ---- */

/* Mode-k product out = T x_k Q^T (Section 2.1) of a dense C-order tensor T with dims
 * tdims[0..nd-1] and Q (I_k x R, row-major, I_k = tdims[k]).  out has dims tdims with
 * tdims[k] replaced by R.  dtype: 0 = FP64 T, Q, out; 1 = FP32 T, Q, out (FFMA, FP32
 * accumulate); 2 = FP32 T, FP64 Q, FP64 out; 3 = split-bf16 tensor-core path: T FP32, Q FP64,
 * out FP32 (tcgen05; T and Q are split into bf16 hi + lo internally; needs K <= 512 and either
 * S a multiple of 8 or S == 1 with K a multiple of 8, S = prod of the dims after k, else
 * CPQR_EUNSUPPORTED).  stream: cudaStream_t. */
cpqr_status cpqr_ttm(const void* T_dev, int32_t nd, const int64_t* tdims, int32_t k,
                     const void* Q_dev, int32_t R, void* out_dev, int32_t dtype, void* stream);

/* Compact QR of an M x R FP64 matrix (row-major, device) by Householder reflections with
 * diag(R) > 0 (Alg. 2 line 10): Q_dev (M x R) and R_dev (R x R) receive the factors.  For
 * 32 < R <= 192 the wide-rank path's Cholesky QR gives the same factors (to rounding).  Returns
 * CPQR_ESINGULAR for a zero column (exactly zero Householder norm) and CPQR_ETIMEOUT if a bounded
 * wait of the cluster kernel gave up; Q and R then hold partial results.  Synchronises the
 * stream. */
cpqr_status cpqr_house_qr(const double* A_dev, int64_t M, int32_t R, double* Q_dev,
                          double* R_dev, void* stream);

/* Same QR as cpqr_house_qr without any device allocation.  The paper has no counterpart; it
 * is for callers that may not allocate device memory (a host application that owns all device
 * memory through its own pool, a latency-critical loop that cannot afford cudaMalloc/cudaFree
 * and the device synchronisation they can cause, a deployment with a fixed memory footprint).
 * Scratch lives in one statically allocated device array of CPQR_NOALLOC_QR_MAX_ELEMS + 32
 * doubles (8 MiB) that every GPU loading the library holds until the process exits.
 * - M * R must not exceed CPQR_NOALLOC_QR_MAX_ELEMS; larger problems return CPQR_EINVAL.
 * - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *   that device current; make that first call before any stream capture.  The address is kept
 *   per device together with the context it belongs to: after cudaDeviceReset the next call
 *   (in the new context) looks it up again, so make that call before any capture too.
 * - Returns CPQR_ETIMEOUT if a bounded wait of the cluster kernel gave up and CPQR_ESINGULAR if
 *   a column became zero (Q and R then hold partial results).
 * - All calls share the one array and it keeps the last call's contents: calls whose GPU work
 *   overlaps (other streams, other host threads) race and must be serialised by the caller.
 * Synchronises the stream before returning. */
#define CPQR_NOALLOC_QR_MAX_ELEMS (1 << 20)
cpqr_status cpqr_house_qr_noalloc(const double* A_dev, int64_t M, int32_t R, double* Q_dev,
                                  double* R_dev, void* stream);

/* QR of Z = R_1 (.) ... (.) R_m, the Khatri-Rao product of m upper-triangular R x R
 * matrices (Alg. 2 lines 3-4), rows (r_1, ..., r_m) with r_m fastest: Rs_dev holds the m
 * triangles back to back (device, FP64).  Q0_dev (R^m x R) and R0_dev (R x R) receive the
 * factors, diag(R0) > 0, by the guarded Gram route (see cpqr_prec) for m >= 2, whose fallback is
 * the Householder staircase QR (nested for m >= 3); for 32 < R <= 192 by the wide-rank Cholesky
 * QR (the Gram is the Hadamard product of the triangles' Grams).  CPQR_ESINGULAR / CPQR_ETIMEOUT as for
 * cpqr_house_qr.  Synchronises the stream. */
cpqr_status cpqr_krp_qr(const double* Rs_dev, int32_t m, int32_t R, double* Q0_dev,
                        double* R0_dev, void* stream);

/* ---- Learned extrapolation proposer (no counterpart in the paper; it proposes the beta of
 *      eq. 19 and is judged against the Section 4.2 rule) ----
 * A multilayer perceptron F -> 128 -> 128 -> 128 -> C (ReLU), weights and activations bf16,
 * FP32 accumulation, FP32 master parameters packed as [W_l (out x in row-major), b_l] for
 * l = 0..3.  Class c proposes beta = cp_als_qr_mlp_beta(c). */
#define CPQR_MLP_FEATURES 32
#define CPQR_MLP_HIDDEN 128
#define CPQR_MLP_CLASSES 8
#define CPQR_MLP_NPARAMS (32 * 128 + 128 + 2 * (128 * 128 + 128) + 128 * 8 + 8)

/* The device proposer state of a CPQR_EXTRAP_LEARNED context after its last sweep: the features
 * (CPQR_MLP_FEATURES floats, as cpqr_mlp_features defines them), the logits (CPQR_MLP_CLASSES)
 * and the proposed class (any pointer may be NULL).  CPQR_EUNSUPPORTED without a learned model. */
cpqr_status cp_als_qr_mlp_state(cpqr_ctx* ctx, float* features_host, float* logits_host, int32_t* cls);

/* beta of class c (0 <= c < CPQR_MLP_CLASSES); class 0 is beta = 0; NaN otherwise. */
double cp_als_qr_mlp_beta(int32_t c);

/* Feature vector (CPQR_MLP_FEATURES floats, host) after sweep n from the fits and betas of
 * sweeps 1..n (host arrays of n doubles), the beta the Section 4.2 rule would use next and
 * whether the rule has activated.  For the last 8 sweeps j (most recent first):
 * log10(1 - fit)/12, signed log of the fit change, log10(beta + 1e-8)/8; then log10(n+1)/3,
 * log10(rule_beta + 1e-8)/8, the activation flag; the rest zero. */
cpqr_status cpqr_mlp_features(const double* fits, const double* betas, int32_t n, double rule_beta,
                              int32_t activated, float* out_host);

/* Device workspace bytes the MLP entry points need for a batch of B rows. */
int64_t cpqr_mlp_work_bytes(int32_t B);

/* logits (device, B x C) of the features X (device, B x F) under params (device, FP32). */
cpqr_status cpqr_mlp_forward(const float* params_dev, const float* X_dev, int32_t B, float* logits_dev,
                             void* work_dev, void* stream);

/* Mean softmax cross-entropy of labels y (device int32, B) and its gradient with respect to
 * params: grad_dev (CPQR_MLP_NPARAMS floats), loss_dev (1 float). */
cpqr_status cpqr_mlp_grad(const float* params_dev, const float* X_dev, const int32_t* y_dev, int32_t B,
                          float* grad_dev, float* loss_dev, void* work_dev, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on params with moments m, v (device). */
cpqr_status cpqr_mlp_adam(float* params_dev, float* m_dev, float* v_dev, const float* grad_dev, float lr,
                          int32_t step, void* stream);

/* ---- Checkpoint / rollback of a context (used for speculative sweeps) ----
 * checkpoint: saves every piece of solver state (factors, their QRs, Q0^{k-1}, weights, beta
 * rule, schedule and cached tree nodes, fit history) in the context's one checkpoint slot.
 * rollback: restores it (the slot stays valid, so several branches can start from it).
 * commit: drops the slot.  One sweep with a forced beta: cp_als_qr_sweep_beta. */
cpqr_status cp_als_qr_checkpoint(cpqr_ctx* ctx);
cpqr_status cp_als_qr_rollback(cpqr_ctx* ctx);
cpqr_status cp_als_qr_commit(cpqr_ctx* ctx);
cpqr_status cp_als_qr_sweep_beta(cpqr_ctx* ctx, double beta, double* fit_host);

/* Failure-detection test hook (no counterpart in the paper).  The next tensor-core TTM of a
 * split-precision context issues no tile loads and its pipeline waits give up after limit_ns
 * nanoseconds: the kernel raises CPQR_DEV_TIMEOUT, every warp leaves its loop, nothing is left
 * in flight and tensor memory is freed, so the GPU context stays usable.  The sweep that ran it
 * returns CPQR_ETIMEOUT, which is sticky: every later call on the context returns it, and
 * cp_als_qr_destroy still releases everything.  CPQR_EUNSUPPORTED for an FP64 context. */
cpqr_status cp_als_qr_test_wait_timeout(cpqr_ctx* ctx, uint64_t limit_ns);

/* Fit and beta history of a context: up to cap sweeps into fits_host / betas_host (either may
 * be NULL); *n = sweeps done.  rule_beta / activated (may be NULL): the Section 4.2 rule state. */
cpqr_status cp_als_qr_history(cpqr_ctx* ctx, double* fits_host, double* betas_host, int32_t cap, int32_t* n,
                              double* rule_beta, int32_t* activated);

#ifdef __cplusplus
}
#endif

#endif /* CPQR_H */
