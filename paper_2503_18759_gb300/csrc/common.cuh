// Shared device helpers and launch declarations of the CP-ALS-QR library.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "cpqr.h"

#define CPQR_MAXR 32        // largest rank of the warp-per-factor kernels
#define CPQR_MAXR_WIDE 192  // largest rank of the wide-rank path (wide.cu)
#define CPQR_MAXN 6

// Device-side error flags (bitwise OR into ctx status word).
#define CPQR_DEV_SINGULAR 1u
#define CPQR_DEV_NONFINITE 2u
#define CPQR_DEV_TIMEOUT 4u

namespace cpqr {

// Device and pinned host blocks from the process-wide cache (memcache.cpp): a freed block is kept
// for the next request of the same size on the same device.
cudaError_t cache_malloc(void** p, size_t bytes);
void cache_free(void* p, size_t bytes);
cudaError_t cache_malloc_host(void** p, size_t bytes);
void cache_free_host(void* p, size_t bytes);

// Library status of a device status word: a timed-out wait first (its results are partial), then
// a zero pivot or norm, then a non-finite value.
inline cpqr_status status_of_device_word(unsigned int w) {
  if (w & CPQR_DEV_TIMEOUT) return CPQR_ETIMEOUT;
  if (w & CPQR_DEV_SINGULAR) return CPQR_ESINGULAR;
  if (w & CPQR_DEV_NONFINITE) return CPQR_ENONFINITE;
  return CPQR_OK;
}

// Programmatic dependent launch: the kernel may be scheduled while the previous kernel of the
// stream drains (its launch latency then overlaps that kernel's tail), so it must call
// pdl_wait() before it reads anything an earlier launch wrote.  Only for kernels that are not
// clusters (whose launch this does not shorten).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
// Waits until the grids this one depends on have completed and their writes are visible
// (returns at once for a launch without the programmatic attribute).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Block size of the FP64 small-QR kernels.
constexpr int kQrThreads = 256;

// ----- TTM (ttm.cu) -----
// out[p, r, s] = sum_i T[p, i, s] * Q[i, r] with T of shape (P, K, S), Q K x R row-major.
// TT = element type of T, TQ = element type of Q and of the accumulator, TO = output type.
template <typename TT, typename TQ, typename TO>
cudaError_t launch_ttm(const TT* T, const TQ* Q, TO* out, int64_t P, int64_t K, int64_t S, int R,
                       cudaStream_t st);

// FP32 register-tiled TTM for S == 1 (K % 4 == 0) or S % 4 == 0; cudaErrorNotSupported
// for other shapes (use launch_ttm<float, float, float>).
cudaError_t launch_ttm_f32_tiled(const float* T, const float* Q, float* out, int64_t P, int64_t K, int64_t S, int R,
                                 cudaStream_t st);

// ----- split-precision tensor-core TTM (ttm_tc.cu) -----
// Stages Q (K x R FP64 row-major) as bf16 hi/lo, transposed and padded for the MMA
// B operand: Qt[2][Rp][Kp] with Rp = R rounded up to 16, Kp = K rounded up to 64.
cudaError_t launch_split_q(const double* Q, int64_t K, int R, __nv_bfloat16* Qt, int Rp, int64_t Kp,
                           cudaStream_t st);
// X (n elements FP32) -> Xhi, Xlo bf16 with X = hi + lo + O(2^-16 |X|).
// X (rows x last, dense FP32) into bf16 hi / lo with rows of ld >= last elements, the padding zero.
cudaError_t launch_split_x_padded(const float* X, __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, int64_t rows, int64_t last,
                                  int64_t ld, cudaStream_t st);
cudaError_t launch_split_x(const float* X, __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, int64_t n,
                           cudaStream_t st);
// Storage of a bf16 split source: dense (ld = 0), or its last dimension (extent last) padded to a
// row stride of ld elements (ld a multiple of 8 >= last, the padding zero), so that TMA's 16-byte
// row strides hold for any last side.
struct SplitLayout {
  int64_t last = 0, ld = 0;
};
// How a TTM of (P, K, S) sees a source with layout lay: the iteration extent of S (Sit), the
// stride between consecutive K (rowS, elements), the dense output extent So, and the remap of an
// iteration index s onto the output, (s / s_pad) s_last + s % s_pad with s % s_pad < s_last, when
// S spans rows of the padded last dimension (s_pad = 0: none).  ok = false: the layout cannot
// serve this TTM.
struct TtmView {
  bool ok;
  int64_t Sit, rowS, So, s_last, s_pad, ldK;
};
TtmView ttm_view(int64_t K, int64_t S, SplitLayout lay);
// out[p, r, s] = sum_i X[p, i, s] Q[i, r] from split operands; out FP32 and, if out_hi /
// out_lo are given, its bf16 split (the operand format of a following tensor-core TTM).
// Dense sources: S % 8 == 0 (MN-major) or S == 1 with K % 8 == 0 (K-major); a padded source
// (lay): any S that ttm_view serves; out_lay: the layout of the split copy of out (padded rows of
// its last dimension, as a padded source).  K <= 512.  Returns cudaErrorNotSupported if the shape is
// outside the kernel's range.
// reserve_sms: SMs the persistent grid leaves free for concurrent work (a cluster QR).
cudaError_t launch_ttm_tc(const __nv_bfloat16* Xhi, const __nv_bfloat16* Xlo, const __nv_bfloat16* Qt,
                          int Rp, int64_t Kp, float* out, int64_t P, int64_t K, int64_t S, int R,
                          unsigned int* dev_status, cudaStream_t st, int reserve_sms = 0,
                          __nv_bfloat16* out_hi = nullptr, __nv_bfloat16* out_lo = nullptr,
                          unsigned long long wait_ns = 0, int skip_x_loads = 0, SplitLayout lay = {},
                          SplitLayout out_lay = {});
bool ttm_tc_supported(int64_t P, int64_t K, int64_t S, int R, SplitLayout lay = {});

// ----- small FP64 kernels (smallqr.cu) -----
struct ZPlan {          // row order of the Khatri-Rao product used by the staircase QR
  int m;                // number of triangles in the product
  int R;
  int64_t M;            // R^m rows
  const int32_t* perm;  // device: sorted row t -> original row index
  int32_t act[CPQR_MAXR];  // column j is active on sorted rows [j, act[j])
};

// SMs one cluster QR occupies (its cluster size).
int qr_cluster_sms();

// Plain QR of an M x R FP64 row-major matrix (device): Q (M x R), R (R x R), diag(R) > 0.
cudaError_t launch_house_qr(const double* A, int64_t M, int R, double* Q, double* Rout, double* work,
                            unsigned int* dev_status, cudaStream_t st);
size_t house_qr_work_doubles(int64_t M, int R);

// QR of Z = R_{k_1} (.) ... (.) R_{k_m}: Rs holds pointers to the m triangles (device).
struct TriPtrs {
  const double* p[CPQR_MAXN];
};
// The first Cholesky pass of a guarded Gram-route QR of an M x R matrix Y (device, row stride
// CPQR_MAXR for F and R1, R for Q1): F = striu(E) + diag(E) / 2 with E = Q1^T Q1 - I, Q1 (M x R)
// and R1 with Q1 R1 = Y.  Given to the fallback QR, a flag of exactly 1 (the first pass's E too
// large for its first-order correction, every pivot positive) makes it finish by a second
// Cholesky pass instead of the Householder QR: R2 = chol(I + E), Q = Q1 R2^{-1}, R = R2 R1.
struct CholQr2Src {
  const double* F;
  const double* Q1;
  const double* R1;
};
// run_if (optional device triple): the QR runs only if run_if[0] != 0; a Householder QR that runs
// adds 1 to run_if[1], a second Cholesky pass (c2 given, run_if[0] == 1) adds 1 to run_if[2].
cudaError_t launch_krp_qr(const ZPlan& plan, TriPtrs Rs, double* Q0, double* R0, double* work,
                          unsigned int* dev_status, cudaStream_t st, float* Q0f = nullptr, int* run_if = nullptr,
                          const CholQr2Src* c2 = nullptr);
size_t krp_qr_work_doubles(const ZPlan& plan);
// QR of a product of m >= 2 triangles as m - 1 staircase QRs of two-triangle products (plan2:
// the plan for m = 2) and m - 2 FP64 assemblies; work: krp_nested_work_doubles(m, R) doubles.
// *nlaunch (optional) receives the number of kernels launched.
size_t krp_nested_work_doubles(int m, int R);
// out[(i, w), c] = sum_j QW[w, j] QY[(i, j), c] (i < R, w < mw): the assembly step of the nested QR,
// for a QY whose row (i, j) is zero left of column max(i, j) (the Gram route's; the Householder
// route assembles with a dense kernel).
cudaError_t launch_krp_assemble(const double* QW, int64_t mw, const double* QY, int R, double* out, float* outf,
                                cudaStream_t st);
// The same with rows (l, i, t) = (l * R + i) * T + t and w = l * T + t (l < L, t < T).
cudaError_t launch_krp_assemble_tri(const double* QW, int64_t L, int64_t T, const double* QY, int R, double* out,
                                    float* outf, cudaStream_t st);
// Buffers of the nested QR inside its work (krp_nested_work_doubles(m, R) doubles): the two level
// triangles S, Q_Y, the staircase QR's scratch and the two Q_W.
struct NestedBufs {
  double* S[2];
  double* QY;
  double* qrw;
  double* QW[2];
};
NestedBufs nested_views(double* work, int m, int R);
// run_if (optional): every launch returns at once unless run_if[0] != 0 (the guarded fallback of
// the Gram route; each staircase QR that runs adds 1 to run_if[1]).
cudaError_t launch_krp_qr_nested(const ZPlan& plan2, TriPtrs Rs, int m, double* Q0, double* R0, double* work,
                                 unsigned int* dev_status, cudaStream_t st, float* Q0f = nullptr,
                                 int* nlaunch = nullptr, int* run_if = nullptr);
// QR of Z = R_1 (.) ... (.) R_m (m >= 2; plan2: the two-triangle plan) by the guarded Gram route
// (krp_gram.cu): for m = 2, Cholesky of the Hadamard product of the triangles' equilibrated Grams,
// FP64 rows over the R^2 rows of Z, one orthogonality correction; for m >= 3 the same for every
// two-triangle level of the nested QR (level d's Gram is the Hadamard product of the last d
// Grams) with the nested assembly between levels.  The Householder QR (the staircase QR, nested
// for m >= 3) is the fallback when a pivot fails or a correction is not small.  gram_work:
// krp_gram_work_doubles(R) doubles; qr_work: krp_nested_work_doubles(m, R) doubles (m >= 3; the
// staircase QR's scratch for m = 2).
size_t krp_gram_work_doubles(int R);
cudaError_t launch_krp_qr_gram(const ZPlan& plan2, TriPtrs tri, int m, double* Q0, double* R0, double* gram_work,
                               double* qr_work, unsigned int* dev_status, cudaStream_t st, float* Q0f = nullptr);
// The same in two phases.  ..._chol: a Cholesky from stored Grams (float-float, 32 x 32 upper) and
// column norms: for the QR, the last two triangles' (level 2; the whole product for m = 2); acc = 1
// keeps the guard of earlier levels.  ..._rows: everything after, with the Grams of all m
// triangles (gp, in the order of tri) for the later levels.  *nlaunch (optional): kernels
// launched by ..._rows.
struct GramPtrs {
  const float2* g[CPQR_MAXN - 1];
  const double* s[CPQR_MAXN - 1];
};
// flag_in (optional, device): a guard raised elsewhere (the split route's W) that the Cholesky
// carries into its own.  fallback = false leaves out the Householder fallback (the split route's
// W, whose guard the final level carries).
cudaError_t launch_krp_chol(const GramPtrs& gp, int m, int R, double* gram_work, cudaStream_t st, int acc = 0,
                            const int* flag_in = nullptr);
cudaError_t launch_krp_rows(const ZPlan& plan2, TriPtrs tri, int m, const GramPtrs& gp, double* Q0, double* R0,
                            double* gram_work, double* qr_work, unsigned int* dev_status, cudaStream_t st,
                            float* Q0f = nullptr, int* nlaunch = nullptr, bool fallback = true);
// Split route of the same QR (m >= 3), for a product whose triangle at position s (tri.p[s]) is the
// only one that changed since the QR of the others, W = Q_W S_W (rows w = (l, t) over the triangles
// before and after s; QW: R^(m-1) x R, SW: R x R), was formed: Y = R_s (.) S_W by the Gram route
// (its Cholesky, the Hadamard product of all m Grams, issued first by launch_krp_chol with W's
// guard as flag_in), Q0[(l, i, t)] = sum_j QW[(l, t), j] Q_Y[(i, j)], R0 = R_Y, and the nested
// Householder QR of tri as the fallback.  gram_work, qr_work: as for launch_krp_rows with m.
cudaError_t launch_krp_rows_split(const ZPlan& plan2, TriPtrs tri, int m, int s, const double* QW, const double* SW,
                                  double* Q0, double* R0, double* gram_work, double* qr_work,
                                  unsigned int* dev_status, cudaStream_t st, float* Q0f = nullptr,
                                  int* nlaunch = nullptr);
// The guard word of a Gram-route workspace (device int: nonzero = fall back).
int* gram_flag(double* gram_work);

// V[i, c] = sum_{p, s} Y[p, i, s] * Qc[p*S + s, c], c < C, Qc = [Q0 | Q0prev] (K x C,
// K = P*S), as *nparts split-K slices of I x C in work (leaf_v_splits(I, K) * I * C
// elements).  FP64 path: Y, Q0, slices FP64; split path: Y, Q0 copies, slices FP32.
int leaf_v_splits(int64_t I, int64_t K);
template <typename TY, typename TQ>
cudaError_t launch_leaf_v(const TY* Y, int64_t P, int64_t I, int64_t S, const TQ* Q0, const TQ* Q0prev, int R, int C,
                          TQ* work, int* nparts, cudaStream_t st);

// Mode update, Alg. 3 lines 5 and 7-8: adds the nparts slices of V = [V0 | V1] (I x C,
// C = R or 2R), V^ = (1+beta) V0 - alpha beta V1 (eq. 19), A^ = V^ R0^{-T} into Ahat (I x R),
// and per-block partials of <V0, V^>, ||V^||^2 into fitpart (finish_prep_blocks(I) x 2);
// hpart (optional): per-block folded partials of A^T A^ (finish_prep_blocks(I) x 17 x 32).
int finish_prep_blocks(int64_t I);
template <typename TP>
cudaError_t launch_finish_prep(const TP* parts, int nparts, int64_t I, int C, int R, const double* R0, double beta,
                               double alpha, double* Ahat, double* fitpart, double* hpart,
                               unsigned int* dev_status, cudaStream_t st);

// Finish of a mode update (Alg. 3 lines 9-10): lambda = column norms of A^, A = A^ / lambda,
// A = Q_n R_n; the fit terms <V0, V^>, ||V^||^2 from the nfit block partials.
struct FinishOut {
  double* A;        // I x R
  double* lambda;   // R
  double* Q;        // I x R
  double* Rn;       // R x R
  float* Qf;        // I x R FP32 copy (may be null)
  double* fit_terms;  // 2 doubles
  // optional: Q^T split into bf16 hi / lo for the tensor-core TTMs, Qt[2][Rp][Kp] with the
  // padding left untouched (zero from the state's initialisation)
  __nv_bfloat16* Qt = nullptr;
  int Rp = 0;
  int64_t Kp = 0;
};
cudaError_t launch_mode_finish(const double* Ahat, const double* fitpart, int nfit, int64_t I, int R, FinishOut out,
                               double* work, unsigned int* dev_status, cudaStream_t st, int* run_if = nullptr,
                               const CholQr2Src* c2 = nullptr);
// The same finish by the guarded Gram route (krp_gram.cu): Gram of A^ from the hpart block
// partials of launch_finish_prep, lambda, Cholesky of the equilibrated Gram (..._chol, which can
// also store the new factor's equilibrated Gram, float-float 32 x 32 upper, and its unit column
// norms), row-parallel substitution and one orthogonality correction (..._rows); the Householder
// finish runs instead (launched last, returning at once otherwise) when a pivot fails or the
// correction is not small.  gram_work: factor_gram_work_doubles(Imax, R) doubles; qr_work: the
// Householder finish's scratch.  launch_finish_gram = ..._chol without the Gram, then ..._rows.
size_t factor_gram_work_doubles(int64_t Imax, int R);
cudaError_t launch_finish_gram_chol(const double* hpart, const double* fitpart, int nblk, int64_t I, int R,
                                    FinishOut out, double* gram_work, float2* gram_out, double* colnorm_out,
                                    cudaStream_t st);
cudaError_t launch_finish_gram_rows(const double* Ahat, const double* fitpart, int nblk, int64_t I, int R,
                                    FinishOut out, double* gram_work, double* qr_work, unsigned int* dev_status,
                                    cudaStream_t st);
cudaError_t launch_finish_gram(const double* Ahat, const double* hpart, const double* fitpart, int nblk, int64_t I,
                               int R, FinishOut out, double* gram_work, double* qr_work, unsigned int* dev_status,
                               cudaStream_t st);
// Equilibrated Gram (float-float, 32 x 32 upper) and column norms of the factor whose QR
// triangle is T (R x R upper, device): for factors without a Gram from the finish.
cudaError_t launch_tri_gram(const double* T, int R, float2* Gf, double* s, cudaStream_t st);
// Runs of the Householder fallback recorded in a Gram-route workspace (device int counter).
int* gram_fallback_counter(double* gram_work);
// Runs of the second Cholesky pass recorded in a Gram-route workspace (device int counter).
int* gram_second_pass_counter(double* gram_work);

// ||X||^2 in FP64: block partials into work (norm2_work_doubles()), summed in a fixed order into
// out[0], so every context on the same tensor gets the same bits.
template <typename TX>
cudaError_t launch_norm2(const TX* X, int64_t n, double* out, double* work, cudaStream_t st);
size_t norm2_work_doubles();
// out[0] = sum of part[0..np-1] in a fixed order (one block).
cudaError_t launch_sum_parts(const double* part, int np, double* out, cudaStream_t st);

// ||X - [[lambda; A]]||^2 (FP32 model entries, FP64 total); X dims d[0..N-1]; A: host array of N
// device pointers; work: device scratch of residual2_work_bytes(N, d, R).  FP32 tensors whose
// last dimension is a multiple of 4 go to the tensor-core kernel (residual_tc.cu), the rest to
// a CUDA-core kernel.  dev_status collects CPQR_DEV_TIMEOUT of the tensor-core kernel.
// parts: RESIDUAL_SNAPSHOT converts the factors (FP32, lambda folded) into work;
// RESIDUAL_EVALUATE computes the residual from the snapshot in work (the two may run on
// different streams, the snapshot first).  reserve_sms: SMs of one cluster QR to leave free.
size_t residual2_work_bytes(int N, const int64_t* d, int R);
constexpr int RESIDUAL_SNAPSHOT = 1, RESIDUAL_EVALUATE = 2;
template <typename TX>
cudaError_t launch_residual2(const TX* X, int N, const int64_t* d, const double* const* A,
                             const double* lambda, int R, double* out, double* work, unsigned int* dev_status,
                             cudaStream_t st, int parts = RESIDUAL_SNAPSHOT | RESIDUAL_EVALUATE, int reserve_sms = 0);

// ----- tensor-core explicit residual (residual_tc.cu) -----
// Af: host array of N device pointers to the FP32 factors (lambda folded into Af[0], Af[N-1]
// stored transposed, R x I_last); accumulates ||X - K||^2 into *out (not cleared).
bool residual_tc_supported(int N, const int64_t* d, int R, const void* X);
cudaError_t launch_residual_tc(const float* X, int N, const int64_t* d, const float* const* Af, int R, double* part,
                               int max_parts, int* nparts, unsigned int* dev_status, cudaStream_t st,
                               int reserve_sms = 0);

cudaError_t launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t st);

// ----- learned proposer (mlp.cu) -----
// ---- wide-rank path (32 < R <= CPQR_MAXR_WIDE), wide.cu ----
bool wide_supported(int R);
size_t wide_work_doubles(int R);
// Cholesky QR (see wide.cu) of Y (M x R rows) or, with tri / m > 0, of the Khatri-Rao product of the
// m upper triangles tri[0..m-1] (rows (i_1, ..., i_m), i_m fastest).
cudaError_t launch_wide_qr(const double* Y, int64_t M, int R, const double* const* tri, int m, double* Q, float* Qf,
                           double* Rout, double* work, unsigned int* status, cudaStream_t st);
// A^ = V^ R0^{-T} (eq. 19 on the V slices), fit terms, lambda and A = A^ / lambda.  work_rows: I (R + 2).
template <typename TV>
cudaError_t launch_wide_finish(const TV* vw, int nparts, int64_t I, int C, int R, const double* R0, double beta,
                               double alpha, double* A, double* lambda, double* fit_terms, double* work_rows,
                               unsigned int* status, cudaStream_t st);
// Tensor-core TTM for 32 < R <= 192 (ttm_tc_wide.cu): operands as for launch_ttm_tc, Rp = R rounded
// up to 16, Qt = bf16 hi / lo of Q^T (2 x Rp x Kp).
bool ttm_tc_wide_supported(int64_t P, int64_t K, int64_t S, int R, SplitLayout lay = {});
cudaError_t launch_ttm_tc_wide(const __nv_bfloat16* Xhi, const __nv_bfloat16* Xlo, const __nv_bfloat16* Qt, int Rp,
                               int64_t Kp, float* out, int64_t P, int64_t K, int64_t S, int R,
                               unsigned int* dev_status, cudaStream_t st, __nv_bfloat16* out_hi = nullptr,
                               __nv_bfloat16* out_lo = nullptr, SplitLayout lay = {}, SplitLayout out_lay = {});
// TTM on the CUDA cores for any R (tiled GEMM, accumulation in TAcc).
template <typename TT, typename TQ, typename TO, typename TAcc>
cudaError_t launch_ttm_wide(const TT* T, const TQ* Q, TO* out, int64_t P, int64_t K, int64_t S, int R,
                            cudaStream_t st);

// Device state of the learned proposer (kept in the solver's state arena, so a checkpoint saves it):
// the fits of the last MLP_RING + 1 sweeps and the betas of the last MLP_RING (most recent last),
// the Section 4.2 rule's state, and the last features, logits and proposed class.
constexpr int MLP_RING = 8;
struct MlpState {
  double fit[MLP_RING + 1];
  double beta[MLP_RING];
  double rule_beta;
  int32_t n, activated, cls, pad;
  float feat[CPQR_MLP_FEATURES];
  float logits[CPQR_MLP_CLASSES];
};
// Where a sweep's fit comes from: the explicit residual r2 (split path), else the fit terms
// <V0, V^>, ||V^||^2 of the last update (FP64 path).
struct MlpFitSource {
  const double* r2;
  const double* terms;
  double normX2;
};
// bf16 transposed weights (CPQR_MLP_NPARAMS slots) from the FP32 parameters.
cudaError_t mlp_prepare_weights(const float* params, __nv_bfloat16* wt, cudaStream_t st);
// After a sweep that used beta_used: update the state and propose the next sweep's class.
cudaError_t mlp_propose(const __nv_bfloat16* wt, const float* params, MlpState* state, MlpFitSource src,
                        double beta_used, cudaStream_t st);
size_t mlp_work_bytes(int B);
cudaError_t mlp_forward(const float* params, const float* X, int B, float* logits, void* work, cudaStream_t st);
cudaError_t mlp_grad(const float* params, const float* X, const int32_t* y, int B, float* grad, float* loss,
                     void* work, cudaStream_t st);
cudaError_t mlp_adam(float* params, float* m, float* v, const float* grad, float lr, int step, cudaStream_t st);

}  // namespace cpqr
