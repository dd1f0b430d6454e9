// QRs by the Gram route, guarded by the Householder QR:
//  - the Khatri-Rao product of two upper triangles, Z = R_a (.) R_b (R^2 x R, Alg. 2 lines 3-4
//    for order-3 tensors and the building block of the nested QR for higher orders);
//  - the factor of a mode update, A = A^ / lambda (I x R, Alg. 2 lines 9-10), whose Gram
//    comes from per-block partials written by the R0^{-T} solve that produces A^.
//
// Z's Gram matrix needs no pass over Z: Z^T Z = (R_a^T R_a) o (R_b^T R_b) (Hadamard product),
// because row (i, k) of Z is R_a[i, :] o R_b[k, :].  Then
//   R1 = chol(Z^T Z),  Q1 = Z R1^{-1}  (row-wise forward substitution),
//   E = Q1^T Q1 - I,   F = striu(E) + diag(E) / 2,
//   Q0 = Q1 (I - F),   R0 = (I + F) R1,
// i.e. CholeskyQR2 with its second Cholesky factor chol(I + E) = I + F + O(E^2) taken to first
// order.  Q0 R0 = Q1 (I - F^2) R1 = Z - O(|E|^2), Q0^T Q0 = I + O(|E|^2), and R0 has a positive
// diagonal, so (Q0, R0) is the unique QR of Z whenever |E| is small; |E| grows like
// kappa(Z)^2 * 2^-53.  If a pivot of the Cholesky is not positive or max |E| > kEMax, a device flag
// makes the QR kernel launched after these (smallqr.cu) recompute Q0 and R0; otherwise it returns at
// once.  The flag has two levels: max |E| in (kEMax, kE2Max] with every pivot positive (bit 0
// alone) sends it to a second Cholesky pass on Q1 (CholeskyQR2: R2 = chol(I + E), Q = Q1 R2^{-1},
// R = R2 R1), which leaves Q^T Q - I at rounding level because Q1 is already within 1e-3 of
// orthonormal; a failed pivot, a larger or non-finite E (bit 1) send it to the Householder QR.  The Householder QR's stability is thus kept for every Z,
// while the common well-conditioned case costs one 32-step Cholesky plus three row-parallel FP64
// passes over all SMs instead of 32 cluster-wide Householder steps.  For Z, the Gram is the
// Hadamard product of the two factors' stored Grams (kg_chol_kernel); for A, it comes from the
// solve's partials.  Either Gram is equilibrated (unit diagonal: G = D^-1 G D^-1, D = the column
// norms, for A lambda) and its Cholesky runs in float-float (~2^-48): R1 serves only as the
// preconditioner of Q1 = Z R1^{-1}, which is formed in FP64 against whatever R1 is, so its
// precision moves E (|E| ~ kappa^2 2^-48, the guard thus trips near kappa ~ 1e3 instead of 1e4)
// and not the accuracy of an accepted (Q0, R0).
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"
#include "ff.cuh"

namespace cpqr {

namespace {

using namespace ffa;
constexpr unsigned FULL = 0xffffffffu;
constexpr int KG_MAXR = CPQR_MAXR;
constexpr int KG_LD = KG_MAXR + 1;
// max |E| accepted: the neglected O(E^2) terms stay below 1e-16
constexpr double kEMax = 1e-8;
// max |E| handed to the second Cholesky pass instead of the Householder QR
constexpr double kE2Max = 1e-3;

// Workspace layout (doubles, every section 128-byte aligned): the int pair {fallback flag,
// fallback count} (at a fixed offset, so the count survives calls with different row counts),
// R1, S (R1 scaled for the substitution), F, rinv, 1/lambda (the equilibration), KG_MAXM Grams in
// float-float and their column norms (for a QR whose triangles come without stored Grams), F in
// float-float, the block partials of E for many rows (KG_EBLK x 17 x 32), Q1 (M x R), Q1^T (R x M).
constexpr size_t KG_HEAD = 16;
constexpr int KG_MAXM = CPQR_MAXN - 1;  // triangles of a Khatri-Rao product
constexpr int KG_EBLK = 152;            // blocks of the many-row E pass
size_t kg_round16(size_t n) { return (n + 15) / 16 * 16; }
struct KgWork {
  int* flag;
  double* R1;
  double* S;
  double* F;
  double* rinv;
  double* il;
  float2* g[KG_MAXM];
  double* s[KG_MAXM];
  float2* Ff;
  double* epart;
  double* Q1;
  double* Q1T;
};

size_t kg_work_doubles(int64_t M, int R) {
  return KG_HEAD + (5 + KG_MAXM) * (size_t)KG_MAXR * KG_MAXR + (2 + KG_MAXM) * KG_MAXR +
         kg_round16((size_t)KG_EBLK * 17 * 32) + 2 * kg_round16((size_t)M * R);
}

KgWork kg_views(double* work, int R, int64_t M) {
  KgWork w;
  const size_t rr = (size_t)KG_MAXR * KG_MAXR;
  w.flag = reinterpret_cast<int*>(work);
  w.R1 = work + KG_HEAD;
  w.S = w.R1 + rr;
  w.F = w.S + rr;
  w.rinv = w.F + rr;
  w.il = w.rinv + KG_MAXR;
  double* p = w.il + KG_MAXR;
  for (int k = 0; k < KG_MAXM; ++k, p += rr) w.g[k] = reinterpret_cast<float2*>(p);
  for (int k = 0; k < KG_MAXM; ++k, p += KG_MAXR) w.s[k] = p;
  w.Ff = reinterpret_cast<float2*>(p);
  w.epart = p + rr;
  w.Q1 = w.epart + kg_round16((size_t)KG_EBLK * 17 * 32);
  w.Q1T = w.Q1 + kg_round16((size_t)M * R);
  return w;
}

// Gram (Hadamard of the two triangles' Grams) and its Cholesky factor on one 16-CTA cluster of
// 256 threads: CTA r forms rows c = r, r + 16 of the Gram (FP64 on one SM is ~8 GFLOP/s, so the
// two triangular products are spread) and stores them into CTA 0's shared memory; CTA 0 then
// runs the Cholesky (chol_pipelined).
constexpr int KG_CL = 16;
constexpr int KG_GK = 17;  // folded Gram entries per lane in the finish-prep partials

// named barriers of 256 threads (barrier 0 is __syncthreads)
__device__ __forceinline__ void nb_arrive(int id) { asm volatile("bar.arrive %0, 256;" ::"r"(id) : "memory"); }
__device__ __forceinline__ void nb_sync(int id) { asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory"); }

// CTA 0 of a Cholesky kernel, G (FP64, R x R block, both triangles) complete: scale = sqrt(diag
// G), il = 1 / scale (rsqrt.approx.f64, measured to 53 bits; 0 for a zero or non-finite column,
// whose zero row then fails its pivot), the equilibrated Gram Gf = D^-1 G D^-1 in float-float
// (unit diagonal, entries in [-1, 1]; upper triangle, entries visited as the folded pairs
// (c, (c + k) % 32), k = 0..16, so that every FP64 warp instruction has 32 live lanes), U = V = 0.
__device__ __forceinline__ void equilibrate_ff(double (*G)[KG_LD], float2 (*Gf)[KG_LD], float2 (*U)[KG_LD],
                                               float2 (*V)[KG_LD], double* scale, double* il, float2* ilf, int R,
                                               const KgWork& w) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < 32) {
    const double g = (lane < R) ? G[lane][lane] : 0.0;
    const long long b = __double_as_longlong(g);
    double y = 0.0;
    if (b > 0x05CD0B15A491EB84LL && b < 0x7A11A0FC668AAC70LL) {  // 1e-280 < g < 1e280
      asm("rsqrt.approx.f64 %0, %1;" : "=d"(y) : "d"(g));
    } else if (g > 0.0 && g < 1e300) {
      y = 1.0 / sqrt(g);
    }
    scale[lane] = (y > 0.0) ? g * y : 0.0;
    il[lane] = y;
    ilf[lane] = ff_st(ff_from_bits(y));
    w.il[lane] = y;
  }
  for (int e = tid; e < KG_MAXR * KG_MAXR; e += blockDim.x) {
    U[e / KG_MAXR][e % KG_MAXR] = make_float2(0.0f, 0.0f);
    V[e / KG_MAXR][e % KG_MAXR] = make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  for (int k = warp; k <= KG_MAXR / 2; k += (int)(blockDim.x >> 5)) {
    const int c = lane, d = (lane + k) & 31;
    const int i = min(c, d), j = max(c, d);
    const ffn x = ff_from_bits(G[i][j]);
    Gf[i][j] = (j < R) ? ff_st(ff_mul(ff_mul(x, ff_ld(ilf[i])), ff_ld(ilf[j]))) : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
}

// Cholesky of the R x R leading block of G (256 threads; shared G, U, V in float-float, U and V
// zero on entry, G overwritten) in square-root-free form: U[j] is row j of the Schur complement
// after j steps (U[j][j] = d_j, the pivot) and V[j] = U[j] / d_j, so that step j subtracts
// V[j][k] U[j][l] from G[k][l], and R1 = diag(d)^-1/2 U (chol_outputs).  The square roots are
// thus off the serial chain, which per row is one fused multiply-subtract, one shuffle and one
// reciprocal.
//
// Pipelining: warp 0 produces the rows and keeps the next one in registers.  At iteration j it
// finishes row j by applying step j - 1 to the copy it prepared (with z = U[j-1][j] U[j-1]
// formed while the reciprocal of d_{j-1} was in flight), and meanwhile prepares row j + 1:
// it loads it once warps 1-7 have applied the steps up to j - 2, then applies step j - 1 itself.
// So warps 1-7 apply step s to rows >= s + 3, and no shared-memory load sits on the chain.
// "Row j of U, V written": warp 0 arrives, warps 1-7 wait, on barrier 1 (j even) or 3 (j odd).
// "Step s applied": warps 1-7 arrive, warp 0 waits at iteration s + 2 before loading row s + 3,
// on barrier 2 (s even) or 4 (s odd).  Two barriers per role because either side may arrive
// one generation ahead: warp 0 posts row j + 1 before the others have taken row j, and a warp may
// post step s + 1 before warp 0 has taken step s.  Row j + 2 is posted only after warp 0 has
// taken step j (so all of warps 1-7 took row j), and step s + 2 only after row s + 2, which
// follows warp 0's wait on step s: each barrier's previous generation is complete before its
// next use.
__device__ __forceinline__ void chol_pipelined(float2 (*G)[KG_LD], float2 (*U)[KG_LD], float2 (*V)[KG_LD], int R,
                                               int* bad) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool in = lane < R;
  const ffn zero = ff_make(0.0f, 0.0f);
  if (warp == 0) {
    // row 0; the prepared copy of row 1 needs no step yet
    ffn u = in ? ff_ld(G[0][lane]) : zero;
    ffn nxt = (in && lane >= 1 && R > 1) ? ff_ld(G[1][lane]) : zero;
    ffn w = ff_recip(ff_shfl(u, 0), bad);
    ffn z = ff_mul(ff_shfl(u, 1), u);         // U[0][1] U[0][l]: step 0 on row 1
    ffn z2 = ff_mul(ff_shfl(u, 2 & 31), u);  // U[0][2] U[0][l]: step 0 on row 2
    if (in) {
      U[0][lane] = ff_st(u);
      V[0][lane] = ff_st(ff_mul(u, w));
    }
    __syncwarp();
    nb_arrive(1);  // row 0
    for (int j = 1; j < R; ++j) {
      const bool live = in && lane >= j;
      u = live ? ff_fms(nxt, w, z) : zero;  // step j - 1 on row j
      // row j + 1 after steps up to j - 2 from warps 1-7 (j >= 2): its load is issued before the
      // reciprocal's dependent chain, which then hides its latency
      if (j >= 2) nb_sync(2 + 2 * ((j - 2) & 1));
      const bool live1 = in && lane >= j + 1;
      const ffn t = live1 ? ff_ld(G[j + 1][lane]) : zero;
      const ffn w1 = w, z21 = z2;
      w = ff_recip(ff_shfl(u, j), bad);
      z = ff_mul(ff_shfl(u, (j + 1) & 31), u);   // step j on row j + 1
      z2 = ff_mul(ff_shfl(u, (j + 2) & 31), u);  // step j on row j + 2
      nxt = live1 ? ff_fms(t, w1, z21) : zero;   // step j - 1 on row j + 1
      if (live) {
        U[j][lane] = ff_st(u);
        V[j][lane] = ff_st(ff_mul(u, w));
      }
      __syncwarp();
      nb_arrive(1 + 2 * (j & 1));  // row j
    }
  } else {
    for (int s = 0; s + 1 < R; ++s) {
      nb_sync(1 + 2 * (s & 1));  // row s of U, V is there
      const ffn us = in ? ff_ld(U[s][lane]) : zero;
      // this warp's rows k = s + 2 + warp + 7 q (rows s + 3, ...; at most 5): every load first
      constexpr int KQ = (KG_MAXR + 6) / 7;
      ffn m[KQ], g[KQ];
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        const int k = s + 2 + warp + 7 * q;
        m[q] = (k < R) ? ff_ld(V[s][k]) : zero;
        g[q] = (k < R && in && lane >= k) ? ff_ld(G[k][lane]) : zero;
      }
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        const int k = s + 2 + warp + 7 * q;
        if (k < R && in && lane >= k) G[k][lane] = ff_st(ff_fms(g[q], m[q], us));
      }
      if (s + 2 < R) nb_arrive(2 + 2 * (s & 1));  // step s
    }
    nb_sync(1 + 2 * ((R - 1) & 1));  // the last row
  }
}

// After chol_pipelined (and a __syncthreads): rinv = d^-1/2 (FP64, rsqrt.approx.f64, measured
// to 53 bits, in the normal range), S[c][c'] = V[c][c'] (c < c', for the substitution of the
// equilibrated rows) and R1 diag(colscale) (colscale: the equilibration scale to undo, or null),
// with R1 taken as the triangle the substitution implies: R1[c][c] = r_c = d_c rinv_c (= 1 /
// rinv_c to FP64 rounding) and R1[c][c'] = S[c][c'] r_c.  So Q1 R1 = Z holds to FP64 rounding
// whatever the float-float rounding of U and V was, which the accuracy of Q0 R0 relies on.
// Upper-triangle entries are visited as folded pairs (all lanes live); the flag last.  rsd, csd:
// 32 doubles of shared scratch each.
__device__ __forceinline__ void chol_outputs(float2 (*U)[KG_LD], float2 (*V)[KG_LD], double* rsd, double* csd,
                                             const double* colscale, int R, const KgWork& w, int* bad,
                                             int acc = 0) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < 32) {
    const double d = (lane < R) ? ff_val(U[lane][lane]) : 1.0;
    const long long b = __double_as_longlong(d);
    double y;
    if (b > 0x05CD0B15A491EB84LL && b < 0x7A11A0FC668AAC70LL) {  // 1e-280 < d < 1e280
      asm("rsqrt.approx.f64 %0, %1;" : "=d"(y) : "d"(d));
    } else {
      y = (d > 0.0) ? 1.0 / sqrt(d) : 0.0;
      if (!(d > 0.0)) *bad = 1;
    }
    if (lane >= R) y = 0.0;
    rsd[lane] = d * y;
    csd[lane] = colscale ? colscale[lane] : 1.0;
    w.rinv[lane] = y;
  }
  for (int e = tid; e < KG_MAXR * KG_MAXR; e += blockDim.x) {  // strict lower triangles
    const int c = e / KG_MAXR, d = e % KG_MAXR;
    if (d < c) {
      w.R1[e] = 0.0;
      w.S[e] = 0.0;
    }
  }
  __syncthreads();
  for (int k = warp; k <= KG_MAXR / 2; k += (int)(blockDim.x >> 5)) {
    const int c = lane, d = (lane + k) & 31;
    const int i = min(c, d), j = max(c, d);
    const bool live = j < R;
    const double sv = (live && j > i) ? ff_val(V[i][j]) : 0.0;
    const double r = live ? ((j == i) ? rsd[i] : sv * rsd[i]) * csd[j] : 0.0;
    w.R1[i * KG_MAXR + j] = r;
    w.S[i * KG_MAXR + j] = sv;
  }
  // bit 1 of the flag: a pivot failed (acc: a later level of one nested QR)
  if (tid == 0) *w.flag = acc ? (*w.flag | (*bad ? 2 : 0)) : (*bad ? 2 : 0);
}

// Equilibrated Gram of an upper triangle T (one CTA of 256 threads per triangle, FP64):
// G = T^T T, s = sqrt(diag G) (the column norms of any A = Q T), Gf = D^-1 G D^-1 in float-float
// (upper triangle, row stride 32), s to global.  For triangles that come without a stored Gram
// (the starting factors, the stand-alone Khatri-Rao QR); not on the sweep's path.
__global__ void __launch_bounds__(256) tri_gram_kernel(TriPtrs tri, int R, float2* __restrict__ Gf_out,
                                                        double* __restrict__ s_out) {
  __shared__ double sT[KG_MAXR][KG_LD], G[KG_MAXR][KG_LD], sil[KG_MAXR];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* T = tri.p[blockIdx.x];
  for (int e = tid; e < KG_MAXR * KG_MAXR; e += 256) {
    const int i = e / KG_MAXR, c = e % KG_MAXR;
    sT[i][c] = (i < R && c < R) ? T[i * R + c] : 0.0;
  }
  __syncthreads();
  for (int c = warp; c < KG_MAXR; c += 8) {
    double g = 0.0;
    const int imax = min(c, lane);
    for (int i = 0; i <= imax; ++i) g = fma(sT[i][c], sT[i][lane], g);
    G[c][lane] = g;
  }
  __syncthreads();
  if (tid < 32) {
    const double sc = (lane < R) ? sqrt(G[lane][lane]) : 0.0;
    sil[lane] = (sc > 0.0 && sc < 1e300) ? 1.0 / sc : 0.0;
    s_out[(size_t)blockIdx.x * KG_MAXR + lane] = sc;
  }
  __syncthreads();
  for (int e = tid; e < KG_MAXR * KG_MAXR; e += 256) {
    const int i = e / KG_MAXR, j = e % KG_MAXR;
    Gf_out[(size_t)blockIdx.x * KG_MAXR * KG_MAXR + e] =
        (i <= j && j < R) ? ff_st(ff_from_bits(G[i][j] * sil[i] * sil[j])) : make_float2(0.0f, 0.0f);
  }
}

// Cholesky of the Khatri-Rao product's equilibrated Gram, one CTA of 256 threads.  A row of
// Z = R_1 (.) ... (.) R_m is the Hadamard product of one row of each triangle, so
// Z^T Z = (R_1^T R_1) o ... o (R_m^T R_m) = (A_1^T A_1) o ... o (A_m^T A_m) (up to the rounding
// of the factor QRs), and with the factors' equilibrated Grams G_k (float-float) and column norms
// s_k: Z^T Z = D (G_1 o ... o G_m) D, D = diag(s_1 ... s_m).  The Gram thus costs float-float
// Hadamard products and no pass over the triangles, and this kernel needs only the Grams: a sweep
// launches it as soon as the previous factor's Gram exists, before that factor's QR has finished.
__global__ void __launch_bounds__(256) kg_chol_kernel(GramPtrs gp, int m, int R, int acc, const int* flag_in,
                                                       KgWork w) {
  __shared__ __align__(16) float2 Gf[KG_MAXR][KG_LD], U[KG_MAXR][KG_LD], V[KG_MAXR][KG_LD];
  __shared__ double scale[KG_MAXR], rsd[KG_MAXR], csd[KG_MAXR];
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31;
  pdl_wait();
  if (tid < 32) {
    double sc = (lane < R) ? 1.0 : 0.0;
    for (int k = 0; k < m; ++k) sc *= (lane < R) ? gp.s[k][lane] : 0.0;
    scale[lane] = sc;
    w.il[lane] = (sc > 0.0 && sc < 1e300) ? 1.0 / sc : 0.0;
  }
  if (tid == 0) bad = 0;
  for (int e = tid; e < KG_MAXR * KG_MAXR; e += 256) {
    const int i = e / KG_MAXR, j = e % KG_MAXR;
    float2 g = make_float2(0.0f, 0.0f);
    if (i <= j && j < R) {
      ffn h = ff_ld(gp.g[0][e]);
      for (int k = 1; k < m; ++k) h = ff_mul(h, ff_ld(gp.g[k][e]));
      g = ff_st(h);
    }
    Gf[i][j] = g;
    U[i][j] = make_float2(0.0f, 0.0f);
    V[i][j] = make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  chol_pipelined(Gf, U, V, R, &bad);
  __syncthreads();
  if (tid == 0 && flag_in && *(volatile const int*)flag_in) bad = 1;
  chol_outputs(U, V, rsd, csd, scale, R, w, &bad, acc);
}

// Factor route, Gram and Cholesky on one 16-CTA cluster of 256 threads: CTA r adds up folded
// row k = r (CTA 0 also k = 16) of the block partials hpart[blk][k][c] = sum a^_c a^_(c+k)%32
// (warp w takes blocks w, w + 8, ...; fixed order) and stores G[c][(c+k)%32] and its mirror into
// CTA 0.  CTA 0 then forms lambda = sqrt(diag G), G = D^-1 G D^-1 (also stored, with unit column
// norms, as the new factor's Gram for the following Khatri-Rao QRs), the fit terms from the
// finish-prep partials, and the Cholesky.
__global__ void __cluster_dims__(KG_CL, 1, 1) __launch_bounds__(256)
    fg_chol_kernel(const double* __restrict__ hpart, int nblk, int R, const double* __restrict__ fitpart,
                   double* __restrict__ lambda, double* __restrict__ fit_terms, float2* __restrict__ gram_out,
                   double* __restrict__ colnorm_out, KgWork w) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  __shared__ __align__(16) double G[KG_MAXR][KG_LD];
  __shared__ __align__(16) float2 Gf[KG_MAXR][KG_LD], U[KG_MAXR][KG_LD], V[KG_MAXR][KG_LD];
  __shared__ double red[8][32], scale[KG_MAXR], il[KG_MAXR];
  __shared__ float2 ilf[KG_MAXR];
  __shared__ double rsd[KG_MAXR], csd[KG_MAXR];
  __shared__ int bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) bad = 0;
  for (int k = rank; k < KG_GK; k += KG_CL) {
    const size_t bs = (size_t)KG_GK * 32;
    // 16 blocks per pass with every load issued before the adds (fixed order); the diagonal row
    // (k = 0) in FP64, the others in float-float as the finish prep wrote them
    if (k == 0) {
      const double* hp = hpart + lane;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      for (int b0 = warp; b0 < nblk; b0 += 128) {
        double x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int b = b0 + 8 * u;
          x[u] = (b < nblk) ? hp[(size_t)b * bs] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 16; u += 4) {
          a0 += x[u];
          a1 += x[u + 1];
          a2 += x[u + 2];
          a3 += x[u + 3];
        }
      }
      red[warp][lane] = (a0 + a1) + (a2 + a3);
    } else {
      const float2* hp = reinterpret_cast<const float2*>(hpart) + (size_t)k * 32 + lane;
      ffn a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = ff_make(0.0f, 0.0f);
      for (int b0 = warp; b0 < nblk; b0 += 128) {
        float2 x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int b = b0 + 8 * u;
          x[u] = (b < nblk) ? hp[(size_t)b * bs] : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) a[u & 3] = ff_add(a[u & 3], ff_ld(x[u]));
      }
      red[warp][lane] = ff_val(ff_add(ff_add(a[0], a[1]), ff_add(a[2], a[3])));
    }
    __syncthreads();
    if (warp == 0) {
      const double g = ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
                       ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
      const int c = lane, d = (lane + k) & 31;
      double* G0 = cluster.map_shared_rank(&G[0][0], 0);
      G0[c * KG_LD + d] = g;
      G0[d * KG_LD + c] = g;
    }
    __syncthreads();
  }
  cluster.sync();  // all of G is in CTA 0; the other CTAs are done
  if (rank != 0) return;
  if (warp == 1) {
    // <V0, V^> and ||V^||^2 from the finish-prep block partials (the Householder finish's order)
    double a = 0.0, b = 0.0;
    for (int k = lane; k < nblk; k += 32) {
      a += fitpart[2 * k];
      b += fitpart[2 * k + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(FULL, a, o);
      b += __shfl_xor_sync(FULL, b, o);
    }
    if (lane == 0) {
      fit_terms[0] = a;
      fit_terms[1] = b;
    }
  }
  equilibrate_ff(G, Gf, U, V, scale, il, ilf, R, w);  // scale = lambda, il = 1 / lambda
  if (tid < R) lambda[tid] = scale[tid];
  // the Gram of A = A^ / lambda (unit columns) for the next Khatri-Rao QRs
  if (gram_out) {
    for (int e = tid; e < KG_MAXR * KG_MAXR; e += 256) {
      const int i = e / KG_MAXR, j = e % KG_MAXR;
      gram_out[e] = (i <= j) ? Gf[i][j] : make_float2(0.0f, 0.0f);
    }
    if (tid < 32) colnorm_out[tid] = (tid < R) ? 1.0 : 0.0;
  }
  chol_pipelined(Gf, U, V, R, &bad);
  __syncthreads();
  chol_outputs(U, V, rsd, csd, nullptr, R, w, &bad);
}

// Factor route, Q1 = A R1^{-1} with A = A^ / lambda: one row of A^ per warp (A also written
// out), the forward substitution of kg_q1_kernel.
__global__ void __launch_bounds__(128) fg_q1_kernel(const double* __restrict__ Ahat, int I, int R, KgWork w,
                                                     double* __restrict__ Aout) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * 4 + (threadIdx.x >> 5);
  pdl_wait();
  if (t >= I) return;
  double scol[KG_MAXR];
#pragma unroll
  for (int c = 0; c < KG_MAXR; ++c) scol[c] = (c < R && lane > c && lane < R) ? w.S[c * KG_MAXR + lane] : 0.0;
  const double ri = (lane < R) ? w.rinv[lane] : 0.0;
  double x = 0.0;
  if (lane < R) {
    x = Ahat[(size_t)t * R + lane] * w.il[lane];
    Aout[(size_t)t * R + lane] = x;
  }
#pragma unroll
  for (int c = 0; c < KG_MAXR - 1; ++c) {
    if (c + 1 < R) {
      const double xc = __shfl_sync(FULL, x, c);
      x = fma(-xc, scol[c], x);
    }
  }
  if (lane < R) {
    const double q = x * ri;
    w.Q1[(size_t)t * R + lane] = q;
    w.Q1T[(size_t)lane * I + t] = q;
  }
}

// Q1 = Z R1^{-1} = (Z D^-1) R1e^{-1} (R1e: the equilibrated factor, D = diag(||Z e_c||)): one row
// (i_1, ..., i_m) of Z per warp, z[c] = prod_k R_k[i_k][c] / D[c]; forward substitution q R1e = z with
// lane = column (x[c'] -= x[c] S[c][c'] after column c, q[c] = x[c] / R1e[c][c]).  Writes Q1
// row-major and transposed.
__global__ void __launch_bounds__(128) kg_q1_kernel(TriPtrs tri, int m, int M, int R, KgWork w) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * 4 + (threadIdx.x >> 5);
  pdl_wait();
  if (t >= M) return;
  // column `lane` of S in registers (every load issued up front)
  double scol[KG_MAXR];
#pragma unroll
  for (int c = 0; c < KG_MAXR; ++c) scol[c] = (c < R && lane > c && lane < R) ? w.S[c * KG_MAXR + lane] : 0.0;
  const double ri = (lane < R) ? w.rinv[lane] : 0.0;
  // row t = (i_1, ..., i_m) of Z (i_m fastest), equilibrated like the Gram (column c times
  // 1 / ||Z e_c||)
  double x = 0.0;
  if (lane < R) {
    x = w.il[lane];
    int rest = t;
    for (int k = m - 1; k >= 0; --k) {
      const int ik = rest % R;
      rest /= R;
      x *= tri.p[k][ik * R + lane];
    }
  }
#pragma unroll
  for (int c = 0; c < KG_MAXR - 1; ++c) {
    if (c + 1 < R) {
      const double xc = __shfl_sync(FULL, x, c);
      x = fma(-xc, scol[c], x);
    }
  }
  if (lane < R) {
    const double q = x * ri;
    w.Q1[(size_t)t * R + lane] = q;
    w.Q1T[(size_t)lane * M + t] = q;
  }
}

// E = Q1^T Q1 - I and F = striu(E) + diag(E) / 2: one warp per upper entry (c, d), lanes over
// the rows (coalesced through Q1^T); raises the fallback flag if |E[c][d]| > kEMax.
__global__ void __launch_bounds__(128) kg_e_kernel(int M, int R, KgWork w) {
  const int lane = threadIdx.x & 31;
  const int npair = R * (R + 1) / 2;
  const int gw = blockIdx.x * 4 + (threadIdx.x >> 5);
  pdl_wait();
  if (gw >= npair) return;
  int c = 0, rem = gw;
  while (rem >= R - c) {
    rem -= R - c;
    ++c;
  }
  const int d = c + rem;
  const double* qc = w.Q1T + (size_t)c * M;
  const double* qd = w.Q1T + (size_t)d * M;
  // 32 rows per lane per pass (1024 rows), every load issued before the products
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t0 = 0; t0 < M; t0 += 1024) {
    double xc[32], xd[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const int t = t0 + 32 * u + lane;
      xc[u] = (t < M) ? qc[t] : 0.0;
      xd[u] = (t < M) ? qd[t] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 32; ++u) acc[u & 3] = fma(xc[u], xd[u], acc[u & 3]);
  }
  double s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  if (lane == 0) {
    const double e = (c == d) ? s - 1.0 : s;
    const double f = (c == d) ? 0.5 * e : e;
    w.F[c * KG_MAXR + d] = f;
    w.Ff[c * KG_MAXR + d] = ff_st(ff_from_bits(f));
    if (!(fabs(e) <= kEMax)) atomicOr(w.flag, (fabs(e) <= kE2Max) ? 1 : 3);  // NaN: 3
  }
}

// E for many rows (M > 1024, where one warp per entry would stream all rows): pass 1, KG_EBLK
// blocks of 4 warps, each warp adding the folded products q[c] q[(c+k)%32] (k = 0..16) of rows
// gw, gw + 4 KG_EBLK, ... (four rows loaded ahead); the block's sums to epart[blk][k][c].
__global__ void __launch_bounds__(128) kg_epart_kernel(int M, int R, KgWork w) {
  __shared__ double red[4][17][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * 4 + warp, nw = gridDim.x * 4;
  pdl_wait();
  double h[17];
#pragma unroll
  for (int k = 0; k < 17; ++k) h[k] = 0.0;
  for (int t0 = gw; t0 < M; t0 += 4 * nw) {
    double q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + u * nw;
      q[u] = (t < M && lane < R) ? w.Q1[(size_t)t * R + lane] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 17; ++k) h[k] = fma(q[u], __shfl_sync(FULL, q[u], (lane + k) & 31), h[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 17; ++k) red[warp][k][lane] = h[k];
  __syncthreads();
  for (int e = threadIdx.x; e < 17 * 32; e += 128) {
    const int k = e >> 5, c = e & 31;
    w.epart[(size_t)blockIdx.x * 17 * 32 + e] = (red[0][k][c] + red[1][k][c]) + (red[2][k][c] + red[3][k][c]);
  }
}

// Pass 2: block k adds folded row k of the partials over the pass-1 blocks (fixed order) and
// writes F, the float-float F and the guard, as kg_e_kernel does.
__global__ void __launch_bounds__(128) kg_ered_kernel(int nblk, int R, KgWork w) {
  __shared__ double red[4][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x;
  pdl_wait();
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b0 = warp; b0 < nblk; b0 += 64) {
    double x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int b = b0 + 4 * u;
      x[u] = (b < nblk) ? w.epart[(size_t)b * 17 * 32 + k * 32 + lane] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) a[u & 3] += x[u];
  }
  red[warp][lane] = (a[0] + a[1]) + (a[2] + a[3]);
  __syncthreads();
  if (warp == 0) {
    const double sum = (red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane]);
    const int c = lane, d = (lane + k) & 31, i = min(c, d), j = max(c, d);
    if (j < R) {
      const double e = (i == j) ? sum - 1.0 : sum;
      const double f = (i == j) ? 0.5 * e : e;
      w.F[i * KG_MAXR + j] = f;
      w.Ff[i * KG_MAXR + j] = ff_st(ff_from_bits(f));
      if (!(fabs(e) <= kEMax)) atomicOr(w.flag, (fabs(e) <= kE2Max) ? 1 : 3);  // NaN: 3
    }
  }
}

// E, F and the guard for M rows: the one-warp-per-entry kernel up to 1024 rows, the two passes
// above beyond.  *n: kernels launched.
cudaError_t launch_e(int M, int R, const KgWork& w, cudaStream_t st, int* n) {
  if (M <= 1024) {
    *n = 1;
    const int npair = R * (R + 1) / 2;
    return launch_pdl(kg_e_kernel, dim3((npair + 3) / 4), dim3(128), 0, st, M, R, w);
  }
  *n = 2;
  cudaError_t e = launch_pdl(kg_epart_kernel, dim3(KG_EBLK), dim3(128), 0, st, M, R, w);
  if (e != cudaSuccess) return e;
  return launch_pdl(kg_ered_kernel, dim3(17), dim3(128), 0, st, (int)KG_EBLK, R, w);
}

// Q0 = Q1 (I - F) (one row per warp, lane = column: q0[c] = q1[c] - sum_{k <= c} q1[k] F[k][c]),
// and, on the first R warps of the grid, row c of R0 = (I + F) R1.  Optional copies: Q0f
// (FP32) and Qt, Q0^T split into bf16 hi / lo for the tensor cores (Qt[2][Rp][Kp], the layout
// the Householder finish writes).  The correction sum runs in float-float on the FP32 pipe:
// every |F[k][c]| <= 1e-8 once the guard accepts, so the sum is below 3.2e-7 and its ~2^-46
// relative error below 1e-20, far under the FP64 rounding of q1; only q1 - sum is FP64.
__global__ void __launch_bounds__(128) kg_q0_kernel(int M, int R, KgWork w, double* __restrict__ Q0,
                                                     float* __restrict__ Q0f, double* __restrict__ R0,
                                                     __nv_bfloat16* __restrict__ Qt, int Rp, int64_t Kp) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * 4 + (threadIdx.x >> 5);
  pdl_wait();
  if (t >= M) return;
  ffn fcol[KG_MAXR];  // F[k][lane], k <= lane
#pragma unroll
  for (int k = 0; k < KG_MAXR; ++k)
    fcol[k] = (k < R && lane >= k && lane < R) ? ff_ld(w.Ff[k * KG_MAXR + lane]) : ff_make(0.0f, 0.0f);
  if (t < R) {
    // R0[t][d] = R1[t][d] + sum_{t <= k <= d} F[t][k] R1[k][d], d = lane
    double r = (lane < R) ? w.R1[t * KG_MAXR + lane] : 0.0;
    double rcol[KG_MAXR], frow[KG_MAXR];
#pragma unroll
    for (int k = 0; k < KG_MAXR; ++k) {
      rcol[k] = (k < R && lane >= k && lane < R) ? w.R1[k * KG_MAXR + lane] : 0.0;
      frow[k] = (k < R && k >= t) ? w.F[t * KG_MAXR + k] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < KG_MAXR; ++k) r = fma(frow[k], rcol[k], r);
    if (lane < R) R0[t * R + lane] = (lane >= t) ? r : 0.0;
  }
  const double q1 = (lane < R) ? w.Q1[(size_t)t * R + lane] : 0.0;
  const ffn q1f = ff_from_bits(q1);
  ffn acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = ff_make(0.0f, 0.0f);
#pragma unroll
  for (int k = 0; k < KG_MAXR; ++k) {
    if (k < R) acc[k & 3] = ff_fms(acc[k & 3], ff_neg(ff_shfl(q1f, k)), fcol[k]);
  }
  const double q = q1 - ff_val(ff_add(ff_add(acc[0], acc[1]), ff_add(acc[2], acc[3])));
  if (lane < R) {
    Q0[(size_t)t * R + lane] = q;
    if (Q0f) Q0f[(size_t)t * R + lane] = (float)q;
    if (Qt) {
      const float q32 = (float)q;
      const __nv_bfloat16 h = __float2bfloat16_rn(q32);
      const size_t e = (size_t)lane * Kp + t;
      Qt[e] = h;
      Qt[(size_t)Rp * Kp + e] = __float2bfloat16_rn(q32 - __bfloat162float(h));
    }
  }
}

// the 16-CTA cluster needs the non-portable size allowed, once per device
cudaError_t kg_cluster_attributes() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (done[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fg_chol_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  done[dev] = true;
  return cudaSuccess;
}

}  // namespace

size_t factor_gram_work_doubles(int64_t Imax, int R) { return kg_work_doubles(Imax, R); }
int* gram_fallback_counter(double* gram_work) { return reinterpret_cast<int*>(gram_work) + 1; }
int* gram_second_pass_counter(double* gram_work) { return reinterpret_cast<int*>(gram_work) + 2; }

cudaError_t launch_tri_gram(const double* T, int R, float2* Gf, double* s, cudaStream_t st) {
  if (R < 1 || R > KG_MAXR) return cudaErrorInvalidValue;
  TriPtrs t{};
  t.p[0] = T;
  tri_gram_kernel<<<1, 256, 0, st>>>(t, R, Gf, s);
  return cudaGetLastError();
}

size_t krp_gram_work_doubles(int R) { return kg_work_doubles((int64_t)R * R, R); }

cudaError_t launch_krp_chol(const GramPtrs& gp, int m, int R, double* gram_work, cudaStream_t st, int acc,
                            const int* flag_in) {
  if (R < 1 || R > KG_MAXR || m < 2 || m > KG_MAXM) return cudaErrorInvalidValue;
  const KgWork w = kg_views(gram_work, R, (int64_t)R * R);
  return launch_pdl(kg_chol_kernel, dim3(1), dim3(256), 0, st, gp, m, R, acc, flag_in, w);
}

int* gram_flag(double* gram_work) { return reinterpret_cast<int*>(gram_work); }

// The rows of a Gram-route QR of a two-triangle product (R^2 rows) after its Cholesky: Q1, E and
// the guard, then Q (and Qf) and the triangle Rt.  *n: kernels launched.
static cudaError_t krp_rows_only(const double* Ra, const double* Rb, int R, const KgWork& w, double* Q, float* Qf,
                                 double* Rt, cudaStream_t st, int* n) {
  const int M = R * R;
  TriPtrs t{};
  t.p[0] = Ra;
  t.p[1] = Rb;
  cudaError_t e = launch_pdl(kg_q1_kernel, dim3((M + 3) / 4), dim3(128), 0, st, t, 2, M, R, w);
  if (e != cudaSuccess) return e;
  int ne = 0;
  e = launch_e(M, R, w, st, &ne);
  if (e != cudaSuccess) return e;
  *n = 2 + ne;
  return launch_pdl(kg_q0_kernel, dim3((M + 3) / 4), dim3(128), 0, st, M, R, w, Q, Qf, Rt, (__nv_bfloat16*)nullptr, 0,
                    (int64_t)0);
}

cudaError_t launch_krp_rows(const ZPlan& plan2, TriPtrs tri, int m, const GramPtrs& gp, double* Q0, double* R0,
                            double* gram_work, double* qr_work, unsigned int* dev_status, cudaStream_t st,
                            float* Q0f, int* nlaunch, bool fallback) {
  const int R = plan2.R;
  if (plan2.m != 2 || R < 1 || R > KG_MAXR || m < 2 || m > KG_MAXM) return cudaErrorInvalidValue;
  const KgWork w = kg_views(gram_work, R, (int64_t)R * R);
  int launches = 0, n = 0;
  cudaError_t e;
  if (m == 2) {
    e = krp_rows_only(tri.p[0], tri.p[1], R, w, Q0, Q0f, R0, st, &n);
    if (e != cudaSuccess) return e;
    launches += n;
    if (!fallback) {
      if (nlaunch) *nlaunch = launches;
      return cudaSuccess;
    }
    // the second Cholesky pass or the Householder staircase QR, which return at once unless the
    // flag was raised
    const CholQr2Src c2{w.F, w.Q1, w.R1};
    e = launch_krp_qr(plan2, tri, Q0, R0, qr_work, dev_status, st, Q0f, w.flag, &c2);
    if (nlaunch) *nlaunch = launches + 1;
    return e;
  }
  // nested: level 2, R_{m-1} (.) R_m = Q_W S (its Cholesky issued by the caller); level d = 3..m,
  // R_{m-d} (.) S = Q_Y S' with the Gram of S the Hadamard product of the later triangles' Grams
  // (S^T S is the previous level's Gram), and Q_W <- (I (x) Q_W) Q_Y; the guard accumulates over
  // the levels, and the nested Householder QR recomputes everything if it tripped
  const NestedBufs nb = nested_views(qr_work, m, R);
  e = krp_rows_only(tri.p[m - 2], tri.p[m - 1], R, w, nb.QW[0], nullptr, nb.S[0], st, &n);
  if (e != cudaSuccess) return e;
  launches += n;
  int cur = 0;
  int64_t mw = (int64_t)R * R;
  for (int d = 3; d <= m; ++d) {
    const bool last = (d == m);
    GramPtrs gd{};
    for (int k = 0; k < d; ++k) {
      gd.g[k] = gp.g[m - d + k];
      gd.s[k] = gp.s[m - d + k];
    }
    e = launch_krp_chol(gd, d, R, gram_work, st, 1);
    if (e != cudaSuccess) return e;
    e = krp_rows_only(tri.p[m - d], nb.S[(d - 3) & 1], R, w, nb.QY, nullptr, last ? R0 : nb.S[(d - 2) & 1], st, &n);
    if (e != cudaSuccess) return e;
    e = launch_krp_assemble(nb.QW[cur], mw, nb.QY, R, last ? Q0 : nb.QW[cur ^ 1], last ? Q0f : nullptr, st);
    if (e != cudaSuccess) return e;
    launches += n + 2;
    cur ^= 1;
    mw *= R;
  }
  if (!fallback) {
    if (nlaunch) *nlaunch = launches;
    return cudaSuccess;
  }
  int nf = 0;
  e = launch_krp_qr_nested(plan2, tri, m, Q0, R0, qr_work, dev_status, st, Q0f, &nf, w.flag);
  if (nlaunch) *nlaunch = launches + nf;
  return e;
}

// Z = R_1 (.) ... (.) R_m with rows (l, i, t): l over the triangles before s, i over R_s, t over
// those after.  With W = R_1 (.) .. R_(s-1) (.) R_(s+1) .. (.) R_m = Q_W S_W (rows w = (l, t)),
// Z[(l, i, t), c] = R_s[i, c] W[(l, t), c] = sum_j Q_W[(l, t), j] R_s[i, c] S_W[j, c], so with
// Y = R_s (.) S_W = Q_Y R_Y (rows (i, j)), Z = P (I_R (x) Q_W) Q_Y R_Y for the row permutation P
// of (i, (l, t)) to (l, i, t): Q0 = P (I (x) Q_W) Q_Y, orthonormal, and R0 = R_Y, positive diagonal.
cudaError_t launch_krp_rows_split(const ZPlan& plan2, TriPtrs tri, int m, int s, const double* QW, const double* SW,
                                  double* Q0, double* R0, double* gram_work, double* qr_work,
                                  unsigned int* dev_status, cudaStream_t st, float* Q0f, int* nlaunch) {
  const int R = plan2.R;
  if (plan2.m != 2 || R < 1 || R > KG_MAXR || m < 3 || m > KG_MAXM || s < 0 || s >= m) return cudaErrorInvalidValue;
  const KgWork w = kg_views(gram_work, R, (int64_t)R * R);
  const NestedBufs nb = nested_views(qr_work, m, R);
  int n = 0;
  cudaError_t e = krp_rows_only(tri.p[s], SW, R, w, nb.QY, nullptr, R0, st, &n);
  if (e != cudaSuccess) return e;
  int64_t L = 1, T = 1;
  for (int k = 0; k < s; ++k) L *= R;
  for (int k = s + 1; k < m; ++k) T *= R;
  e = launch_krp_assemble_tri(QW, L, T, nb.QY, R, Q0, Q0f, st);
  if (e != cudaSuccess) return e;
  int nf = 0;
  e = launch_krp_qr_nested(plan2, tri, m, Q0, R0, qr_work, dev_status, st, Q0f, &nf, w.flag);
  if (nlaunch) *nlaunch = n + 1 + nf;
  return e;
}

cudaError_t launch_krp_qr_gram(const ZPlan& plan2, TriPtrs tri, int m, double* Q0, double* R0, double* gram_work,
                               double* qr_work, unsigned int* dev_status, cudaStream_t st, float* Q0f) {
  const int R = plan2.R;
  if (plan2.m != 2 || R < 1 || R > KG_MAXR || m < 2 || m > KG_MAXM) return cudaErrorInvalidValue;
  const KgWork w = kg_views(gram_work, R, (int64_t)R * R);
  GramPtrs gp{};
  for (int k = 0; k < m; ++k) {
    cudaError_t e = launch_tri_gram(tri.p[k], R, w.g[k], w.s[k], st);
    if (e != cudaSuccess) return e;
    gp.g[k] = w.g[k];
    gp.s[k] = w.s[k];
  }
  GramPtrs g2{};  // level 2 (or the whole product for m = 2): the last two triangles
  g2.g[0] = gp.g[m - 2];
  g2.s[0] = gp.s[m - 2];
  g2.g[1] = gp.g[m - 1];
  g2.s[1] = gp.s[m - 1];
  cudaError_t e = launch_krp_chol(g2, 2, R, gram_work, st, 0);
  if (e != cudaSuccess) return e;
  return launch_krp_rows(plan2, tri, m, gp, Q0, R0, gram_work, qr_work, dev_status, st, Q0f, nullptr);
}

cudaError_t launch_finish_gram_chol(const double* hpart, const double* fitpart, int nblk, int64_t I, int R,
                                    FinishOut out, double* gram_work, float2* gram_out, double* colnorm_out,
                                    cudaStream_t st) {
  if (I < 1 || I > (int64_t(1) << 30) || R < 1 || R > KG_MAXR || nblk < 1) return cudaErrorInvalidValue;
  if ((gram_out == nullptr) != (colnorm_out == nullptr)) return cudaErrorInvalidValue;
  const KgWork w = kg_views(gram_work, R, I);
  cudaError_t e = kg_cluster_attributes();
  if (e != cudaSuccess) return e;
  fg_chol_kernel<<<KG_CL, 256, 0, st>>>(hpart, nblk, R, fitpart, out.lambda, out.fit_terms, gram_out, colnorm_out, w);
  return cudaGetLastError();
}

cudaError_t launch_finish_gram_rows(const double* Ahat, const double* fitpart, int nblk, int64_t I, int R,
                                    FinishOut out, double* gram_work, double* qr_work, unsigned int* dev_status,
                                    cudaStream_t st) {
  if (I < 1 || I > (int64_t(1) << 30) || R < 1 || R > KG_MAXR || nblk < 1) return cudaErrorInvalidValue;
  const int M = (int)I;
  const KgWork w = kg_views(gram_work, R, M);
  cudaError_t e = launch_pdl(fg_q1_kernel, dim3((M + 3) / 4), dim3(128), 0, st, Ahat, M, R, w, out.A);
  if (e != cudaSuccess) return e;
  int ne = 0;
  e = launch_e(M, R, w, st, &ne);
  if (e != cudaSuccess) return e;
  e = launch_pdl(kg_q0_kernel, dim3((M + 3) / 4), dim3(128), 0, st, M, R, w, out.Q, out.Qf, out.Rn, out.Qt, out.Rp,
                 out.Kp);
  if (e != cudaSuccess) return e;
  // the second Cholesky pass or the Householder finish, which return at once unless the flag was
  // raised
  const CholQr2Src c2{w.F, w.Q1, w.R1};
  return launch_mode_finish(Ahat, fitpart, nblk, I, R, out, qr_work, dev_status, st, w.flag, &c2);
}

cudaError_t launch_finish_gram(const double* Ahat, const double* hpart, const double* fitpart, int nblk, int64_t I,
                               int R, FinishOut out, double* gram_work, double* qr_work, unsigned int* dev_status,
                               cudaStream_t st) {
  cudaError_t e = launch_finish_gram_chol(hpart, fitpart, nblk, I, R, out, gram_work, nullptr, nullptr, st);
  if (e != cudaSuccess) return e;
  return launch_finish_gram_rows(Ahat, fitpart, nblk, I, R, out, gram_work, qr_work, dev_status, st);
}

}  // namespace cpqr
