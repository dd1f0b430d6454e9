// FP64 Householder QRs of tall, skinny matrices (R <= 32 columns) on one
// thread-block cluster, for the three QRs of a CP-ALS-QR mode update:
//  * the factor QR A^(n) = Q_n R_n (Alg. 2 line 10), preceded by the
//    extrapolated right-hand side V^ = (1+beta) V0 - alpha beta V1 (eq. 19),
//    the solve A^ R0^T = V^ (line 8) and the column normalisation (line 9);
//  * the QR of the Khatri-Rao product Z_n = R_{k1} (.) ... (.) R_{km} of the
//    other factors' triangles (lines 3-4);
//  * a plain QR (initial factors).
//
// GB300 has ~8 GFLOP/s of FP64 per SM, so these run on one thread-block
// cluster of 16 CTAs (8 where 16 cannot be scheduled) that own the rows
// round-robin; every row stays with one warp from start to end.  The 32
// Householder columns form a serial chain, so the kernel is built around the
// latency of one column:
//  * one exchange per column: every CTA reduces x_j^T a_c over its rows for
//    all c (c >= j gives the norm and the reflector products, c < j gives the
//    entries v_c^T v_j of V^T V for the compact-WY form at no extra cost) and
//    stores the sums into every peer's shared memory with st.async, which
//    completes the bytes on the peer's mbarrier: no cluster barrier, and the
//    pivot row, pushed by its owner, also gives the top block of V;
//  * the reflector of column j-1 is applied row by row in the same pass that
//    forms the products of column j;
//  * the norm uses the 53-bit rsqrt.approx.f64 and the reflector scale a
//    reciprocal from rcp.approx.f64 refined by two Newton-Raphson steps.
// Q is formed with the compact-WY (UT) representation: Q = E - V T V_top^T with
// T^{-1} = striu(V^T V) + diag(V^T V)/2; the columns of W2 = T V_top^T are
// back-substituted by different CTAs and all-gathered with st.async.
//
// Khatri-Rao rows are processed sorted by the largest index among their
// digits: a row whose digits are <= m is zero in columns < m because every
// R_k is upper triangular, so column j's reflector only touches the first
// (j+1)^m sorted rows and no fill-in escapes that staircase.
#include <cooperative_groups.h>

#include <cstdlib>

#include "common.cuh"
#include "ff.cuh"
#include "tc_common.cuh"

namespace cg = cooperative_groups;


namespace cpqr {

namespace {

using tc::smem_u32;

constexpr int NT = kQrThreads;
constexpr int NW = NT / 32;
constexpr int MAXCL = 16;
constexpr int PSLOT = 2 * CPQR_MAXR + 2;  // partial-sum slots of the finish prologue exchange
constexpr int RR = CPQR_MAXR * CPQR_MAXR;
constexpr int W2LD = CPQR_MAXR + 2;       // row stride of W2T (16-byte aligned rows, few bank conflicts)
constexpr unsigned FULL = 0xffffffffu;

enum { MODE_PLAIN = 0, MODE_KRP = 1, MODE_FINISH = 2 };

struct QrParams {
  int mode;
  int M;
  int R;
  // rows: smem if use_smem, else global work (M x R)
  int use_smem;
  double* work;
  int32_t act[CPQR_MAXR];
  // MODE_PLAIN
  const double* A_in;
  // MODE_KRP
  const int32_t* perm;
  int krp_m;
  TriPtrs tri;
  // MODE_FINISH
  const double* Ahat;      // I x R rows of A^ = V^ R0^{-T} (finish_prep_kernel)
  const double* fitpart;   // nfit x 2 per-block partial fit terms (finish_prep_kernel)
  int nfit;
  FinishOut fin;
  // outputs
  double* Q;
  float* Qf;  // FP32 copy of Q (may be null)
  double* Rout;
  unsigned int* status;
  int* run_if;  // when set: the QR runs only if run_if[0] != 0 (a guarded fallback) and counts
                // its runs in run_if[1]
  // the guarded QR's first Cholesky pass (optional): with run_if[0] == 1 a second pass finishes
  // the QR (counted in run_if[2]) and the Householder QR runs only if its Cholesky fails
  const double* c2F;   // F = striu(E) + diag(E) / 2, E = Q1^T Q1 - I (row stride CPQR_MAXR)
  const double* c2Q1;  // M x R, row stride R
  const double* c2R1;  // R x R upper, row stride CPQR_MAXR
};

struct SmemLayout {
  alignas(16) double cbox[2][MAXCL][CPQR_MAXR];  // per-column sums of every CTA (st.async, 2 buffers)
  alignas(16) double pbox[2][CPQR_MAXR];         // pivot row of the column (st.async by its owner)
  alignas(16) double W2T[CPQR_MAXR][W2LD];       // W2T[c][a] = (T V_top^T)[a][c] (st.async all-gather)
  unsigned long long bar[3];                     // mbarriers: cbox/pbox buffer 0, 1; W2T
  int abort_flag;
  int pad_;
  double inbox1[MAXCL][PSLOT];  // finish prologue: partial sums pushed by every CTA (cluster barrier)
  double red[NW][PSLOT];        // per-warp partial sums
  double pivloc[CPQR_MAXR];     // pivot row as seen by the owning warp
  double dvec[CPQR_MAXR];       // cluster-wide x_j^T a_c of the current column
  double bcw[CPQR_MAXR];        // tau (x_j^T a_c - alpha a_jc): reflector product per column
  double alpha[CPQR_MAXR];
  double tau[CPQR_MAXR];
  double vpiv[CPQR_MAXR];
  // ST[b][a] = v_a^T v_b (a < b) in [0, RR), VT[c][a] = v_a[c] (a <= c, top block of V) in
  // [RR, 2 RR); before the Householder columns: the Khatri-Rao triangles (up to 3 RR doubles)
  double big[3 * RR];
};

// Row t's lowest column with a nonzero reflector entry (staircase) for KRP mode.
__device__ __forceinline__ int row_alo(const QrParams& p, int t) {
  if (p.mode != MODE_KRP) return 0;
  int a = 0;
  while (a < p.R - 1 && p.act[a] <= t) ++a;
  return a;
}

// Entry (orig, c) of Z = R_{k1} (.) ... (.) R_{km}; orig = digits (r_1 .. r_m) base R, r_m
// fastest; tri = the m triangles back to back (R x R each) in shared memory, or null (global).
__device__ __forceinline__ double krp_value(const QrParams& p, const double* tri, int orig, int c) {
  double v = 1.0;
  int x = orig;
  const int RR2 = p.R * p.R;
  for (int k = p.krp_m - 1; k >= 0; --k) {
    int r = x % p.R;
    x /= p.R;
    v *= tri ? tri[k * RR2 + r * p.R + c] : p.tri.p[k][r * p.R + c];
  }
  return v;
}

__device__ __forceinline__ double tree8(const double* v, int stride) {
  return ((v[0] + v[stride]) + (v[2 * stride] + v[3 * stride])) +
         ((v[4 * stride] + v[5 * stride]) + (v[6 * stride] + v[7 * stride]));
}

// Householder scalars of a column with squared norm s and pivot entry xj:
// alpha = -sign(xj) sqrt(s), tau = 2 / ||v||^2 = 1 / (s - alpha xj).  Inside the normal range
// the square root comes from rsqrt.approx.f64 (measured to 53 bits on sm_103) and the reciprocal
// from rcp.approx.ftz.f64 (about 20 bits) refined by two Newton-Raphson steps
// z <- z + z (1 - d z), each squaring the relative error; outside it the IEEE operations.  The
// range and sign tests are integer tests on the bit patterns: FP64 compares would sit on the
// column's critical path at FP64 latency.
__device__ __forceinline__ void house_scalars(double s, double xj, double& alpha, double& tau) {
  const long long sb = __double_as_longlong(s), xb = __double_as_longlong(xj);
  const bool xpos = (xb >= 0) || (xb == (long long)0x8000000000000000ull);  // xj >= 0, including -0
  alpha = 0.0;
  tau = 0.0;
  if (sb <= 0) return;  // s == 0 (a zero column); s is a sum of squares, so never negative
  // [1e-280, 1e280]: s * (1 + |xj| / sqrt(s)) <= 2 s stays normal for the reciprocal
  constexpr long long kLo = 0x05CD0B15A491EB84LL;  // bit pattern of 1e-280
  constexpr long long kHi = 0x7A11A0FC668AAC70LL;  // bit pattern of 1e280
  if (sb > kLo && sb < kHi) {
    double y;
    asm("rsqrt.approx.f64 %0, %1;" : "=d"(y) : "d"(s));
    const double nx = s * y;
    alpha = xpos ? -nx : nx;
    const double d = fma(-alpha, xj, s);
    double z;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(z) : "d"(d));
    z = fma(z, fma(-d, z, 1.0), z);
    tau = fma(z, fma(-d, z, 1.0), z);
  } else {
    const double nx = sqrt(s);
    alpha = xpos ? -nx : nx;
    tau = 1.0 / (s - alpha * xj);
  }
}

// Second Cholesky pass of a guarded Gram-route QR (CholeskyQR2), on the whole cluster; returns
// false (every CTA alike) when it does not converge, and the caller then runs the Householder QR.
// With E = Q1^T Q1 - I (max |E| <= 1e-3) and F = striu(E) + diag(E) / 2, the second Cholesky
// factor is chol(I + E) = I + D with D upper triangular and D + D^T + D^T D = E, i.e. the fixed
// point of D = F - up(D^T D), up(S) = striu(S) + diag(S) / 2 (a contraction by ~2 ||D||).  Its
// inverse is I + X with X = -D - D X (a contraction by ~||D||).  Both iterations run on small
// quantities only, in float-float on CTA 0 (~2^-48 relative of entries below 5e-4), until no
// entry moves by more than 1e-17; then R = (I + D) R1 = R1 + D R1 and every row of
// Q = Q1 (I + X) = Q1 + Q1 X take one FP64 addition each (as the first pass's correction does):
// GB300's FP64 pipe is ~64 times slower than FP32, so an FP64 Cholesky and substitution here would
// cost tens of microseconds.  Q R = Q1 R1 = the input, and Q^T Q = (I + D)^{-T} (I + E) (I + D)^{-1}
// = I, both to the rounding of the final additions.  Every CTA copies X out of CTA 0's shared
// memory and forms its rows t = rank + CL u, written where the Householder QR would write them
// (with the FP32 copy and the tensor cores' hi / lo staging).  scr: 4 x 32 x 33 float2 + a flag of
// this CTA's shared memory (the rows region, unused until the Householder prologue, which follows
// a cluster barrier).
template <int CL>
__device__ bool second_pass(const QrParams& p, cg::cluster_group& cluster, int rank, double* scr) {
  using namespace ffa;
  constexpr int LD = CPQR_MAXR + 1;
  constexpr int RR32 = CPQR_MAXR * CPQR_MAXR;
  constexpr int EPT = RR32 / NT;  // entries per thread
  constexpr float kMove = 1e-17f;
  constexpr int kIters = 16;
  float2 (*Dm)[LD] = reinterpret_cast<float2 (*)[LD]>(scr);
  float2 (*Fm)[LD] = Dm + CPQR_MAXR;
  float2 (*Xm)[LD] = Fm + CPQR_MAXR;
  float2 (*Tm)[LD] = Xm + CPQR_MAXR;  // R1 in float-float
  int* okp = reinterpret_cast<int*>(Tm + CPQR_MAXR);
  const int tid = threadIdx.x, lane = tid & 31, R = p.R;
  const ffn zero = ff_make(0.0f, 0.0f);
  if (rank == 0) {
    for (int e = tid; e < RR32; e += NT) {
      const int i = e / CPQR_MAXR, j = e % CPQR_MAXR;
      const bool up = (i <= j && j < R);
      const float2 f = up ? ff_st(ff_from_bits(p.c2F[i * CPQR_MAXR + j])) : make_float2(0.0f, 0.0f);
      Fm[i][j] = f;
      Dm[i][j] = f;
      Tm[i][j] = up ? ff_st(ff_from_bits(p.c2R1[i * CPQR_MAXR + j])) : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    // D = F - up(D^T D), (D^T D)[i][j] = sum_{k <= i} D[k][i] D[k][j]
    bool conv = false;
    for (int it = 0; it < kIters && !conv; ++it) {
      ffn nv[EPT];
      int moved = 0;
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = tid + q * NT, i = e / CPQR_MAXR, j = e % CPQR_MAXR;
        nv[q] = zero;
        if (i <= j && j < R) {
          ffn s = zero;
          for (int k = 0; k <= i; ++k) s = ff_fms(s, ff_neg(ff_ld(Dm[k][i])), ff_ld(Dm[k][j]));
          if (i == j) s = ff_make(0.5f * s.hi, 0.5f * s.lo);
          nv[q] = ff_add(ff_ld(Fm[i][j]), ff_neg(s));
          if (!(fabsf(ff_add(nv[q], ff_neg(ff_ld(Dm[i][j]))).hi) <= kMove)) moved = 1;  // NaN moves
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = tid + q * NT, i = e / CPQR_MAXR, j = e % CPQR_MAXR;
        if (i <= j && j < R) Dm[i][j] = ff_st(nv[q]);
      }
      conv = (__syncthreads_or(moved) == 0);
    }
    // X = -D - D X, (D X)[i][j] = sum_{i <= k <= j} D[i][k] X[k][j]; X_0 = -D
    bool convx = false;
    if (conv) {
      for (int e = tid; e < RR32; e += NT) {
        const int i = e / CPQR_MAXR, j = e % CPQR_MAXR;
        Xm[i][j] = (i <= j && j < R) ? ff_st(ff_neg(ff_ld(Dm[i][j]))) : make_float2(0.0f, 0.0f);
      }
      __syncthreads();
      for (int it = 0; it < kIters && !convx; ++it) {
        ffn nv[EPT];
        int moved = 0;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          const int e = tid + q * NT, i = e / CPQR_MAXR, j = e % CPQR_MAXR;
          nv[q] = zero;
          if (i <= j && j < R) {
            ffn s = ff_ld(Dm[i][j]);
            for (int k = i; k <= j; ++k) s = ff_fms(s, ff_neg(ff_ld(Dm[i][k])), ff_ld(Xm[k][j]));
            nv[q] = ff_neg(s);
            if (!(fabsf(ff_add(nv[q], ff_neg(ff_ld(Xm[i][j]))).hi) <= kMove)) moved = 1;
          }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          const int e = tid + q * NT, i = e / CPQR_MAXR, j = e % CPQR_MAXR;
          if (i <= j && j < R) Xm[i][j] = ff_st(nv[q]);
        }
        convx = (__syncthreads_or(moved) == 0);
      }
    }
    if (convx) {
      // R = R1 + D R1, (D R1)[i][j] = sum_{i <= k <= j} D[i][k] R1[k][j]
      for (int e = tid; e < RR32; e += NT) {
        const int i = e / CPQR_MAXR, j = e % CPQR_MAXR;
        if (i < R && j < R) {
          double r = 0.0;
          if (i <= j) {
            ffn s = zero;
            for (int k = i; k <= j; ++k) s = ff_fms(s, ff_neg(ff_ld(Dm[i][k])), ff_ld(Tm[k][j]));
            r = p.c2R1[i * CPQR_MAXR + j] + ff_val(s);
          }
          p.Rout[i * R + j] = r;
        }
      }
      if (tid == 0) atomicAdd(p.run_if + 2, 1);
    }
    if (tid == 0) *okp = convx ? 1 : 0;
  }
  cluster.sync();
  float2 (*X0)[LD] = cluster.map_shared_rank(Xm, 0);
  // not converged: every CTA goes on to the Householder QR, whose prologue writes this shared
  // memory only after its first cluster barrier
  if (*cluster.map_shared_rank(okp, 0) == 0) return false;
  if (rank != 0) {
    for (int e = tid; e < CPQR_MAXR * LD; e += NT) Xm[e / LD][e % LD] = X0[e / LD][e % LD];
    __syncthreads();
  }
  cluster.sync();  // no CTA reads CTA 0's copy any more
  const int M = p.M;
  const int L = (M > rank) ? (M - rank + CL - 1) / CL : 0;
  ffn xcol[CPQR_MAXR];  // X[k][lane], k <= lane
#pragma unroll
  for (int k = 0; k < CPQR_MAXR; ++k) xcol[k] = (k <= lane && lane < R) ? ff_ld(Xm[k][lane]) : zero;
  for (int u = (int)(threadIdx.x >> 5); u < L; u += NW) {
    const int t = rank + CL * u;
    const double q1 = (lane < R) ? p.c2Q1[(size_t)t * R + lane] : 0.0;
    const ffn qf = ff_from_bits(q1);
    ffn acc[4] = {zero, zero, zero, zero};
#pragma unroll
    for (int k = 0; k < CPQR_MAXR; ++k)
      if (k < R) acc[k & 3] = ff_fms(acc[k & 3], ff_neg(ff_shfl(qf, k)), xcol[k]);
    const double q = q1 + ff_val(ff_add(ff_add(acc[0], acc[1]), ff_add(acc[2], acc[3])));
    if (lane < R) {
      p.Q[(size_t)t * R + lane] = q;
      if (p.Qf) p.Qf[(size_t)t * R + lane] = (float)q;
      if (p.mode == MODE_FINISH && p.fin.Qt) {
        const float q32 = (float)q;
        const __nv_bfloat16 h = __float2bfloat16_rn(q32);
        const size_t e = (size_t)lane * p.fin.Kp + t;
        p.fin.Qt[e] = h;
        p.fin.Qt[(size_t)p.fin.Rp * p.fin.Kp + e] = __float2bfloat16_rn(q32 - __bfloat162float(h));
      }
    }
  }
  return true;
}

// Named barrier for warps 0..3 (128 threads).
__device__ __forceinline__ void sync_warps0to3() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

template <int CL>
__global__ void __launch_bounds__(NT, 1) qr_cluster_kernel(QrParams p) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = p.R;
  const int M = p.M;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SmemLayout& sm = *reinterpret_cast<SmemLayout*>(smem_raw);
  double* rows_smem = reinterpret_cast<double*>(smem_raw + ((sizeof(SmemLayout) + 15) / 16) * 16);
  // bytes that complete one column exchange on each CTA: CL partial-sum vectors + the pivot row
  constexpr uint32_t kColBytes = (uint32_t)((CL + 1) * CPQR_MAXR * sizeof(double));
  const uint32_t kW2Bytes = (uint32_t)(R * CPQR_MAXR * sizeof(double));

  const int L = (M > rank) ? (M - rank + CL - 1) / CL : 0;  // local rows: t = rank + CL * u
  double* Wb;
  int ldw;
  if (p.use_smem) {
    Wb = rows_smem;
    ldw = R;
  } else {
    Wb = p.work + (size_t)rank * R;
    ldw = CL * R;
  }
  auto W = [&](int u) -> double* { return Wb + (size_t)u * ldw; };
  auto grow = [&](int u) -> int { return rank + CL * u; };
  double (*ST)[CPQR_MAXR] = reinterpret_cast<double (*)[CPQR_MAXR]>(&sm.big[0]);
  double (*VT)[CPQR_MAXR] = reinterpret_cast<double (*)[CPQR_MAXR]>(&sm.big[RR]);

  if (p.run_if) {
    const int flag = *(volatile const int*)p.run_if;  // every CTA reads the same flag
    if (flag == 0) return;
    if (flag == 1 && p.c2F && second_pass<CL>(p, cluster, rank, rows_smem)) return;
    if (rank == 0 && tid == 0) atomicAdd(p.run_if + 1, 1);
  }
  // mbarriers of the st.async exchanges, armed for their first phase before any peer can send
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) tc::mbar_init(smem_u32(&sm.bar[b]), 1);
    tc::fence_mbar_init_cluster();
    tc::mbar_expect_tx(smem_u32(&sm.bar[0]), kColBytes);
    if (R > 1) tc::mbar_expect_tx(smem_u32(&sm.bar[1]), kColBytes);
    tc::mbar_expect_tx(smem_u32(&sm.bar[2]), kW2Bytes);
    sm.abort_flag = 0;
  }
  cluster.sync();

  // ---------------- prologue: fill the local rows ----------------
  if (p.mode == MODE_PLAIN) {
    for (int u = warp; u < L; u += NW)
      if (lane < R) W(u)[lane] = p.A_in[(size_t)grow(u) * R + lane];
  } else if (p.mode == MODE_KRP) {
    // The triangles are read R times each and the row permutation once per row: both go into
    // shared memory first with loads issued all at once (this QR runs beside HBM-bound TTMs,
    // where a chain of dependent global loads per row would pay the loaded memory latency).
    double* tri = nullptr;
    const int ntri = p.krp_m * R * R;
    int* sperm = nullptr;
    if (ntri * 8 + L * 4 <= 3 * RR * 8) {
      tri = sm.big;
      sperm = reinterpret_cast<int*>(sm.big + ntri);
      for (int e = tid; e < ntri; e += NT) tri[e] = p.tri.p[e / (R * R)][e % (R * R)];
      for (int u = tid; u < L; u += NT) sperm[u] = p.perm[grow(u)];
      __syncthreads();
    }
    for (int u = warp; u < L; u += NW)
      if (lane < R) W(u)[lane] = krp_value(p, tri, sperm ? sperm[u] : p.perm[grow(u)], lane);
  } else {
    // MODE_FINISH: rows of A^ (Alg. 2 line 8, solved by finish_prep_kernel), column norms
    // lambda_r = ||a^_r|| over the cluster and the normalisation A = A^ / lambda (line 9).
    double nrm = 0.0;
    for (int u = warp; u < L; u += NW) {
      const double a = (lane < R) ? p.Ahat[(size_t)grow(u) * R + lane] : 0.0;
      if (lane < R) W(u)[lane] = a;
      nrm = fma(a, a, nrm);
    }
    sm.red[warp][lane] = nrm;
    __syncthreads();
    if (warp == 0) {
      const double v = tree8(&sm.red[0][lane], PSLOT);
      for (int r = 0; r < CL; ++r) cluster.map_shared_rank(&sm.inbox1[rank][0], r)[lane] = v;
    }
    cluster.sync();
    if (warp == 0) {
      double s[MAXCL / 2];
#pragma unroll
      for (int h = 0; h < CL / 2; ++h) s[h] = sm.inbox1[2 * h][lane] + sm.inbox1[2 * h + 1][lane];
#pragma unroll
      for (int w = CL / 4; w >= 1; w >>= 1)
#pragma unroll
        for (int h = 0; h < w; ++h) s[h] += s[h + w];
      const double lam = sqrt(s[0]);
      if (lane < R) {
        sm.bcw[lane] = (lam > 0.0) ? 1.0 / lam : 0.0;
        if (lam == 0.0 && rank == 0) atomicOr(p.status, CPQR_DEV_SINGULAR);
        if (rank == 0) p.fin.lambda[lane] = lam;
      }
    }
    __syncthreads();
    for (int u = warp; u < L; u += NW) {
      if (lane < R) {
        double a = W(u)[lane] * sm.bcw[lane];
        W(u)[lane] = a;
        p.fin.A[(size_t)grow(u) * R + lane] = a;
      }
    }
  }
  __syncthreads();

  // ---------------- Householder columns: one st.async exchange per column ----------------
  // Step j applies reflector j-1 to the rows it touches and, in the same pass, accumulates
  // x_j^T a_c (x_j = column j after that update) over the rows [j, act[j]) for every c.
  for (int j = 0; j < R; ++j) {
    const int buf = j & 1;
    const int pj = j - 1;
    const bool upd = (j > 0);
    const int t_lo = upd ? pj : 0;
    const int t_hi = p.act[j];
    const int act_prev = upd ? p.act[pj] : 0;
    const double tw = upd ? sm.bcw[lane] : 0.0;  // zero outside pj < lane < R
    const double vpp = upd ? sm.vpiv[pj] : 0.0;
    const double alp = upd ? sm.alpha[pj] : 0.0;
    const int u0 = (t_lo <= rank) ? 0 : (t_lo - rank + CL - 1) / CL;
    const int u1 = (t_hi > rank) ? (t_hi - rank + CL - 1) / CL : 0;
    const int us = u0 + ((warp - (u0 % NW)) + NW) % NW;
    double acc = 0.0;
    for (int u = us; u < u1; u += NW) {
      double* w = W(u);
      const int t = grow(u);
      double a = (lane < R) ? w[lane] : 0.0;
      if (t < act_prev) {  // reflector j-1 touches this row
        const bool pivrow = (t == pj);
        const double v = pivrow ? vpp : w[pj];
        a = fma(-tw, v, a);
        if (lane > pj && lane < R) w[lane] = a;
        if (pivrow && lane == pj) w[lane] = alp;
      }
      if (t >= j) {
        const double x = __shfl_sync(FULL, a, j);
        acc = fma(x, a, acc);
        if (t == j) sm.pivloc[lane] = a;
      }
    }
    sm.red[warp][lane] = acc;
    __syncthreads();
    if (warp < 4) {
      // CTA sums of 8 columns per warp, stored into every CTA of the cluster
      const int slot = 8 * warp + (lane & 7), g = lane >> 3;
      double v = sm.red[2 * g][slot] + sm.red[2 * g + 1][slot];
      v += __shfl_xor_sync(FULL, v, 8);
      v += __shfl_xor_sync(FULL, v, 16);
      const int pr = lane & 3;
      const double lo = __shfl_sync(FULL, v, 2 * pr), hi = __shfl_sync(FULL, v, 2 * pr + 1);
      const uint32_t src = smem_u32(&sm.cbox[buf][rank][8 * warp + 2 * pr]);
      const uint32_t bar = smem_u32(&sm.bar[buf]);
      for (int r = lane >> 2; r < CL; r += 8) tc::st_async_v2(tc::mapa(src, r), lo, hi, tc::mapa(bar, r));
    } else if (warp == 4 && rank == j % CL) {
      // the pivot row, owned here
      const int pr = lane & 15;
      const double lo = sm.pivloc[2 * pr], hi = sm.pivloc[2 * pr + 1];
      const uint32_t src = smem_u32(&sm.pbox[buf][2 * pr]);
      const uint32_t bar = smem_u32(&sm.bar[buf]);
      for (int r = lane >> 4; r < CL; r += 2) tc::st_async_v2(tc::mapa(src, r), lo, hi, tc::mapa(bar, r));
    }
    if (warp < 4) {
      tc::mbar_wait_cluster(smem_u32(&sm.bar[buf]), (uint32_t)((j >> 1) & 1), &sm.abort_flag, p.status);
      // re-arm this buffer for column j + 2: its bytes can only come after this CTA's column j + 1
      // sums, which it sends after every read of this buffer
      if (tid == 0 && j + 2 < R) tc::mbar_expect_tx(smem_u32(&sm.bar[buf]), kColBytes);
      constexpr int IPG = CL / 4;  // partial vectors summed by each of the 4 lane groups
      const int slot = 8 * warp + (lane & 7), g = lane >> 3;
      double v = sm.cbox[buf][g * IPG][slot];
#pragma unroll
      for (int q = 1; q < IPG; ++q) v += sm.cbox[buf][g * IPG + q][slot];
      v += __shfl_xor_sync(FULL, v, 8);
      v += __shfl_xor_sync(FULL, v, 16);
      if (g == 0) sm.dvec[slot] = v;
      sync_warps0to3();
      if (warp == 0) {
        const double s = sm.dvec[j], xj = sm.pbox[buf][j];
        double alpha, tau;
        house_scalars(s, xj, alpha, tau);
        const double vp = xj - alpha;
        const double pl = sm.pbox[buf][lane];
        const double num = sm.dvec[lane] - alpha * pl;  // v_j^T a_lane (lane > j), v_lane^T v_j (lane < j)
        sm.bcw[lane] = (lane > j && lane < R) ? tau * num : 0.0;
        ST[j][lane] = (lane < j) ? num : 0.0;
        VT[j][lane] = (lane < j) ? pl : (lane == j ? vp : 0.0);
        if (lane == 0) {
          sm.alpha[j] = alpha;
          sm.tau[j] = tau;
          sm.vpiv[j] = vp;
          if (rank == 0 && tau == 0.0) atomicOr(p.status, CPQR_DEV_SINGULAR);
        }
      }
    }
    __syncthreads();
  }

  // ---------------- R factor (positive diagonal) ----------------
  for (int u = warp; u < L; u += NW) {
    int t = grow(u);
    if (t >= R) break;
    if (lane < R) {
      double sg = (sm.alpha[t] < 0.0) ? -1.0 : 1.0;
      double v = (lane < t) ? 0.0 : (lane == t ? sm.alpha[t] : W(u)[lane]);
      p.Rout[t * R + lane] = sg * v;
    }
  }

  // ---------------- W2 = T V_top^T: column cc by warp cc / CL of CTA cc % CL ----------------
  // Tinv W2 = V_top^T with Tinv = striu(S) + diag(S)/2 upper triangular and diag(S)/2 = 1/tau;
  // column cc has nonzeros in rows a <= cc, found by back substitution (lane = row).
  {
    const int cc = rank + CL * warp;
    if (cc < R) {
      double rhs = (lane <= cc) ? VT[cc][lane] : 0.0;
      double mine = 0.0;
      for (int a = cc; a >= 0; --a) {
        const double w = __shfl_sync(FULL, rhs, a) * sm.tau[a];
        if (lane == a) mine = w;
        if (lane < a) rhs = fma(-ST[a][lane], w, rhs);
      }
      const int pr = lane & 15;
      const double lo = __shfl_sync(FULL, mine, 2 * pr), hi = __shfl_sync(FULL, mine, 2 * pr + 1);
      const uint32_t src = smem_u32(&sm.W2T[cc][2 * pr]);
      const uint32_t bar = smem_u32(&sm.bar[2]);
      for (int r = lane >> 4; r < CL; r += 2) tc::st_async_v2(tc::mapa(src, r), lo, hi, tc::mapa(bar, r));
    }
  }
  tc::mbar_wait_cluster(smem_u32(&sm.bar[2]), 0u, &sm.abort_flag, p.status);

  // ---------------- Q rows: Q[t, c] = sign_c (delta_tc - sum_a v_a[t] W2[a][c]) ----------------
  // Khatri-Rao mode: the output row of each local row, staged once (V^T V and V_top are dead:
  // every column of W2 has arrived, so every warp of this CTA finished its back substitution)
  int* sperm = nullptr;
  if (p.mode == MODE_KRP && L * 4 <= 3 * RR * 8) {
    sperm = reinterpret_cast<int*>(sm.big);
    for (int u = tid; u < L; u += NT) sperm[u] = p.perm[grow(u)];
    __syncthreads();
  }
  {
    const int c = lane;
    double w2[CPQR_MAXR];
#pragma unroll
    for (int a = 0; a < CPQR_MAXR; ++a) w2[a] = (c < R) ? sm.W2T[c][a] : 0.0;
    const double sg = (c < R && sm.alpha[c] < 0.0) ? -1.0 : 1.0;
    for (int u = warp; u < L; u += NW) {
      const int t = grow(u);
      const double* w = W(u);
      const int alo = row_alo(p, t);
      const int ahi = (t < R - 1) ? t : R - 1;
      double q = (t == c) ? 1.0 : 0.0;
#pragma unroll
      for (int a = 0; a < CPQR_MAXR; ++a) {
        if (a >= alo && a <= ahi) {
          const double va = (a == t) ? sm.vpiv[a] : w[a];
          q = fma(-va, w2[a], q);
        }
      }
      q *= sg;
      if (c < R) {
        const size_t orow = (p.mode == MODE_KRP) ? (size_t)(sperm ? sperm[u] : p.perm[t]) : (size_t)t;
        p.Q[orow * R + c] = q;
        if (p.Qf) p.Qf[orow * R + c] = (float)q;
        if (p.mode == MODE_FINISH && p.fin.Qt) {
          // the tensor cores' B operand, as the separate staging would write it
          const float q32 = (float)q;
          const __nv_bfloat16 h = __float2bfloat16_rn(q32);
          const size_t e = (size_t)c * p.fin.Kp + orow;
          p.fin.Qt[e] = h;
          p.fin.Qt[(size_t)p.fin.Rp * p.fin.Kp + e] = __float2bfloat16_rn(q32 - __bfloat162float(h));
        }
      }
    }
  }
  if (p.mode == MODE_FINISH && rank == 0 && warp == 0) {
    // <V0, V^> and ||V^||^2: per-block partials of finish_prep_kernel, added in a fixed order
    double a = 0.0, b = 0.0;
    for (int k = lane; k < p.nfit; k += 32) {
      a += p.fitpart[2 * k];
      b += p.fitpart[2 * k + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(FULL, a, o);
      b += __shfl_xor_sync(FULL, b, o);
    }
    if (lane == 0) {
      p.fin.fit_terms[0] = a;
      p.fin.fit_terms[1] = b;
    }
  }
  // no CTA leaves while a peer may still store into its shared memory
  cluster.sync();
}

// Alg. 2 line 8 with eq. 19, one warp per row of V and one row per SM sub-partition (the
// 32-step back substitution is FP64-bound): the split-K slices of V = Y_(n) [Q0 | Q0^{k-1}]
// are added in a fixed order (FP32 slices in FP32: the split path's V carries the split TTMs'
// ~2^-16 relative error), V^ = (1 + beta) V0 - alpha beta V1, and A^ R0^T = V^ is solved by
// back substitution with lane = column.  Each block also adds up <V0, V^> and ||V^||^2 over
// its rows; the finish kernel adds the block partials.  With hpart set, each block also writes
// its rows' share of the Gram A^T A^ folded into 17 x 32 entries of 8 bytes: hpart[blk][k][c] =
// sum_i a^_ic a^_i,(c+k)%32 for k = 0..16 (every unordered pair once, k = 16 twice); the
// diagonal (k = 0, which gives lambda) as FP64, the rest as float-float (float2), which is all
// the Gram-route Cholesky uses them for, off the slow FP64 pipe.
constexpr int PREP_WARPS = 4;
constexpr int PREP_GK = 17;  // folded Gram entries per lane

template <typename TP>
__global__ void __launch_bounds__(PREP_WARPS * 32) finish_prep_kernel(const TP* __restrict__ part, int nparts, int I,
                                                                      int C, int R, const double* __restrict__ R0,
                                                                      double c0, double c1, double* __restrict__ Ahat,
                                                                      double* __restrict__ fitpart,
                                                                      double* __restrict__ hpart,
                                                                      unsigned int* status) {
  __shared__ double sM[CPQR_MAXR][CPQR_MAXR + 1];  // sM[l][c] = R0[l][c] / R0[c][c], l < c
  __shared__ double rdiag[CPQR_MAXR];
  __shared__ double red[PREP_WARPS][2];
  __shared__ double hred0[PREP_WARPS][32];
  __shared__ float2 hredf[PREP_WARPS][PREP_GK - 1][32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pdl_wait();
  if (tid < R) {
    const double d = R0[tid * R + tid];
    rdiag[tid] = (d != 0.0) ? 1.0 / d : 0.0;
    if (d == 0.0 && blockIdx.x == 0) atomicOr(status, CPQR_DEV_SINGULAR);
  }
  __syncthreads();
  for (int e = tid; e < R * R; e += PREP_WARPS * 32) sM[e / R][e % R] = R0[e] * rdiag[e % R];
  __syncthreads();
  const bool ext = (C == 2 * R);
  const size_t n = (size_t)I * C;
  double f_in = 0.0, f_nn = 0.0;
  double h0 = 0.0;
  ffa::ffn hf[PREP_GK - 1];
#pragma unroll
  for (int k = 0; k < PREP_GK - 1; ++k) hf[k] = ffa::ff_make(0.0f, 0.0f);
  const int i = blockIdx.x * PREP_WARPS + warp;
  if (i < I) {
    double v0 = 0.0, v1 = 0.0;
    if (lane < R) {
      // eight independent partial sums keep eight loads in flight; fixed order, deterministic
      const TP* p0 = part + (size_t)i * C + lane;
      TP a0[8], a1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a0[u] = a1[u] = TP(0);
      int q = 0;
      for (; q + 8 <= nparts; q += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          a0[u] += p0[(size_t)(q + u) * n];
          if (ext) a1[u] += p0[(size_t)(q + u) * n + R];
        }
      }
      for (; q < nparts; ++q) {  // fixed registers: a runtime index would move the arrays to local memory
        a0[0] += p0[(size_t)q * n];
        if (ext) a1[0] += p0[(size_t)q * n + R];
      }
      v0 = (double)(((a0[0] + a0[1]) + (a0[2] + a0[3])) + ((a0[4] + a0[5]) + (a0[6] + a0[7])));
      v1 = (double)(((a1[0] + a1[1]) + (a1[2] + a1[3])) + ((a1[4] + a1[5]) + (a1[6] + a1[7])));
    }
    const double vh = ext ? fma(c0, v0, c1 * v1) : v0;
    f_in = v0 * vh;
    f_nn = vh * vh;
    // column c of the back substitution: a^_c = res_c / R0[c][c], res_l -= R0[l][c] a^_c (l < c);
    // with the scaled R0 the serial chain is one shuffle and one FMA per column, and lane c keeps
    // its res_c (a move, not an FP64 instruction) for one scaling after the loop
    double res = vh, xk = 0.0;
    for (int c = R - 1; c >= 0; --c) {
      const double x = __shfl_sync(FULL, res, c);
      if (lane == c) xk = x;
      if (lane < c) res = fma(-sM[lane][c], x, res);
    }
    const double ahat = (lane < R) ? xk * rdiag[lane] : 0.0;
    if (lane < R) Ahat[(size_t)i * R + lane] = ahat;
    if (hpart) {
      h0 = ahat * ahat;
      const ffa::ffn af = ffa::ff_from_bits(ahat);
#pragma unroll
      for (int k = 1; k < PREP_GK; ++k) hf[k - 1] = ffa::ff_mul(af, ffa::ff_shfl(af, (lane + k) & 31));
    }
  }
  if (hpart) {
    hred0[warp][lane] = h0;
#pragma unroll
    for (int k = 1; k < PREP_GK; ++k) hredf[warp][k - 1][lane] = ffa::ff_st(hf[k - 1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    f_in += __shfl_xor_sync(FULL, f_in, o);
    f_nn += __shfl_xor_sync(FULL, f_nn, o);
  }
  if (lane == 0) {
    red[warp][0] = f_in;
    red[warp][1] = f_nn;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < PREP_WARPS; ++w) {
      a += red[w][0];
      b += red[w][1];
    }
    fitpart[2 * blockIdx.x] = a;
    fitpart[2 * blockIdx.x + 1] = b;
  }
  if (hpart) {
    for (int e = tid; e < PREP_GK * 32; e += PREP_WARPS * 32) {  // warp-uniform k
      const int k = e >> 5, c = e & 31;
      const size_t o = (size_t)blockIdx.x * PREP_GK * 32 + e;
      if (k == 0) {
        double a = 0.0;
#pragma unroll
        for (int w = 0; w < PREP_WARPS; ++w) a += hred0[w][c];
        hpart[o] = a;
      } else {
        ffa::ffn a = ffa::ff_ld(hredf[0][k - 1][c]);
#pragma unroll
        for (int w = 1; w < PREP_WARPS; ++w) a = ffa::ff_add(a, ffa::ff_ld(hredf[w][k - 1][c]));
        reinterpret_cast<float2*>(hpart)[o] = ffa::ff_st(a);
      }
    }
  }
}

size_t smem_bytes(int M, int R, int CL, bool use_smem) {
  size_t base = ((sizeof(SmemLayout) + 15) / 16) * 16;
  if (!use_smem) return base;
  size_t L = (size_t)(M + CL - 1) / CL;
  return base + L * R * sizeof(double);
}

constexpr size_t kSmemMax = 227 * 1024;

int g_cluster = 0;  // cluster size in use (16 if the device allows it, else 8)

// Function attributes of qr_cluster_kernel<CL>, set once per device.
template <int CL>
cudaError_t ensure_attributes() {
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(qr_cluster_kernel<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
  if (e != cudaSuccess) return e;
  if (CL > 8) {
    e = cudaFuncSetAttribute(qr_cluster_kernel<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  if (dev >= 0 && dev < 64) done[dev] = true;
  return cudaSuccess;
}

// Every launch takes the whole shared memory of its SMs: no other kernel's CTA can share an SM
// with the QR, whose serial FP64 chain would otherwise compete for issue slots (the Khatri-Rao
// QR runs beside the TTM chain on another stream).
template <int CL>
cudaError_t launch_cl(QrParams& p, cudaStream_t st) {
  const size_t full = smem_bytes(p.M, p.R, CL, true);
  p.use_smem = (full <= kSmemMax) ? 1 : 0;
  if (!p.use_smem && p.work == nullptr) return cudaErrorInvalidValue;
  cudaError_t e = ensure_attributes<CL>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = kSmemMax;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, qr_cluster_kernel<CL>, p);
}

// Chooses 16-CTA clusters when the device can schedule one with the largest
// shared-memory footprint, else 8.
int cluster_size() {
  if (g_cluster) return g_cluster;
  int use = 8;
  const char* env = getenv("CPQR_QR_CLUSTER");  // tuning override: 8 or 16
  if (env && atoi(env) == 8) {
    g_cluster = 8;
    return 8;
  }
  if (cudaFuncSetAttribute(qr_cluster_kernel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(qr_cluster_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax) ==
          cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = kSmemMax;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, qr_cluster_kernel<16>, &cfg) == cudaSuccess && n > 0) use = 16;
  }
  cudaGetLastError();
  g_cluster = use;
  return use;
}

cudaError_t run(QrParams& p, cudaStream_t st) {
  if (p.M < p.R || p.R < 1 || p.R > CPQR_MAXR) return cudaErrorInvalidValue;
  return cluster_size() == 16 ? launch_cl<16>(p, st) : launch_cl<8>(p, st);
}

}  // namespace

int qr_cluster_sms() { return cluster_size(); }


size_t house_qr_work_doubles(int64_t M, int R) { return (size_t)M * R; }
size_t krp_qr_work_doubles(const ZPlan& plan) { return (size_t)plan.M * plan.R; }

cudaError_t launch_house_qr(const double* A, int64_t M, int R, double* Q, double* Rout, double* work,
                            unsigned int* dev_status, cudaStream_t st) {
  if (R < 1 || R > CPQR_MAXR || M < R) return cudaErrorInvalidValue;
  QrParams p{};
  p.mode = MODE_PLAIN;
  if (M > (int64_t(1) << 30)) return cudaErrorInvalidValue;
  p.M = (int)M;
  p.R = R;
  p.work = work;
  for (int j = 0; j < CPQR_MAXR; ++j) p.act[j] = (int32_t)M;
  p.A_in = A;
  p.Q = Q;
  p.Rout = Rout;
  p.status = dev_status;
  return run(p, st);
}

cudaError_t launch_krp_qr(const ZPlan& plan, TriPtrs Rs, double* Q0, double* R0, double* work,
                          unsigned int* dev_status, cudaStream_t st, float* Q0f, int* run_if, const CholQr2Src* c2) {
  QrParams p{};
  p.mode = MODE_KRP;
  if (plan.M > (int64_t(1) << 30)) return cudaErrorInvalidValue;
  p.M = (int)plan.M;
  p.R = plan.R;
  p.work = work;
  for (int j = 0; j < CPQR_MAXR; ++j) p.act[j] = plan.act[j];
  p.perm = plan.perm;
  p.krp_m = plan.m;
  p.tri = Rs;
  p.Q = Q0;
  p.Qf = Q0f;
  p.Rout = R0;
  p.status = dev_status;
  p.run_if = run_if;
  if (c2 && run_if) {
    p.c2F = c2->F;
    p.c2Q1 = c2->Q1;
    p.c2R1 = c2->R1;
  }
  return run(p, st);
}

// ---------------------------------------------------------------------------
// Nested QR of a Khatri-Rao product of m >= 3 upper triangles.
//
// With W = R_{k2} (.) ... (.) R_{km} = Q_W S_W, the rows (i, w) of Z = R_{k1} (.) W are
// R_{k1}[i, r] (Q_W S_W)[w, r], so Z = (I_R (x) Q_W) Y with Y = R_{k1} (.) S_W, again a
// product of two upper triangles (R^2 rows, the staircase QR above).  Hence Z = Q0 R0 with
// R0 = R_Y and Q0 = (I_R (x) Q_W) Q_Y: m - 1 staircase QRs of R^2 x R products, from the
// right, and m - 2 assemblies Q <- (I (x) Q_W) Q_Y in FP64.  Every step is orthogonal and every
// R has a positive diagonal, so Q0 and R0 are those of the direct QR of Z up to rounding.
// ---------------------------------------------------------------------------

// out[(i, w), c] = sum_j QW[w, j] QY[(i, j), c] for i < R, w < Mw (row (i, w) = i * Mw + w);
// one row per Rpad lanes (Rpad = R rounded up to a power of two), lane = column c.  run_if (a
// guarded fallback): returns at once unless *run_if != 0.
__global__ void __launch_bounds__(256) krp_assemble_kernel(const double* __restrict__ QW, int64_t Mw,
                                                            const double* __restrict__ QY, int R, int Rpad,
                                                            double* __restrict__ out, float* __restrict__ outf,
                                                            const int* run_if) {
  if (run_if && *(volatile const int*)run_if == 0) return;
  const int lane = threadIdx.x & 31, sub = lane / Rpad, c = lane % Rpad;
  const int rpw = 32 / Rpad;
  const int64_t rows = (int64_t)R * Mw;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t wr = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wr * rpw < rows; wr += nwarps) {
    const int64_t row = wr * rpw + sub;
    const bool live = row < rows && c < R;
    const int64_t i = live ? row / Mw : 0, w = live ? row - i * Mw : 0;
    const double qw = live ? QW[w * R + c] : 0.0;
    const double* qy = QY + (size_t)i * R * R + c;
    double acc = 0.0;
    for (int j = 0; j < R; ++j) {
      const double a = __shfl_sync(FULL, qw, sub * Rpad + j);
      if (live) acc = fma(a, qy[(size_t)j * R], acc);
    }
    if (live) {
      out[row * R + c] = acc;
      if (outf) outf[row * R + c] = (float)acc;
    }
  }
}

// The same assembly when QY comes from the Gram route's rows kernels: row (i, j) of QY is the row
// R_a[i, :] * S[j, :] of two upper triangles times upper-triangular factors, so it is exactly zero
// left of column max(i, j), and only the terms j <= c of the columns c >= i can be nonzero (about
// a third of the dense multiply-adds, the part that bounds the dense kernel on GB300's FP64 pipe).
// The kept terms are summed in the dense kernel's order, so the results agree up to the sign of
// zero.  Rows (l, i, t) = (l * R + i) * T + t with w = l * T + t: T = mw, L = 1 is the assembly
// above.  One output row per thread and 32 consecutive w per warp; a warp takes the rows i and
// R - 1 - i, whose costs add up to about the mean, and of each the part `part` of P column
// ranges of equal cost, so every warp does about the same work, i (hence every QY address) is
// the same across the warp, and P brings small assemblies up to a few warps per SM quarter.
template <int RP>
__global__ void __launch_bounds__(128) krp_assemble_tri_kernel(const double* __restrict__ QW, int64_t LT, int64_t T,
                                                                const double* __restrict__ QY, int R, int P,
                                                                double* __restrict__ out, float* __restrict__ outf) {
  const int lane = threadIdx.x & 31;
  const int ng = (R + 1) / 2;
  const int64_t gw = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  const int part = (int)(gw % P);
  const int64_t rest = gw / P;
  const int64_t chunk = rest / ng;
  const int grp = (int)(rest - chunk * ng);
  if (chunk * 32 >= LT) return;
  const int64_t w = chunk * 32 + lane;
  const bool live = w < LT;
  double qw[RP];
#pragma unroll
  for (int j = 0; j < RP; ++j) qw[j] = (live && j < R) ? QW[w * R + j] : 0.0;
  const int64_t l = live ? w / T : 0, t = live ? w - l * T : 0;
  for (int h = 0; h < 2; ++h) {
    const int i = h ? R - 1 - grp : grp;
    if (h && i == grp) break;
    // column c >= i costs c + 1 and starts at cost (c (c + 1) - i (i + 1)) / 2 of the row's total;
    // it belongs to part min(P - 1, floor(start * P / total)), the zero columns c < i to part 0
    const int total = (R * (R + 1) - i * (i + 1)) / 2;
    const double* qy = QY + (size_t)i * R * R;
    const int64_t o = ((l * R + i) * T + t) * R;
#pragma unroll
    for (int c = 0; c < RP; ++c) {
      const int sp = (c * (c + 1) - i * (i + 1)) / 2 * P;
      const bool mine = (c < i) ? (part == 0) : (sp >= part * total && (part == P - 1 || sp < (part + 1) * total));
      if (c < R && mine) {
        double v = 0.0;
        if (c >= i) {
#pragma unroll
          for (int j = 0; j <= c; ++j) v = fma(qw[j], qy[j * R + c], v);
        }
        if (live) {
          out[o + c] = v;
          if (outf) outf[o + c] = (float)v;
        }
      }
    }
  }
}

cudaError_t launch_krp_assemble(const double* QW, int64_t mw, const double* QY, int R, double* out, float* outf,
                                cudaStream_t st) {
  return launch_krp_assemble_tri(QW, 1, mw, QY, R, out, outf, st);
}

cudaError_t launch_krp_assemble_tri(const double* QW, int64_t L, int64_t T, const double* QY, int R, double* out,
                                    float* outf, cudaStream_t st) {
  if (R < 1 || R > CPQR_MAXR || L < 1 || T < 1) return cudaErrorInvalidValue;
  const int64_t LT = L * T;
  const int64_t base = (LT + 31) / 32 * ((R + 1) / 2);
  // column parts for small assemblies: about 1024 warps (measured: 65536 rows of R = 16 ran in
  // 22.7 us as 1024 warps and 26 us as 3072; 4096 rows in 17.4 us as 64 warps, 8.5 us as 512)
  const int P = (int)std::max<int64_t>(1, std::min<int64_t>((1024 + base - 1) / base, std::max(1, R / 2)));
  const int64_t grid = (base * P + 3) / 4;
  if (grid > 0x7fffffff) return cudaErrorInvalidValue;
  if (R <= 8) krp_assemble_tri_kernel<8><<<(unsigned)grid, 128, 0, st>>>(QW, LT, T, QY, R, P, out, outf);
  else if (R <= 16) krp_assemble_tri_kernel<16><<<(unsigned)grid, 128, 0, st>>>(QW, LT, T, QY, R, P, out, outf);
  else krp_assemble_tri_kernel<32><<<(unsigned)grid, 128, 0, st>>>(QW, LT, T, QY, R, P, out, outf);
  return cudaGetLastError();
}

NestedBufs nested_views(double* work, int m, int R) {
  size_t Mw = 1;
  for (int k = 0; k < m - 1; ++k) Mw *= (size_t)R;
  NestedBufs b;
  b.S[0] = work;
  b.S[1] = work + (size_t)R * R;
  b.QY = work + 2 * (size_t)R * R;
  b.qrw = b.QY + (size_t)R * R * R;
  b.QW[0] = b.qrw + (size_t)R * R * R;
  b.QW[1] = b.QW[0] + Mw * R;
  return b;
}

size_t krp_nested_work_doubles(int m, int R) {
  size_t Mw = 1;
  for (int k = 0; k < m - 1; ++k) Mw *= (size_t)R;
  // two triangles, Q_Y, the staircase QR's rows, two Q_W
  return 2 * (size_t)R * R + 2 * (size_t)R * R * R + 2 * Mw * R;
}

cudaError_t launch_krp_qr_nested(const ZPlan& plan2, TriPtrs Rs, int m, double* Q0, double* R0, double* work,
                                 unsigned int* dev_status, cudaStream_t st, float* Q0f, int* nlaunch, int* run_if) {
  const int R = plan2.R;
  if (plan2.m != 2 || m < 2 || m > CPQR_MAXN || R < 1 || R > CPQR_MAXR) return cudaErrorInvalidValue;
  int launches = 0;
  TriPtrs t2{};
  t2.p[0] = Rs.p[m - 2];
  t2.p[1] = Rs.p[m - 1];
  if (m == 2) {
    if (nlaunch) *nlaunch = 1;
    return launch_krp_qr(plan2, t2, Q0, R0, work, dev_status, st, Q0f, run_if);
  }
  const NestedBufs nb = nested_views(work, m, R);
  double* const* S = nb.S;
  double* QY = nb.QY;
  double* qrw = nb.qrw;
  double* const* QW = nb.QW;
  // level 2: R_{k(m-1)} (.) R_{km} = Q_{W,2} S_2
  cudaError_t e = launch_krp_qr(plan2, t2, QW[0], S[0], qrw, dev_status, st, nullptr, run_if);
  if (e != cudaSuccess) return e;
  ++launches;
  int cur = 0;
  int64_t mw = (int64_t)R * R;  // rows of Q_{W,d-1}
  int Rpad = 1;
  while (Rpad < R) Rpad <<= 1;
  for (int d = 3; d <= m; ++d) {
    const bool last = (d == m);
    TriPtrs t{};
    t.p[0] = Rs.p[m - d];
    t.p[1] = S[(d - 3) & 1];
    e = launch_krp_qr(plan2, t, QY, last ? R0 : S[(d - 2) & 1], qrw, dev_status, st, nullptr, run_if);
    if (e != cudaSuccess) return e;
    double* out = last ? Q0 : QW[cur ^ 1];
    const int64_t rows = (int64_t)R * mw;
    const int64_t warps = (rows + (32 / Rpad) - 1) / (32 / Rpad);
    const int grid = (int)std::min<int64_t>((warps + 7) / 8, 152 * 8);
    krp_assemble_kernel<<<grid, 256, 0, st>>>(QW[cur], mw, QY, R, Rpad, out, last ? Q0f : nullptr, run_if);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    launches += 2;
    cur ^= 1;
    mw *= R;
  }
  if (nlaunch) *nlaunch = launches;
  return cudaSuccess;
}

int finish_prep_blocks(int64_t I) { return (int)((I + PREP_WARPS - 1) / PREP_WARPS); }

template <typename TP>
cudaError_t launch_finish_prep(const TP* parts, int nparts, int64_t I, int C, int R, const double* R0, double beta,
                               double alpha, double* Ahat, double* fitpart, double* hpart,
                               unsigned int* dev_status, cudaStream_t st) {
  if (I < 1 || I > (int64_t(1) << 30) || R < 1 || R > CPQR_MAXR || (C != R && C != 2 * R) || nparts < 1)
    return cudaErrorInvalidValue;
  const double c0 = 1.0 + beta, c1 = -alpha * beta;
  return launch_pdl(finish_prep_kernel<TP>, dim3(finish_prep_blocks(I)), dim3(PREP_WARPS * 32), 0, st, parts, nparts,
                    (int)I, C, R, R0, c0, c1, Ahat, fitpart, hpart, dev_status);
}
template cudaError_t launch_finish_prep<double>(const double*, int, int64_t, int, int, const double*, double, double,
                                                double*, double*, double*, unsigned int*, cudaStream_t);
template cudaError_t launch_finish_prep<float>(const float*, int, int64_t, int, int, const double*, double, double,
                                               double*, double*, double*, unsigned int*, cudaStream_t);

cudaError_t launch_mode_finish(const double* Ahat, const double* fitpart, int nfit, int64_t I, int R, FinishOut out,
                               double* work, unsigned int* dev_status, cudaStream_t st, int* run_if,
                               const CholQr2Src* c2) {
  QrParams p{};
  p.mode = MODE_FINISH;
  if (I > (int64_t(1) << 30)) return cudaErrorInvalidValue;
  p.M = (int)I;
  p.R = R;
  p.work = work;
  for (int j = 0; j < CPQR_MAXR; ++j) p.act[j] = (int32_t)I;
  p.Ahat = Ahat;
  p.fitpart = fitpart;
  p.nfit = nfit;
  p.fin = out;
  p.Q = out.Q;
  p.Qf = out.Qf;
  p.Rout = out.Rn;
  p.status = dev_status;
  p.run_if = run_if;
  if (c2 && run_if) {
    p.c2F = c2->F;
    p.c2Q1 = c2->Q1;
    p.c2R1 = c2->R1;
  }
  return run(p, st);
}

}  // namespace cpqr
