// QR of the Khatri-Rao product of two upper triangles, Z = R_a (.) R_b (R^2 x R, Alg. 2
// lines 3-4 for order-3 tensors and the building block of the nested QR for higher orders),
// by the Gram route, guarded by the Householder QR.
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
// makes the Householder staircase QR (smallqr.cu), launched after these kernels, recompute Q0 and
// R0; otherwise it returns at once.  The Householder QR's stability is thus kept for every Z,
// while the common well-conditioned case costs one 32-step Cholesky (after a Gram spread over one
// cluster) plus three row-parallel FP64 passes over all SMs instead of 32 cluster-wide
// Householder steps.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace cpqr {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int KG_MAXR = CPQR_MAXR;
constexpr int KG_LD = KG_MAXR + 1;
// max |E| accepted: the neglected O(E^2) terms stay below 1e-16
constexpr double kEMax = 1e-8;

// Workspace layout (doubles): R1, S (R1 scaled for the substitution), F, rinv, Q1 (R^2 x R),
// Q1^T (R x R^2), then the int flag.
struct KgWork {
  double* R1;
  double* S;
  double* F;
  double* rinv;
  double* Q1;
  double* Q1T;
  int* flag;
};

KgWork kg_views(double* work, int R) {
  KgWork w;
  const size_t rr = (size_t)KG_MAXR * KG_MAXR, M = (size_t)R * R;
  w.R1 = work;
  w.S = w.R1 + rr;
  w.F = w.S + rr;
  w.rinv = w.F + rr;
  w.Q1 = w.rinv + KG_MAXR;
  w.Q1T = w.Q1 + M * R;
  w.flag = reinterpret_cast<int*>(w.Q1T + M * R);
  return w;
}

// Gram (Hadamard of the two triangles' Grams) and its Cholesky factor on one 16-CTA cluster of
// 256 threads: CTA r forms rows c = r, r + 16 of the Gram (FP64 on one SM is ~8 GFLOP/s, so the
// two triangular products are spread) and stores them into CTA 0's shared memory; CTA 0 then
// runs the Cholesky.  Right-looking: at step j warp 0 forms row j of R1 from the pivot
// (rsqrt.approx.f64, measured to 53 bits, in the normal range), then all warps update the
// trailing rows.
constexpr int KG_CL = 16;

// named barriers of 256 threads (barrier 0 is __syncthreads)
__device__ __forceinline__ void nb_arrive(int id) { asm volatile("bar.arrive %0, 256;" ::"r"(id) : "memory"); }
__device__ __forceinline__ void nb_sync(int id) { asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory"); }

__global__ void __cluster_dims__(KG_CL, 1, 1) __launch_bounds__(256)
    kg_chol_kernel(const double* __restrict__ Ra, const double* __restrict__ Rb, int R, KgWork w) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  __shared__ double sa[KG_MAXR][KG_LD], sb[KG_MAXR][KG_LD], G[KG_MAXR][KG_LD], R1[KG_MAXR][KG_LD];
  __shared__ int bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < KG_MAXR * KG_MAXR; e += 256) {
    const int i = e / KG_MAXR, c = e % KG_MAXR;
    const bool in = i < R && c < R;
    sa[i][c] = in ? Ra[i * R + c] : 0.0;
    sb[i][c] = in ? Rb[i * R + c] : 0.0;
    R1[i][c] = 0.0;
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  // G[c][d] = (sum_i Ra[i][c] Ra[i][d]) (sum_i Rb[i][c] Rb[i][d]), i <= min(c, d), into CTA 0
  {
    const int c = rank + KG_CL * warp;
    if (warp < (KG_MAXR + KG_CL - 1) / KG_CL && c < R) {
      double ga = 0.0, gb = 0.0;
      const int d = lane;
      const int imax = min(c, d);
      for (int i = 0; i <= imax && d < R; ++i) {
        ga = fma(sa[i][c], sa[i][d], ga);
        gb = fma(sb[i][c], sb[i][d], gb);
      }
      cluster.map_shared_rank(&G[0][0], 0)[c * KG_LD + d] = (d < R) ? ga * gb : 0.0;
    }
  }
  cluster.sync();  // every row of G is in CTA 0; the other CTAs are done
  if (rank != 0) return;
  // Pipelined right-looking Cholesky.  Warp 0 produces the rows of R1: for row s + 1 it applies
  // step s's update itself (look-ahead) and starts the next square root at once, while warps
  // 1-7 apply step s to rows >= s + 2.  "Row k of R1 written": warp 0 arrives, warps 1-7 wait,
  // on barrier 1 (k even) or 3 (k odd).  "Step s applied to rows >= s + 2": warps 1-7 arrive,
  // warp 0 waits before its look-ahead on row s + 2, on barrier 2 (s even) or 4 (s odd).  Two
  // barriers per role because either side may arrive one generation ahead: warp 0 posts row
  // k + 1 before the others have taken row k, and a warp may post step s + 1 before warp 0
  // has taken step s.  Row k + 2 is posted only after warp 0 has taken step k (so all of
  // warps 1-7 took row k), and step s + 2 only after row s + 2, which follows warp 0's wait on
  // step s: each barrier's previous generation is complete before its next use.
  auto pivot_row = [&](int j) {  // warp 0: row j of R1 from the up-to-date row j of G
    const double g = G[j][j];
    const long long gbits = __double_as_longlong(g);
    double y;
    if (gbits > 0x05CD0B15A491EB84LL && gbits < 0x7A11A0FC668AAC70LL) {  // 1e-280 < g < 1e280
      asm("rsqrt.approx.f64 %0, %1;" : "=d"(y) : "d"(g));
    } else {
      y = (g > 0.0) ? 1.0 / sqrt(g) : 0.0;
      if (!(g > 0.0) && lane == 0) bad = 1;
    }
    const double r = (lane >= j && lane < R) ? G[j][lane] * y : 0.0;
    if (lane >= j && lane < R) R1[j][lane] = r;
    if (lane == j) w.rinv[j] = y;
    return r;
  };
  if (warp == 0) {
    double r = pivot_row(0);
    __syncwarp();
    nb_arrive(1);  // row 0
    for (int s = 0; s + 1 < R; ++s) {
      if (s >= 1) nb_sync(2 + 2 * ((s - 1) & 1));  // step s - 1 reached row s + 1
      const double rk = __shfl_sync(FULL, r, s + 1);  // R1[s][s + 1]
      if (lane >= s + 1 && lane < R) G[s + 1][lane] = fma(-rk, r, G[s + 1][lane]);
      __syncwarp();
      r = pivot_row(s + 1);
      __syncwarp();
      nb_arrive(1 + 2 * ((s + 1) & 1));  // row s + 1
    }
  } else {
    for (int s = 0; s + 1 < R; ++s) {
      nb_sync(1 + 2 * (s & 1));                     // row s of R1 is there
      for (int k = s + 1 + warp; k < R; k += 7) {   // rows s + 2, ...
        const double rk = R1[s][k];
        if (lane >= k && lane < R) G[k][lane] = fma(-rk, R1[s][lane], G[k][lane]);
      }
      if (s + 2 < R) nb_arrive(2 + 2 * (s & 1));    // step s
    }
    nb_sync(1 + 2 * ((R - 1) & 1));  // the last row
  }
  __syncthreads();
  // outputs: R1, S[c][c'] = R1[c][c'] / R1[c][c] (c < c') for the substitution, the flag
  for (int e = tid; e < KG_MAXR * KG_MAXR; e += 256) {
    const int c = e / KG_MAXR, d = e % KG_MAXR;
    w.R1[e] = R1[c][d];
    w.S[e] = (c < R && d < R && d > c) ? R1[c][d] * w.rinv[c] : 0.0;
  }
  if (tid == 0) *w.flag = bad;
}

// Q1 = Z R1^{-1}: one row (i, k) of Z per warp, z[c] = Ra[i][c] Rb[k][c]; forward substitution
// q R1 = z with lane = column (x[c'] -= x[c] S[c][c'] after column c, q[c] = x[c] / R1[c][c]).
// Writes Q1 row-major and transposed.
__global__ void __launch_bounds__(128) kg_q1_kernel(const double* __restrict__ Ra, const double* __restrict__ Rb,
                                                     int R, KgWork w) {
  const int lane = threadIdx.x & 31;
  const int M = R * R;
  const int t = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (t >= M) return;
  // column `lane` of S in registers (every load issued up front)
  double scol[KG_MAXR];
#pragma unroll
  for (int c = 0; c < KG_MAXR; ++c) scol[c] = (c < R && lane > c && lane < R) ? w.S[c * KG_MAXR + lane] : 0.0;
  const double ri = (lane < R) ? w.rinv[lane] : 0.0;
  const int i = t / R, k = t - i * R;
  double x = (lane < R) ? Ra[i * R + lane] * Rb[k * R + lane] : 0.0;
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
__global__ void __launch_bounds__(128) kg_e_kernel(int R, KgWork w) {
  const int lane = threadIdx.x & 31;
  const int M = R * R;
  const int npair = R * (R + 1) / 2;
  const int gw = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (gw >= npair) return;
  int c = 0, rem = gw;
  while (rem >= R - c) {
    rem -= R - c;
    ++c;
  }
  const int d = c + rem;
  const double* qc = w.Q1T + (size_t)c * M;
  const double* qd = w.Q1T + (size_t)d * M;
  // eight rows per lane per pass, every load issued before the products
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t0 = 0; t0 < M; t0 += 256) {
    double xc[8], xd[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + 32 * u + lane;
      xc[u] = (t < M) ? qc[t] : 0.0;
      xd[u] = (t < M) ? qd[t] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u & 3] = fma(xc[u], xd[u], acc[u & 3]);
  }
  double s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  if (lane == 0) {
    const double e = (c == d) ? s - 1.0 : s;
    w.F[c * KG_MAXR + d] = (c == d) ? 0.5 * e : e;
    if (!(fabs(e) <= kEMax)) atomicOr(w.flag, 1);  // also catches NaN
  }
}

// Q0 = Q1 (I - F) (one row per warp, lane = column: q0[c] = q1[c] - sum_{k <= c} q1[k] F[k][c]),
// and, on the first R warps of the grid, row c of R0 = (I + F) R1.
__global__ void __launch_bounds__(128) kg_q0_kernel(int R, KgWork w, double* __restrict__ Q0, float* __restrict__ Q0f,
                                                     double* __restrict__ R0) {
  const int lane = threadIdx.x & 31;
  const int M = R * R;
  const int t = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (t >= M) return;
  double fcol[KG_MAXR];  // F[k][lane], k <= lane
#pragma unroll
  for (int k = 0; k < KG_MAXR; ++k) fcol[k] = (k < R && lane >= k && lane < R) ? w.F[k * KG_MAXR + lane] : 0.0;
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
  double q = q1;
#pragma unroll
  for (int k = 0; k < KG_MAXR; ++k) {
    if (k < R) {
      const double qk = __shfl_sync(FULL, q1, k);
      q = fma(-qk, fcol[k], q);
    }
  }
  if (lane < R) {
    Q0[(size_t)t * R + lane] = q;
    if (Q0f) Q0f[(size_t)t * R + lane] = (float)q;
  }
}

}  // namespace

size_t krp_gram_work_doubles(int R) {
  const size_t M = (size_t)R * R;
  return 3 * (size_t)KG_MAXR * KG_MAXR + KG_MAXR + 2 * M * R + 1;
}

cudaError_t launch_krp_qr_gram(const ZPlan& plan2, const double* Ra, const double* Rb, double* Q0, double* R0,
                               double* gram_work, double* qr_work, unsigned int* dev_status, cudaStream_t st,
                               float* Q0f) {
  const int R = plan2.R;
  if (plan2.m != 2 || R < 1 || R > KG_MAXR || plan2.M != (int64_t)R * R) return cudaErrorInvalidValue;
  const KgWork w = kg_views(gram_work, R);
  const int M = R * R;
  static bool attr_done[64] = {};  // per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_done[dev]) {
    cudaError_t ea = cudaFuncSetAttribute(kg_chol_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (ea != cudaSuccess) return ea;
    attr_done[dev] = true;
  }
  kg_chol_kernel<<<KG_CL, 256, 0, st>>>(Ra, Rb, R, w);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  kg_q1_kernel<<<(M + 3) / 4, 128, 0, st>>>(Ra, Rb, R, w);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int npair = R * (R + 1) / 2;
  kg_e_kernel<<<(npair + 3) / 4, 128, 0, st>>>(R, w);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  kg_q0_kernel<<<(M + 3) / 4, 128, 0, st>>>(R, w, Q0, Q0f, R0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the Householder staircase QR, which returns at once unless the flag was raised
  TriPtrs t2{};
  t2.p[0] = Ra;
  t2.p[1] = Rb;
  return launch_krp_qr(plan2, t2, Q0, R0, qr_work, dev_status, st, Q0f, w.flag);
}

}  // namespace cpqr
