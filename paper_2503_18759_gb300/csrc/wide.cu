// Kernels of the wide-rank path (32 < R <= 192): the high-rank regime of Section 4.2 (Table 7 runs
// R = 75, 150, 175).  The R <= 32 kernels map the R columns of a factor onto the lanes of one warp;
// these tile the columns instead.  Every QR of this path (the factor QRs of Alg. 2 line 10 and the
// Khatri-Rao QR of lines 3-4) is a Cholesky QR:
//   G = Y^T Y (for a Khatri-Rao product Z: the Hadamard product of the triangles' Grams, exact),
//   equilibrated (unit diagonal) and shifted by R 2^-40, R1 = chol(G) in float-float on the FP32
//   pipe (square-root free: Schur rows and their pivots, scaled at the end), Q1 = Y R1^{-1} (FP64);
//   E = Q1^T Q1 - I; if max|E| > 1e-8 a second pass R2 = chol(Q1^T Q1), Q2 = Q1 R2^{-1}, R = R2 R1
//   runs (a device flag gates its kernels) and E is formed again; finally, to first order,
//   Q = Q1 (I - F), R = (I + F) R1 with F = striu(E) + diag(E) / 2.
// The result is the unique QR with a positive diagonal, to O(u + |E|^2).  FP64 carries every
// quantity the method uses (Q, R, the solve); float-float only preconditions (R1, R2), as on the
// narrow path.
#include <algorithm>

#include "common.cuh"
#include "ff.cuh"

namespace cpqr {

namespace {

using namespace ffa;

constexpr int WR_MAX = 192;  // largest R of the wide path (packed triangle of WR_MAX in float-float fits a CTA)
constexpr int GT = 64, GK = 16, GNT = 256;  // GEMM tile: 64 x 64 outputs, 16-deep K chunks, 4 x 4 per thread

__host__ __device__ __forceinline__ int64_t tri_off(int i, int R) { return (int64_t)i * R - (int64_t)i * (i - 1) / 2; }

// ---------------------------------------------------------------------------
// Batched tiled GEMM: P[z][b](m, n) = sum_{k in split z} A[b](m, k) B[b](k, n), written to the
// partial buffer of split z (or straight to C when there is one split).  Accessors by strides.
// ---------------------------------------------------------------------------
struct GemmView {
  int64_t M, N, K;
  int64_t sAm, sAk, sAb, sBk, sBn, sBb, sCm, sCn, sCb;
  int ksplit;      // K splits (grid.z); partials land at C + z * sCz
  int64_t sCz;
  int upper_only;  // only output tiles with tile column >= tile row (symmetric products)
};

template <typename TA, typename TB, typename TC, typename TAcc>
__global__ void __launch_bounds__(GNT) wide_gemm_kernel(const TA* __restrict__ A, const TB* __restrict__ B,
                                                         TC* __restrict__ C, GemmView v, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int tm = blockIdx.x, tn = blockIdx.y % ((int)((v.N + GT - 1) / GT));
  const int64_t b = blockIdx.y / ((int)((v.N + GT - 1) / GT));
  const int z = blockIdx.z;
  if (v.upper_only && tn < tm) return;
  __shared__ TAcc sA[GK][GT + 1];
  __shared__ TAcc sB[GK][GT + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)tm * GT, n0 = (int64_t)tn * GT;
  const int64_t kper = (v.K + v.ksplit - 1) / v.ksplit;
  const int64_t kb = (int64_t)z * kper, ke = std::min<int64_t>(v.K, kb + kper);
  const TA* Ab = A + b * v.sAb;
  const TB* Bb = B + b * v.sBb;
  TAcc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = TAcc(0);
  for (int64_t k0 = kb; k0 < ke; k0 += GK) {
    for (int e = tid; e < GK * GT; e += GNT) {
      // consecutive threads walk the operand's contiguous index when it is m / n
      const int kk = (v.sAm == 1) ? e / GT : e % GK, mm = (v.sAm == 1) ? e % GT : e / GK;
      const int64_t k = k0 + kk, m = m0 + mm;
      sA[kk][mm] = (k < ke && m < v.M) ? (TAcc)Ab[m * v.sAm + k * v.sAk] : TAcc(0);
      const int kb2 = (v.sBn == 1) ? e / GT : e % GK, nn = (v.sBn == 1) ? e % GT : e / GK;
      const int64_t k2 = k0 + kb2, n = n0 + nn;
      sB[kb2][nn] = (k2 < ke && n < v.N) ? (TAcc)Bb[k2 * v.sBk + n * v.sBn] : TAcc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      TAcc a[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = sA[kk][ty * 4 + i];
        bv[i] = sB[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bv[j];
    }
    __syncthreads();
  }
  TC* Cz = C + (int64_t)z * v.sCz + b * v.sCb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty * 4 + i;
    if (m >= v.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t n = n0 + tx * 4 + j;
      if (n < v.N) Cz[m * v.sCm + n * v.sCn] = (TC)acc[i][j];
    }
  }
}

// C(m, n) = sum_z P[z](m, n) in z order (then optionally D(m, n) - that sum), m < M, n < N.
template <typename TP, typename TC>
__global__ void wide_reduce_kernel(const TP* __restrict__ P, int nz, int64_t sPz, int64_t M, int64_t N,
                                   int64_t sPm, TC* __restrict__ C, int64_t sCm, const TC* __restrict__ D,
                                   int64_t sDm, int upper_only, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e / N, n = e - m * N;
    if (upper_only && (n / GT) < (m / GT)) continue;
    TP s = TP(0);
    for (int z = 0; z < nz; ++z) s += P[(int64_t)z * sPz + m * sPm + n];
    C[m * sCm + n] = D ? (TC)(D[m * sDm + n] - s) : (TC)s;
  }
}

// ---------------------------------------------------------------------------
// Cholesky of an R x R SPD matrix (FP64, full, row-major) in float-float: G is equilibrated to a
// unit diagonal and shifted by R 2^-40; the Schur rows S_j and pivots p_j give
// R1 = diag(p)^{-1/2} S diag(d)^{-1}, d = sqrt(diag(G)).  One CTA; the upper triangle stays in
// shared memory (packed rows).  gate: run only if *gate != 0 (nullptr: always).  A pivot that is not
// positive sets CPQR_DEV_SINGULAR.
// ---------------------------------------------------------------------------
constexpr int CHT = 1024;

__global__ void __launch_bounds__(CHT) wide_chol_kernel(const double* __restrict__ G, int R, double* __restrict__ R1,
                                                        const int* __restrict__ gate, unsigned int* status) {
  if (gate && *gate == 0) return;
  extern __shared__ float2 tri[];  // packed upper rows: (i, c) at tri_off(i) + c - i
  __shared__ double dsc[WR_MAX];    // 1 / sqrt(G_jj)
  __shared__ float2 wrow[WR_MAX];   // S_j,i / p_j of the current step
  __shared__ float2 piv[WR_MAX];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int j = tid; j < R; j += CHT) {
    const double g = G[(int64_t)j * R + j];
    dsc[j] = (g > 0.0) ? 1.0 / sqrt(g) : 0.0;
  }
  __syncthreads();
  const double shift = (double)R * 0x1p-40;
  for (int64_t e = tid; e < (int64_t)R * R; e += CHT) {
    const int i = (int)(e / R), c = (int)(e - (int64_t)i * R);
    if (c < i) continue;
    double g = G[e] * dsc[i] * dsc[c];
    if (c == i) g += shift;
    const ffn f = ff_from_bits(g);
    tri[tri_off(i, R) + c - i] = ff_st(f);
  }
  __syncthreads();
  for (int j = 0; j < R; ++j) {
    const int64_t oj = tri_off(j, R);
    if (tid == 0) {
      int b = 0;
      const ffn p = ff_ld(tri[oj]);
      piv[j] = tri[oj];
      const ffn inv = ff_recip(p, &b);
      if (b || !(p.hi > 0.f)) bad = 1;
      wrow[j] = ff_st(inv);
    }
    __syncthreads();
    const ffn inv = ff_ld(wrow[j]);
    // w_i = S_j,i / p_j for i > j
    for (int i = j + 1 + tid; i < R; i += CHT) wrow[i] = ff_st(ff_mul(ff_ld(tri[oj + i - j]), inv));
    __syncthreads();
    // trailing update S_i,c -= w_i S_j,c for j < i <= c: warps take rows, lanes columns
    const int warp = tid >> 5, lane = tid & 31;
    for (int i = j + 1 + warp; i < R; i += CHT / 32) {
      const ffn wi = ff_ld(wrow[i]);
      const int64_t oi = tri_off(i, R);
      for (int c = i + lane; c < R; c += 32) {
        const ffn s = ff_ld(tri[oi + c - i]);
        tri[oi + c - i] = ff_st(ff_fms(s, wi, ff_ld(tri[oj + c - j])));
      }
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicOr(status, CPQR_DEV_SINGULAR);
    return;
  }
  // R1[j][c] = S_j,c / sqrt(p_j) / d_c  (d_c = sqrt(G_cc): undo the equilibration)
  for (int64_t e = tid; e < (int64_t)R * R; e += CHT) {
    const int j = (int)(e / R), c = (int)(e - (int64_t)j * R);
    double v = 0.0;
    if (c >= j) {
      const double pj = ff_val(piv[j]);
      v = ff_val(tri[tri_off(j, R) + c - j]) / sqrt(pj) / dsc[c];
    }
    R1[e] = v;
  }
}

// ---------------------------------------------------------------------------
// Row substitution Q1 = Y R1^{-1} (R1 upper, FP64): one warp per row, lane l owns columns
// l, l + 32, ...  Rows of Y are either read (ld = row stride) or, for a Khatri-Rao product of m
// triangles, generated: row (i_1, ..., i_m) (i_m fastest) is the Hadamard product of the triangles'
// rows, zero left of max(i_k), where the substitution starts.  gate as above.  Optional FP32 copy.
// ---------------------------------------------------------------------------
struct KrpRows {
  const double* tri[CPQR_MAXN];  // m upper triangles (R x R row-major), or nullptr
  int m;
};

// (Y may be Q: each warp reads its whole row before it writes it.)
__global__ void __launch_bounds__(256) wide_trsm_rows_kernel(const double* Y, int64_t M, int R, KrpRows kr,
                                                            const double* __restrict__ R1, double* Q,
                                                            float* __restrict__ Qf, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  extern __shared__ double sR[];  // packed R1 upper rows, then 1 / diag
  double* rinv = sR + tri_off(R, R);
  for (int64_t e = threadIdx.x; e < (int64_t)R * R; e += blockDim.x) {
    const int i = (int)(e / R), c = (int)(e - (int64_t)i * R);
    if (c >= i) sR[tri_off(i, R) + c - i] = R1[e];
    if (c == i) rinv[i] = 1.0 / R1[e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < M; row += warps) {
    double y[WR_MAX / 32];
    int c0 = 0;
    if (kr.m > 0) {
      int idx[CPQR_MAXN];
      int64_t t = row;
      for (int k = kr.m - 1; k >= 0; --k) {
        idx[k] = (int)(t % R);
        t /= R;
      }
      for (int k = 0; k < kr.m; ++k) c0 = max(c0, idx[k]);
#pragma unroll
      for (int q = 0; q < WR_MAX / 32; ++q) {
        const int c = lane + 32 * q;
        double v = 0.0;
        if (c < R && c >= c0) {
          v = 1.0;
          for (int k = 0; k < kr.m; ++k) v *= kr.tri[k][(int64_t)idx[k] * R + c];
        }
        y[q] = v;
      }
    } else {
#pragma unroll
      for (int q = 0; q < WR_MAX / 32; ++q) {
        const int c = lane + 32 * q;
        y[q] = (c < R) ? Y[row * R + c] : 0.0;
      }
    }
    // forward substitution over columns: x_c = y_c / R1_cc, then y_l -= x_c R1_cl (l > c)
    for (int c = c0; c < R; ++c) {
      const int q = c >> 5;
      double xc = 0.0;
#pragma unroll
      for (int qq = 0; qq < WR_MAX / 32; ++qq)
        if (qq == q) xc = y[qq];
      xc = __shfl_sync(0xffffffffu, xc, c & 31) * rinv[c];
      const int64_t oc = tri_off(c, R);
#pragma unroll
      for (int qq = 0; qq < WR_MAX / 32; ++qq) {
        const int l = lane + 32 * qq;
        if (l > c && l < R) y[qq] -= xc * sR[oc + l - c];
        if (l == c) y[qq] = xc;
      }
    }
#pragma unroll
    for (int q = 0; q < WR_MAX / 32; ++q) {
      const int c = lane + 32 * q;
      if (c < R) {
        Q[row * R + c] = y[q];
        if (Qf) Qf[row * R + c] = (float)y[q];
      }
    }
  }
}

// E = G - I (G = Q1^T Q1 upper, full R x R row-major in), F = striu(E) + diag(E) / 2, and the
// guard: *need2 = (max |E| > 1e-8) when need2 is given (and then nothing else is written),
// otherwise IF = I + F and F itself.  One block.
__global__ void wide_e_kernel(const double* __restrict__ G, int R, int* __restrict__ need2, double* __restrict__ F,
                              double* __restrict__ IF, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  __shared__ int big;
  if (threadIdx.x == 0) big = 0;
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)R * R; e += blockDim.x) {
    const int i = (int)(e / R), c = (int)(e - (int64_t)i * R);
    const double gi = (c >= i) ? G[e] : G[(int64_t)c * R + i];
    const double E = gi - (i == c ? 1.0 : 0.0);
    if (need2) {
      if (!(fabs(E) <= 1e-8)) big = 1;
    } else {
      const double f = (c > i) ? E : (c == i ? 0.5 * E : 0.0);
      F[e] = f;
      IF[e] = f + (i == c ? 1.0 : 0.0);
    }
  }
  __syncthreads();
  if (need2 && threadIdx.x == 0) *need2 = big;
}

// Rows of A^ = V^ R0^{-T}: v^ = (1 + beta) v0 - alpha beta v1 (eq. 19, by linearity on V) from the
// nparts split-K slices of [V0 | V1] (FP32 or FP64, I x C each), then back substitution with R0
// (upper): a_c = (v_c - sum_{l > c} R0_cl a_l) / R0_cc.  One warp per row; per-row fit terms
// <v0, v^>, |v^|^2 to fitrow (I x 2).
template <typename TV>
__global__ void __launch_bounds__(256) wide_finish_prep_kernel(const TV* __restrict__ vw, int nparts, int64_t I,
                                                              int C, int R, const double* __restrict__ R0,
                                                              double beta, double alpha, double* __restrict__ Ahat,
                                                              double* __restrict__ fitrow) {
  extern __shared__ double sR[];  // packed R0 upper rows, then 1 / diag
  double* rinv = sR + tri_off(R, R);
  for (int64_t e = threadIdx.x; e < (int64_t)R * R; e += blockDim.x) {
    const int i = (int)(e / R), c = (int)(e - (int64_t)i * R);
    if (c >= i) sR[tri_off(i, R) + c - i] = R0[e];
    if (c == i) rinv[i] = 1.0 / R0[e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < I; row += warps) {
    double v[WR_MAX / 32];
    double in = 0.0, nn = 0.0;
#pragma unroll
    for (int q = 0; q < WR_MAX / 32; ++q) {
      const int c = lane + 32 * q;
      double v0 = 0.0, v1 = 0.0;
      if (c < R) {
        for (int s = 0; s < nparts; ++s) {
          const TV* sl = vw + ((int64_t)s * I + row) * C;
          v0 += (double)sl[c];
          if (C > R) v1 += (double)sl[R + c];
        }
      }
      const double vh = (C > R) ? (1.0 + beta) * v0 - alpha * beta * v1 : v0;
      in += v0 * vh;
      nn += vh * vh;
      v[q] = vh;
    }
    // back substitution from the last column
    for (int c = R - 1; c >= 0; --c) {
      const int q = c >> 5;
      double ac = 0.0;
#pragma unroll
      for (int qq = 0; qq < WR_MAX / 32; ++qq)
        if (qq == q) ac = v[qq];
      ac = __shfl_sync(0xffffffffu, ac, c & 31) * rinv[c];
#pragma unroll
      for (int qq = 0; qq < WR_MAX / 32; ++qq) {
        const int l = lane + 32 * qq;
        if (l < c) v[qq] -= ac * sR[tri_off(l, R) + c - l];
        if (l == c) v[qq] = ac;
      }
    }
#pragma unroll
    for (int q = 0; q < WR_MAX / 32; ++q) {
      const int c = lane + 32 * q;
      if (c < R) Ahat[row * R + c] = v[q];
    }
    for (int o = 16; o > 0; o >>= 1) {
      in += __shfl_xor_sync(0xffffffffu, in, o);
      nn += __shfl_xor_sync(0xffffffffu, nn, o);
    }
    if (lane == 0) {
      fitrow[2 * row] = in;
      fitrow[2 * row + 1] = nn;
    }
  }
}

// Column norms lambda_c = |A^(:, c)| (fixed order: thread t sums rows t, t + 256, ..., then a tree),
// A = A^ / lambda; block 0 also sums the per-row fit terms into fit_terms.  One block per column.
__global__ void __launch_bounds__(256) wide_colnorm_kernel(const double* __restrict__ Ahat, int64_t I, int R,
                                                          double* __restrict__ A, double* __restrict__ lambda,
                                                          const double* __restrict__ fitrow,
                                                          double* __restrict__ fit_terms, unsigned int* status) {
  __shared__ double red[256];
  __shared__ double red2[256];
  const int c = blockIdx.x, t = threadIdx.x;
  double s = 0.0;
  for (int64_t i = t; i < I; i += 256) {
    const double a = Ahat[i * R + c];
    s += a * a;
  }
  red[t] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) red[t] += red[t + w];
    __syncthreads();
  }
  const double lam = sqrt(red[0]);
  if (t == 0) {
    lambda[c] = lam;
    if (!(lam > 0.0)) atomicOr(status, CPQR_DEV_SINGULAR);
  }
  const double il = (lam > 0.0) ? 1.0 / lam : 0.0;
  for (int64_t i = t; i < I; i += 256) A[i * R + c] = Ahat[i * R + c] * il;
  if (c == 0) {
    double a = 0.0, b = 0.0;
    for (int64_t i = t; i < I; i += 256) {
      a += fitrow[2 * i];
      b += fitrow[2 * i + 1];
    }
    __syncthreads();
    red[t] = a;
    red2[t] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (t < w) {
        red[t] += red[t + w];
        red2[t] += red2[t + w];
      }
      __syncthreads();
    }
    if (t == 0) {
      fit_terms[0] = red[0];
      fit_terms[1] = red2[0];
    }
  }
}

// C = A B for upper-triangular R x R A, B (row-major): one block per row i, c >= i.  With a gate
// that is zero: C = B.
__global__ void wide_trmm_kernel(const double* __restrict__ A, const double* __restrict__ B, int R,
                                 double* __restrict__ C, const int* __restrict__ gate) {
  const int i = blockIdx.x;
  const bool on = !gate || *gate != 0;
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    double s = 0.0;
    if (!on) {
      s = B[(int64_t)i * R + c];
    } else if (c >= i) {
      for (int l = i; l <= c; ++l) s += A[(int64_t)i * R + l] * B[(int64_t)l * R + c];
    }
    C[(int64_t)i * R + c] = s;
  }
}

// In place, row by row: q <- q (I - F) (F upper, R x R row-major), and the FP32 copy.  The
// correction q F is summed in float-float on the FP32 pipe (F in shared memory as float-float,
// q_l split once per row): its ~2^-48 relative error is of the correction, not of q, and one FP64
// subtraction per entry remains, so the result equals the FP64 form to FP64 rounding at a fraction
// of the FP64 pipe's time.  Each warp takes two rows at a time (two independent chains per
// column) and reads q_l from its own rows staged in shared memory (a broadcast load per l).
constexpr int RM_ROWS = 2;
__global__ void __launch_bounds__(256) wide_rowmul_kernel(double* __restrict__ Q, int64_t M, int R,
                                                         const double* __restrict__ F, float* __restrict__ Qf) {
  using namespace ffa;
  extern __shared__ float2 sFf[];  // packed upper rows of F (float-float), then the staged rows
  const int64_t nF = tri_off(R, R);
  float2* sQ = sFf + nF + (threadIdx.x >> 5) * RM_ROWS * WR_MAX;  // this warp's rows
  for (int64_t e = threadIdx.x; e < (int64_t)R * R; e += blockDim.x) {
    const int i = (int)(e / R), c = (int)(e - (int64_t)i * R);
    if (c >= i) sFf[tri_off(i, R) + c - i] = ff_st(ff_from_bits(F[e]));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const ffn zero = ff_make(0.0f, 0.0f);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * RM_ROWS; row0 < M;
       row0 += warps * RM_ROWS) {
    ffn acc[RM_ROWS][WR_MAX / 32];
#pragma unroll
    for (int r = 0; r < RM_ROWS; ++r)
#pragma unroll
      for (int qq = 0; qq < WR_MAX / 32; ++qq) {
        const int c = lane + 32 * qq;
        const int64_t row = row0 + r;
        if (c < R) sQ[r * WR_MAX + c] = ff_st(ff_from_bits(row < M ? Q[row * R + c] : 0.0));
        acc[r][qq] = zero;
      }
    __syncwarp();
    // acc_c = sum_{l <= c} q_l F_lc, l in order
    for (int l = 0; l < R; ++l) {
      const int64_t ol = tri_off(l, R);
      ffn ql[RM_ROWS];
#pragma unroll
      for (int r = 0; r < RM_ROWS; ++r) ql[r] = ff_ld(sQ[r * WR_MAX + l]);
#pragma unroll
      for (int qq = 0; qq < WR_MAX / 32; ++qq) {
        const int c = lane + 32 * qq;
        if (c >= l && c < R) {
          const ffn f = ff_ld(sFf[ol + c - l]);
#pragma unroll
          for (int r = 0; r < RM_ROWS; ++r) acc[r][qq] = ff_fms(acc[r][qq], ff_neg(ql[r]), f);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RM_ROWS; ++r) {
      const int64_t row = row0 + r;
      if (row >= M) break;
#pragma unroll
      for (int qq = 0; qq < WR_MAX / 32; ++qq) {
        const int c = lane + 32 * qq;
        if (c < R) {
          const double o = Q[row * R + c] - ff_val(acc[r][qq]);  // q read again (L2): fewer registers
          Q[row * R + c] = o;
          if (Qf) Qf[row * R + c] = (float)o;
        }
      }
    }
    __syncwarp();
  }
}

// G = the Hadamard product of the m triangles' Grams T_k^T T_k (each R x R, FP64, given in Gk).
__global__ void wide_hadamard_kernel(const double* __restrict__ Gk, int m, int R, double* __restrict__ G) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * R;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = 1.0;
    for (int k = 0; k < m; ++k) v *= Gk[(int64_t)k * R * R + e];
    G[e] = v;
  }
}

}  // namespace

bool wide_supported(int R) { return R > CPQR_MAXR && R <= WR_MAX; }

// ---- GEMM launches ----
template <typename TA, typename TB, typename TC, typename TAcc>
static cudaError_t gemm(const TA* A, const TB* B, TC* C, GemmView v, int batches, TAcc* part, size_t part_elems,
                        const TC* D, int64_t sDm, const int* gate, cudaStream_t st) {
  const int64_t tm = (v.M + GT - 1) / GT, tn = (v.N + GT - 1) / GT;
  if (tm > 0x7fffffff || tn * batches > 65535 || v.ksplit > 65535) return cudaErrorInvalidValue;
  if (v.ksplit > 1 || D) {
    // split-K partials (sCz apart) into part, then a fixed-order reduction into C
    if (!part || (size_t)v.ksplit * v.M * v.N > part_elems || batches != 1) return cudaErrorInvalidValue;
    GemmView pv = v;
    pv.sCm = v.N;
    pv.sCn = 1;
    pv.sCb = 0;
    pv.sCz = v.M * v.N;
    wide_gemm_kernel<TA, TB, TAcc, TAcc><<<dim3((unsigned)tm, (unsigned)(tn * batches), (unsigned)v.ksplit), GNT, 0,
                                           st>>>(A, B, part, pv, gate);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t n = v.M * v.N;
    wide_reduce_kernel<TAcc, TC><<<(unsigned)std::min<int64_t>((n + 255) / 256, 1216), 256, 0, st>>>(
        part, v.ksplit, pv.sCz, v.M, v.N, v.N, C, v.sCm, D, sDm, v.upper_only, gate);
    return cudaGetLastError();
  }
  wide_gemm_kernel<TA, TB, TC, TAcc><<<dim3((unsigned)tm, (unsigned)(tn * batches), 1), GNT, 0, st>>>(A, B, C, v,
                                                                                                     gate);
  return cudaGetLastError();
}

// Split-K count: at most two CTAs per SM in all (the FP64 pipe is the limit and two CTAs fit an SM;
// one more CTA than that makes its SM run a third K-range after the others have finished), and
// K-ranges of at least 32.
static int ksplits(int64_t M, int64_t N, int64_t K, bool upper) {
  int64_t tm = (M + GT - 1) / GT, tiles = tm * ((N + GT - 1) / GT);
  if (upper) tiles = (tiles + tm) / 2;
  int64_t want = std::max<int64_t>(1, (2 * 152) / tiles);
  want = std::min<int64_t>(want, std::max<int64_t>(1, K / 32));
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, 64));
}

struct WideWork {
  double* part;  // split-K partials: 64 R^2
  double* G;     // R^2 each below
  double* R1;
  double* R2;
  double* T;
  double* F;
  double* IF;
  double* Gk;    // CPQR_MAXN R^2: the triangles' Grams
  int* need2;    // second-pass flag
};

static WideWork carve(double* w, int R) {
  const size_t rr = (size_t)R * R;
  WideWork k;
  k.part = w;
  k.G = w + 64 * rr;
  k.R1 = k.G + rr;
  k.R2 = k.R1 + rr;
  k.T = k.R2 + rr;
  k.F = k.T + rr;
  k.IF = k.F + rr;
  k.Gk = k.IF + rr;
  k.need2 = reinterpret_cast<int*>(k.Gk + CPQR_MAXN * rr);
  return k;
}

size_t wide_work_doubles(int R) { return (size_t)(70 + CPQR_MAXN) * R * R + 8; }

// G = Y^T Y (M x R rows, FP64): the upper 64 x 64 tiles (all the Cholesky and E read).
static cudaError_t gram(const double* Y, int64_t M, int R, double* G, double* part, const int* gate,
                        cudaStream_t st) {
  GemmView v{};
  v.M = R; v.N = R; v.K = M;
  v.sAm = 1; v.sAk = R; v.sBk = R; v.sBn = 1; v.sCm = R; v.sCn = 1;
  v.upper_only = 1;
  v.ksplit = ksplits(R, R, M, true);
  return gemm<double, double, double, double>(Y, Y, G, v, 1, part, (size_t)64 * R * R, nullptr, 0, gate, st);
}

static size_t chol_smem(int R) { return (size_t)tri_off(R, R) * sizeof(float2); }
static size_t tri_smem(int R) { return ((size_t)tri_off(R, R) + R) * sizeof(double); }
static size_t rowmul_smem(int R) { return ((size_t)tri_off(R, R) + 8 * RM_ROWS * WR_MAX) * sizeof(float2); }

static cudaError_t set_smem_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(wide_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)chol_smem(WR_MAX));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wide_trsm_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tri_smem(WR_MAX));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wide_rowmul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rowmul_smem(WR_MAX));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wide_finish_prep_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tri_smem(WR_MAX));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wide_finish_prep_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tri_smem(WR_MAX));
  if (e == cudaSuccess) done = true;
  return e;
}

static int rows_grid(int64_t M) { return (int)std::max<int64_t>(1, std::min<int64_t>((M + 7) / 8, 152 * 4)); }

// out[p, r, s] = sum_k T[p, k, s] Q[k, r] on the CUDA cores (accumulation in TAcc).
template <typename TT, typename TQ, typename TO, typename TAcc>
cudaError_t launch_ttm_wide(const TT* T, const TQ* Q, TO* out, int64_t P, int64_t K, int64_t S, int R,
                            cudaStream_t st) {
  GemmView v{};
  v.ksplit = 1;
  if (S == 1) {  // one GEMM: (P x K) (K x R)
    v.M = P; v.N = R; v.K = K;
    v.sAm = K; v.sAk = 1; v.sBk = R; v.sBn = 1; v.sCm = R; v.sCn = 1;
    return gemm<TT, TQ, TO, TAcc>(T, Q, out, v, 1, nullptr, 0, nullptr, 0, nullptr, st);
  }
  // per p: (R x K) Q^T times (K x S) T_p, batches of p in grid.y chunks (grid.y <= 65535)
  v.M = R; v.N = S; v.K = K;
  v.sAm = 1; v.sAk = R; v.sAb = 0;
  v.sBk = S; v.sBn = 1; v.sBb = K * S;
  v.sCm = S; v.sCn = 1; v.sCb = (int64_t)R * S;
  const int64_t tn = (S + GT - 1) / GT;
  if (tn > 65535) return cudaErrorInvalidValue;
  const int64_t chunk = 65535 / tn;
  for (int64_t p0 = 0; p0 < P; p0 += chunk) {
    const int nb = (int)std::min<int64_t>(chunk, P - p0);
    cudaError_t e = gemm<TQ, TT, TO, TAcc>(Q, T + p0 * K * S, out + p0 * (int64_t)R * S, v, nb, nullptr, 0, nullptr,
                                           0, nullptr, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
template cudaError_t launch_ttm_wide<double, double, double, double>(const double*, const double*, double*, int64_t,
                                                                     int64_t, int64_t, int, cudaStream_t);
template cudaError_t launch_ttm_wide<float, double, double, double>(const float*, const double*, double*, int64_t,
                                                                    int64_t, int64_t, int, cudaStream_t);
template cudaError_t launch_ttm_wide<float, float, float, float>(const float*, const float*, float*, int64_t, int64_t,
                                                                 int64_t, int, cudaStream_t);

// The Cholesky QR of the file comment.  Y: M x R rows (FP64), or (tri, m > 0) the Khatri-Rao
// product of the m upper R x R triangles tri[0..m-1] (its Gram is the Hadamard product of theirs).
// Q (M x R; may not alias Y), Qf (optional FP32 copy), Rout (R x R upper).  work: wide_work_doubles(R).
cudaError_t launch_wide_qr(const double* Y, int64_t M, int R, const double* const* tri, int m, double* Q, float* Qf,
                           double* Rout, double* work, unsigned int* status, cudaStream_t st) {
  if (!wide_supported(R) || M < R || (m > 0 && (!tri || m > CPQR_MAXN))) return cudaErrorInvalidValue;
  if (M > (int64_t(1) << 40)) return cudaErrorInvalidValue;
  cudaError_t e = set_smem_attrs();
  if (e != cudaSuccess) return e;
  WideWork k = carve(work, R);
  KrpRows kr{};
  kr.m = m > 0 ? m : 0;
  for (int i = 0; i < kr.m; ++i) kr.tri[i] = tri[i];
  // pass 1: R1 = chol(G), Q = Y R1^{-1}
  if (kr.m > 0) {
    for (int i = 0; i < kr.m && e == cudaSuccess; ++i) {
      GemmView v{};  // T_i^T T_i (both triangles: the Hadamard product reads all of it)
      v.M = R; v.N = R; v.K = R;
      v.sAm = 1; v.sAk = R; v.sBk = R; v.sBn = 1; v.sCm = R; v.sCn = 1;
      v.ksplit = ksplits(R, R, R, false);
      e = gemm<double, double, double, double>(tri[i], tri[i], k.Gk + (size_t)i * R * R, v, 1, k.part,
                                               (size_t)64 * R * R, nullptr, 0, nullptr, st);
    }
    if (e != cudaSuccess) return e;
    wide_hadamard_kernel<<<(R * R + 255) / 256, 256, 0, st>>>(k.Gk, kr.m, R, k.G);
    e = cudaGetLastError();
  } else {
    e = gram(Y, M, R, k.G, k.part, nullptr, st);
  }
  if (e != cudaSuccess) return e;
  wide_chol_kernel<<<1, CHT, chol_smem(R), st>>>(k.G, R, k.R1, nullptr, status);
  wide_trsm_rows_kernel<<<rows_grid(M), 256, tri_smem(R), st>>>(Y, M, R, kr, k.R1, Q, nullptr, nullptr);
  // E of pass 1; a second pass when max |E| > 1e-8
  e = gram(Q, M, R, k.G, k.part, nullptr, st);
  if (e != cudaSuccess) return e;
  wide_e_kernel<<<1, 256, 0, st>>>(k.G, R, k.need2, nullptr, nullptr, nullptr);
  wide_chol_kernel<<<1, CHT, chol_smem(R), st>>>(k.G, R, k.R2, k.need2, status);
  KrpRows none{};
  wide_trsm_rows_kernel<<<rows_grid(M), 256, tri_smem(R), st>>>(Q, M, R, none, k.R2, Q, nullptr, k.need2);
  wide_trmm_kernel<<<R, 128, 0, st>>>(k.R2, k.R1, R, k.T, k.need2);  // T = need2 ? R2 R1 : R1
  e = gram(Q, M, R, k.G, k.part, k.need2, st);
  if (e != cudaSuccess) return e;
  // first-order correction from the last E: Q <- Q (I - F), R = (I + F) T
  wide_e_kernel<<<1, 256, 0, st>>>(k.G, R, nullptr, k.F, k.IF, nullptr);
  wide_rowmul_kernel<<<rows_grid((M + RM_ROWS - 1) / RM_ROWS), 256, rowmul_smem(R), st>>>(Q, M, R, k.F, Qf);
  wide_trmm_kernel<<<R, 128, 0, st>>>(k.IF, k.T, R, Rout, nullptr);
  return cudaGetLastError();
}

// Alg. 2 lines 6-9 on the wide path: A^ = V^ R0^{-T} from the V slices (eq. 19 by linearity), the
// fit terms, lambda and A = A^ / lambda.  work_rows: I x (R + 2) doubles.
template <typename TV>
cudaError_t launch_wide_finish(const TV* vw, int nparts, int64_t I, int C, int R, const double* R0, double beta,
                               double alpha, double* A, double* lambda, double* fit_terms, double* work_rows,
                               unsigned int* status, cudaStream_t st) {
  if (!wide_supported(R)) return cudaErrorInvalidValue;
  cudaError_t e = set_smem_attrs();
  if (e != cudaSuccess) return e;
  double* Ahat = work_rows;
  double* fitrow = work_rows + I * R;
  wide_finish_prep_kernel<TV><<<rows_grid(I), 256, tri_smem(R), st>>>(vw, nparts, I, C, R, R0, beta, alpha, Ahat,
                                                                      fitrow);
  wide_colnorm_kernel<<<R, 256, 0, st>>>(Ahat, I, R, A, lambda, fitrow, fit_terms, status);
  return cudaGetLastError();
}
template cudaError_t launch_wide_finish<float>(const float*, int, int64_t, int, int, const double*, double, double,
                                               double*, double*, double*, double*, unsigned int*, cudaStream_t);
template cudaError_t launch_wide_finish<double>(const double*, int, int64_t, int, int, const double*, double, double,
                                                double*, double*, double*, double*, unsigned int*, cudaStream_t);

}  // namespace cpqr
