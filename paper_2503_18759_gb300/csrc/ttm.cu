// CUDA-core kernels of the CP-ALS-QR hot path:
//  * the mode-k product T x_k Q^T (Section 2.1) on any node of the dimension
//    tree, FP64 or FP32 (the tensor-core variant for the full tensor lives in
//    ttm_tc.cu);
//  * V = Y_(n) [Q0 | Q0^{k-1}] (Alg. 3 line 7; eq. 19 is applied to V by
//    linearity in the finish kernel);
//  * ||X||^2 and the explicit residual ||X - [[lambda; A]]||^2 (Section 4.1).
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace cpqr {

namespace {

// ----------------------------------------------------------------------------
// Mode-k product: out[p, r, s] = sum_i T[p, i, s] Q[i, r].
// Output rows m = p * S + s are tiled by BM; every CTA computes all R <= 32
// columns; the contraction runs in KC-deep shared-memory tiles loaded with
// coalesced reads along s (S > 1) or along i (S == 1).
// ----------------------------------------------------------------------------
constexpr int BM = 64, KC = 32, NT = 256;

template <typename TT, typename TQ, typename TO>
__global__ void __launch_bounds__(NT) ttm_kernel(const TT* __restrict__ T, const TQ* __restrict__ Q,
                                                 TO* __restrict__ out, int64_t P, int64_t K, int64_t S,
                                                 int R) {
  __shared__ TQ sT[KC][BM + 1];
  __shared__ TQ sQ[KC][CPQR_MAXR];
  const int tid = threadIdx.x;
  const int64_t M = P * S;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int ml = tid % BM, rg = tid / BM;  // compute mapping: row ml, columns rg*8..rg*8+7
  TQ acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = TQ(0);

  // per-thread row for the S > 1 load mapping (ml fixed per thread)
  const int64_t mrow = m0 + ml;
  int64_t p_ld = 0, s_ld = 0;
  if (S > 1 && mrow < M) {
    p_ld = mrow / S;
    s_ld = mrow - p_ld * S;
  }
  for (int64_t i0 = 0; i0 < K; i0 += KC) {
    if (S == 1) {
#pragma unroll
      for (int q = 0; q < (KC * BM) / NT; ++q) {
        int e = tid + NT * q;
        int i = e % KC, mm = e / KC;
        int64_t m = m0 + mm, ii = i0 + i;
        TQ v = TQ(0);
        if (m < M && ii < K) v = (TQ)T[m * K + ii];
        sT[i][mm] = v;
      }
    } else {
#pragma unroll
      for (int q = 0; q < (KC * BM) / NT; ++q) {
        int i = tid / BM + (NT / BM) * q;
        int64_t ii = i0 + i;
        TQ v = TQ(0);
        if (mrow < M && ii < K) v = (TQ)T[(p_ld * K + ii) * S + s_ld];
        sT[i][ml] = v;
      }
    }
#pragma unroll
    for (int q = 0; q < (KC * CPQR_MAXR) / NT; ++q) {
      int e = tid + NT * q;
      int i = e / CPQR_MAXR, r = e % CPQR_MAXR;
      int64_t ii = i0 + i;
      sQ[i][r] = (r < R && ii < K) ? Q[ii * R + r] : TQ(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int i = 0; i < KC; ++i) {
      TQ x = sT[i][ml];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += x * sQ[i][rg * 8 + j];
    }
    __syncthreads();
  }
  if (mrow < M) {
    if (S == 1) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int r = rg * 8 + j;
        if (r < R) out[mrow * R + r] = (TO)acc[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int r = rg * 8 + j;
        if (r < R) out[(p_ld * R + r) * S + s_ld] = (TO)acc[j];
      }
    }
  }
}

// ----------------------------------------------------------------------------
// FP32 mode-k product for the deeper tree levels, register-tiled: a CTA computes
// 128 output rows x 32 columns with a 4 x 4 tile per thread from KC-deep shared
// memory chunks (A stored k-major, B = Q rows), double buffered through registers.
// Rows are s (S % 4 == 0, one p per tile, float4 loads along s) or p (S == 1, the
// plain GEMM out[p, :] = T[p, :] Q, float4 loads along i, K % 4 == 0).
// ----------------------------------------------------------------------------
constexpr int TBM = 128, TKC = 16, TNT = 256;

template <bool LASTMODE>
__global__ void __launch_bounds__(TNT) ttm_f32_tiled_kernel(const float* __restrict__ T, const float* __restrict__ Q,
                                                             float* __restrict__ out, int64_t P, int64_t K, int64_t S,
                                                             int R, int64_t sblocks) {
  __shared__ __align__(16) float sA[2][TKC][TBM];
  __shared__ __align__(16) float sB[2][TKC][CPQR_MAXR];
  const int tid = threadIdx.x;
  const int tx = tid & 7, ty = tid >> 3;  // columns tx*4.., rows ty*4..
  int64_t p = 0, m0 = 0;
  if (LASTMODE) {
    m0 = (int64_t)blockIdx.x * TBM;  // rows are p
  } else {
    p = (int64_t)blockIdx.x / sblocks;
    m0 = ((int64_t)blockIdx.x % sblocks) * TBM;  // rows are s
  }
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  // loader mapping: A chunk = TKC x TBM floats = 512 float4, 2 per thread; B chunk 128 float4
  float4 ra[2], rb;
  auto load = [&](int64_t i0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + TNT * q;  // 0..511
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (LASTMODE) {
        const int m = e >> 2, kq = (e & 3) * 4;  // row m, k = kq..kq+3
        const int64_t row = m0 + m, ii = i0 + kq;
        if (row < P && ii < K) v = *reinterpret_cast<const float4*>(T + row * K + ii);
      } else {
        const int k = e >> 5, mq = (e & 31) * 4;  // k, rows mq..mq+3 (s)
        const int64_t ii = i0 + k, ss = m0 + mq;
        if (ii < K && ss < S) v = *reinterpret_cast<const float4*>(T + (p * K + ii) * S + ss);
      }
      ra[q] = v;
    }
    {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tid < TKC * CPQR_MAXR / 4) {
        const int k = tid >> 3, rq = (tid & 7) * 4;
        const int64_t ii = i0 + k;
        if (ii < K) {
          const float* q = Q + ii * R + rq;
          v.x = (rq + 0 < R) ? q[0] : 0.f;
          v.y = (rq + 1 < R) ? q[1] : 0.f;
          v.z = (rq + 2 < R) ? q[2] : 0.f;
          v.w = (rq + 3 < R) ? q[3] : 0.f;
        }
      }
      rb = v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + TNT * q;
      if (LASTMODE) {
        const int m = e >> 2, kq = (e & 3) * 4;
        sA[buf][kq + 0][m] = ra[q].x;
        sA[buf][kq + 1][m] = ra[q].y;
        sA[buf][kq + 2][m] = ra[q].z;
        sA[buf][kq + 3][m] = ra[q].w;
      } else {
        const int k = e >> 5, mq = (e & 31) * 4;
        *reinterpret_cast<float4*>(&sA[buf][k][mq]) = ra[q];
      }
    }
    if (tid < TKC * CPQR_MAXR / 4) {
      const int k = tid >> 3, rq = (tid & 7) * 4;
      *reinterpret_cast<float4*>(&sB[buf][k][rq]) = rb;
    }
  };
  const int nchunks = (int)((K + TKC - 1) / TKC);
  load(0);
  store(0);
  __syncthreads();
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    if (c + 1 < nchunks) load((int64_t)(c + 1) * TKC);
#pragma unroll
    for (int k = 0; k < TKC; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&sA[buf][k][ty * 4]);
      const float4 bq = *reinterpret_cast<const float4*>(&sB[buf][k][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (c + 1 < nchunks) store(buf ^ 1);
    __syncthreads();
  }
  if (LASTMODE) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t row = m0 + ty * 4 + i;
      const int r0 = tx * 4;
      if (row >= P) continue;
      if (r0 + 3 < R && (R % 4) == 0) {
        *reinterpret_cast<float4*>(out + row * R + r0) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (r0 + j < R) out[row * R + r0 + j] = acc[i][j];
      }
    }
  } else {
    const int64_t s0 = m0 + ty * 4;
    if (s0 < S) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = tx * 4 + j;
        if (r < R)
          *reinterpret_cast<float4*>(out + (p * R + r) * S + s0) =
              make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
      }
    }
  }
}

// ----------------------------------------------------------------------------
// V[i, c] = sum_k Y[p, i, s] Qc[k, c], k = p*S + s, Qc = [Q0 | Q0prev].
// CTA tile: 64 rows i x 64 columns c (C <= 64) x one K chunk, staged through
// shared memory 32 k at a time; each thread keeps a 4 x 4 register tile.  Every
// chunk writes its partial sums to its own slice of a workspace; the finish
// preparation kernel adds the slices in a fixed order (deterministic, no
// atomics).  TQ = type of Q0 and of the slices (FP64 on the FP64 path; FP32
// copies on the split path, whose Y carries the split TTMs' 2^-16 relative
// error anyway).
// ----------------------------------------------------------------------------
constexpr int VI = 64, VC = 64, VK = 32;

template <typename TY, typename TA, typename TQ>
__global__ void __launch_bounds__(256) leaf_v_kernel(const TY* __restrict__ Y, int P, int I, int S,
                                                     const TQ* __restrict__ Q0,
                                                     const TQ* __restrict__ Q0p, int R, int C, int kchunk,
                                                     TQ* __restrict__ part) {
  __shared__ TA sY[VK][VI + 1];  // padded: the S > 1 fill walks k fastest
  __shared__ __align__(16) TA sQ[VK][VC];
  constexpr int NLY = (VK * VI) / 256, NLQ = (VK * VC) / 256;
  const int tid = threadIdx.x;
  // rows ty*4 .. +3, columns tx*4 .. +3.  For C <= 32 a warp holds two column groups, so the
  // warps whose columns all lie at or past C skip the multiply; wider C keeps two row groups per
  // warp (one shared-memory broadcast of the rows instead of one of the columns)
  const bool narrow = C <= 32;
  const int cb = blockIdx.z * VC;  // column tile (C > 64 on the wide-rank path)
  const int tx = narrow ? tid >> 4 : tid & 15, ty = narrow ? tid & 15 : tid >> 4;
  const bool busy = !narrow || (tid >> 5) * 8 < C;
  const int i0 = blockIdx.x * VI;
  const int K = P * S;
  const int kbeg = blockIdx.y * kchunk;
  const int kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
  TA acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = TA(0);
  pdl_wait();
  // the next chunk's operands are loaded into registers while the current one is multiplied
  TY ybuf[NLY];
  TQ qbuf[NLQ];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < NLY; ++q) {
      const int e = tid + 256 * q;
      // consecutive threads along the contiguous index: s (S > 1) or i (S == 1)
      const int kk = (S > 1) ? e % VK : e / VI, ii = (S > 1) ? e / VK : e % VI;
      const int k = k0 + kk, i = i0 + ii;
      ybuf[q] = TY(0);
      if (k < kend && i < I) {
        const int pp = k / S, ss = k - pp * S;
        ybuf[q] = Y[((int64_t)pp * I + i) * S + ss];
      }
    }
#pragma unroll
    for (int q = 0; q < NLQ; ++q) {
      const int e = tid + 256 * q;
      const int kk = e / VC, c = cb + e % VC;
      const int k = k0 + kk;
      qbuf[q] = TQ(0);
      if (k < kend && c < C) qbuf[q] = (c < R) ? Q0[(int64_t)k * R + c] : Q0p[(int64_t)k * R + (c - R)];
    }
  };
  if (kbeg < kend) fetch(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += VK) {
#pragma unroll
    for (int q = 0; q < NLY; ++q) {
      const int e = tid + 256 * q;
      const int kk = (S > 1) ? e % VK : e / VI, ii = (S > 1) ? e / VK : e % VI;
      sY[kk][ii] = (TA)ybuf[q];
    }
#pragma unroll
    for (int q = 0; q < NLQ; ++q) {
      const int e = tid + 256 * q;
      sQ[e / VC][e % VC] = (TA)qbuf[q];
    }
    __syncthreads();
    if (k0 + VK < kend) fetch(k0 + VK);
#pragma unroll 4
    for (int kk = 0; kk < (busy ? VK : 0); ++kk) {
      TA y[4], qv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        y[a] = sY[kk][ty * 4 + a];
        qv[a] = sQ[kk][tx * 4 + a];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += y[a] * qv[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty * 4 + a;
    if (i >= I) continue;
    TQ* dst = part + ((size_t)blockIdx.y * I + i) * C;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = cb + tx * 4 + b;
      if (c < C) dst[c] = (TQ)acc[a][b];
    }
  }
}

// ----------------------------------------------------------------------------
// Reductions in FP64.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

template <typename TX>
__global__ void norm2_kernel(const TX* __restrict__ X, int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)X[i];
    acc += v * v;
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// ||X||^2 of an FP32 tensor off the FP64 pipe (GB300 runs FP64 at 1/64 of FP32; one DFMA per
// element held the FP64 version at ~1 TB/s).  Each square is kept exactly as a float pair
// (p = x * x rounded, e = fma(x, x, -p) its error), and the pairs of a thread are summed in
// float-float (two-sum for the high part, the errors added into the low part) over runs of 16
// elements, whose sum then goes into an FP64 accumulator: the float-float error of a run is at
// most ~16 * 2^-48 of it.  Round-to-nearest intrinsics keep the compiler from contracting the
// error-free steps.  Values whose square (or a run of 16 squares) would leave FP32's normal range
// (|x| >= 1e18, or 0 < |x| < 1e-15, where the product's error term would be subnormal), NaN and
// Inf, are squared in FP64 instead.
__global__ void norm2_f32_kernel(const float* __restrict__ X, int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  float hi = 0.f, lo = 0.f;
  int run = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float x = X[i];
    const float ax = fabsf(x);
    if (!(ax < 1e18f && (ax >= 1e-15f || x == 0.f))) {
      acc += (double)x * (double)x;
      continue;
    }
    const float p = __fmul_rn(x, x);
    const float e = fmaf(x, x, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(t, e));
    if (++run == 16) {
      acc += (double)hi + (double)lo;
      hi = lo = 0.f;
      run = 0;
    }
  }
  acc += (double)hi + (double)lo;
  double tt = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tt;
}

// Sum of the block partials in a fixed order (the same ||X||^2 in every context).
__global__ void sum_parts_kernel(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) out[0] = t;
}

// Explicit residual ||X - [[lambda; A]]||^2.  X is viewed as rows (modes 0..N-2) x I_last.
// The factors are first copied to FP32 (lambda folded into the first).  A CTA takes tiles of
// RT rows: the Khatri-Rao weights w[row, r] = prod_{n<N-1} A_n[i_n, r] go to shared memory,
// every thread holds one column l of A_last (R values) in registers and forms the model
// entries k = sum_r w[row, r] A_last[l, r] of its column for the RT rows, all in FP32; (x - k)^2
// is summed in FP32 per thread and the per-thread totals in FP64 (FP64 runs at 1/64 of FP32 on
// GB300: it stays out of the per-element work).  Rounding of w and k (~(N + R) 2^-24 |k|)
// perturbs ||X - K||^2 by a relative ~1e-6 at a 1e-3 residual, the fit by ~1e-9.
struct ResParams {
  int N, R;
  int d[CPQR_MAXN];
  const float* A[CPQR_MAXN];  // FP32 copies, lambda folded into A[0]
};

__global__ void factors_to_f32_kernel(ResParams rp, const double* const* A64, const double* __restrict__ lambda,
                                      float* __restrict__ dst, int total) {
  // dst holds A_0 .. A_{N-2} back to back (I_n x R each), then A_{N-1} transposed (R x I_{N-1})
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int off = 0, n = 0;
    while (e >= off + rp.d[n] * rp.R) {
      off += rp.d[n] * rp.R;
      ++n;
    }
    const int loc = e - off;
    double v = A64[n][loc];
    if (n == 0) v *= lambda[loc % rp.R];
    int o = e;
    if (n == rp.N - 1) {
      const int i = loc / rp.R, r = loc % rp.R;
      o = off + r * rp.d[n] + i;
    }
    dst[o] = (float)v;
  }
}

// Work items of 128 rows x 64 columns of X, numbered row tile major; every CTA takes one
// contiguous range of items, so all CTAs get the same number of items (to within one).
// The Khatri-Rao weights w[row, r] = prod_{n<N-1} A_n[i_n, r] of a row tile are formed in
// shared memory when the CTA enters the tile and are reused by all of its column items:
// lane = r, so every factor row is one coalesced 128-byte load, and every thread writes four
// rows at once into sW[r][row], the row index XOR-swizzled by (r mod 8) * 4 (groups of four
// rows stay contiguous; the 128-bit stores and reads are conflict-free).  The A_last^T chunk
// of the next item is prefetched into registers during the product and stored into the other
// of two buffers.  Each warp computes a 32 x 32 block of model entries K = W A_last^T, 8 rows x
// 4 columns per thread (three 128-bit shared loads per 32 FMAs), with the thread's X values
// loaded before the product, and accumulates (x - k)^2.
constexpr int RM = 128, RC = 64, RNT = 256;

__device__ __forceinline__ int wswz(int r, int row) { return row ^ ((r & 7) << 2); }

template <typename TX>
__global__ void __launch_bounds__(RNT, 2) residual2_kernel(const TX* __restrict__ X, const __grid_constant__ ResParams rp,
                                                           int rows, double* __restrict__ out) {
  __shared__ __align__(16) float sW[CPQR_MAXR][RM];
  __shared__ __align__(16) float sA[2][CPQR_MAXR][RC];
  __shared__ double sh[32];
  const int R = rp.R, N = rp.N;
  const int Il = rp.d[N - 1];
  const int nchunks = (Il + RC - 1) / RC;
  const int64_t total = (int64_t)((rows + RM - 1) / RM) * nchunks;
  const int64_t u0 = total * blockIdx.x / gridDim.x, u1 = total * (blockIdx.x + 1) / gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tx = lane & 7, ty = lane >> 3;
  const int rloc = (warp >> 1) * 32 + ty * 8;  // first of this thread's 8 rows in the tile
  const int cloc = (warp & 1) * 32 + tx * 4;   // first of its 4 columns in the item
  const bool vec4 = std::is_same<TX, float>::value && (Il % 4) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  const float* AlT = rp.A[N - 1];  // R x I_last

  // A_last^T chunk q: element e = threadIdx.x + 256 j is (r = e / 64, column e % 64)
  // element j of a thread: r = threadIdx.x / 64 + 4 j, column threadIdx.x % 64 of the chunk
  const int ar = threadIdx.x / RC, ac = threadIdx.x % RC;
  float an[8];
  auto loadA = [&](int q) {
    const int col = q * RC + ac;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = ar + 4 * j;
      an[j] = (r < R && col < Il) ? AlT[(int64_t)r * Il + col] : 0.f;
    }
  };
  auto storeA = [&](int buf) {
#pragma unroll
    for (int j = 0; j < 8; ++j) sA[buf][ar + 4 * j][ac] = an[j];
  };
  // rows of sW and sA beyond R hold zeros, so the product may run over R rounded up to 8
  const int R8 = (R + 7) & ~7;
  double acc = 0.0;
  int cur_rt = -1, buf = 0;
  int rt = (int)(u0 / nchunks), q = (int)(u0 % nchunks);  // item u0; advanced incrementally
  if (u0 < u1) {
    loadA(q);
    storeA(0);
  }
  for (int64_t u = u0; u < u1; ++u) {
    const int r0 = rt * RM;
    if (rt != cur_rt) {
      __syncthreads();  // every warp is done with the previous tile's weights
      // rows r0 + 4g .. r0 + 4g + 3 for g = warp, warp + 8, warp + 16, warp + 24; r = lane
#pragma unroll
      for (int gg = 0; gg < 4; ++gg) {
        const int g = warp + 8 * gg;
        float w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int row = r0 + 4 * g + i;
          float v = 0.f;
          if (row < rows && lane < R) {
            v = 1.f;
            int x = row;
            for (int n = N - 2; n > 0; --n) {
              const int qd = x / rp.d[n];
              v *= rp.A[n][(int64_t)(x - qd * rp.d[n]) * R + lane];
              x = qd;
            }
            v *= rp.A[0][(int64_t)x * R + lane];
          }
          w[i] = v;
        }
        *reinterpret_cast<float4*>(&sW[lane][wswz(lane, 4 * g)]) = make_float4(w[0], w[1], w[2], w[3]);
      }
      cur_rt = rt;
    }
    __syncthreads();  // weights and sA[buf] complete
    // X values of this thread's 8 x 4 block, issued before the product
    const int cb = q * RC + cloc;
    float xv[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int xrow = r0 + rloc + i;
#pragma unroll
      for (int j = 0; j < 4; ++j) xv[i][j] = 0.f;
      if (xrow >= rows) continue;
      const TX* xr = X + (int64_t)xrow * Il + cb;
      if (vec4) {
        if (cb < Il) {  // Il % 4 == 0: the whole float4 is inside the row
          const float4 x4 = *reinterpret_cast<const float4*>(xr);
          xv[i][0] = x4.x; xv[i][1] = x4.y; xv[i][2] = x4.z; xv[i][3] = x4.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (cb + j < Il) xv[i][j] = (float)xr[j];
      }
    }
    const bool more = u + 1 < u1;
    const int qn = (q + 1 == nchunks) ? 0 : q + 1;
    if (more) loadA(qn);
    float k[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) k[i][j] = 0.f;
    for (int rb = 0; rb < R8; rb += 8) {
#pragma unroll
      for (int t = 0; t < 8; ++t) {  // r = rb + t, so r mod 8 = t is known here
        const int r = rb + t;
        const float4 w0 = *reinterpret_cast<const float4*>(&sW[r][wswz(t, rloc)]);
        const float4 w1 = *reinterpret_cast<const float4*>(&sW[r][wswz(t, rloc + 4)]);
        const float4 a4 = *reinterpret_cast<const float4*>(&sA[buf][r][cloc]);
        const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w}, av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) k[i][j] = fmaf(wv[i], av[j], k[i][j]);
      }
    }
    // entries outside X have x = 0 and k = 0 (zero weights / zero A_last columns)
    float racc = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float e = xv[i][j] - k[i][j];
        racc = fmaf(e, e, racc);
      }
    acc += (double)racc;
    if (more) storeA(buf ^ 1);  // that buffer was last read in the previous item, before this item's barrier
    buf ^= 1;
    q = qn;
    if (q == 0) ++rt;
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = t;  // per-block partial, summed in a fixed order afterwards
}

// The residual for ranks above 32 (the wide-rank path): 64 x 64 tiles of X (rows = modes 0..N-2,
// columns = the last mode), the model tile K = W A_last^T in FP32 over R in 16-deep chunks, the
// Khatri-Rao weights W of each chunk formed in shared memory from the FP32 factors, and the
// (x - k)^2 of the tile summed per thread in FP32 and per block in FP64 (one partial per block,
// added in a fixed order afterwards).
constexpr int WRT = 64, WRK = 16;

template <typename TX>
__global__ void __launch_bounds__(256) residual_wide_kernel(const TX* __restrict__ X, const __grid_constant__ ResParams rp,
                                                           int64_t rows, double* __restrict__ part) {
  __shared__ float sW[WRK][WRT + 1];
  __shared__ float sA[WRK][WRT + 1];
  __shared__ double sh[32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int Il = rp.d[rp.N - 1], R = rp.R;
  const int64_t rtiles = (rows + WRT - 1) / WRT, ctiles = (Il + WRT - 1) / WRT;
  const float* AlT = rp.A[rp.N - 1];  // R x I_last
  double acc_tot = 0.0;
  for (int64_t t = blockIdx.x; t < rtiles * ctiles; t += gridDim.x) {
    const int64_t r0 = (t / ctiles) * WRT, c0 = (t % ctiles) * WRT;
    float k[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) k[i][j] = 0.f;
    for (int q0 = 0; q0 < R; q0 += WRK) {
      for (int e = tid; e < WRK * WRT; e += 256) {
        const int rr = e / WRT, m = e % WRT;
        const int r = q0 + rr;
        const int64_t row = r0 + m;
        float w = 0.f;
        if (r < R && row < rows) {
          w = 1.f;
          int64_t x = row;
          for (int n = rp.N - 2; n >= 0; --n) {
            const int in = (int)(x % rp.d[n]);
            x /= rp.d[n];
            w *= rp.A[n][(int64_t)in * R + r];
          }
        }
        sW[rr][m] = w;
        const int64_t col = c0 + m;
        sA[rr][m] = (r < R && col < Il) ? AlT[(int64_t)r * Il + col] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int rr = 0; rr < WRK; ++rr) {
        float a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          a[i] = sW[rr][ty * 4 + i];
          bb[i] = sA[rr][tx * 4 + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) k[i][j] = fmaf(a[i], bb[j], k[i][j]);
      }
      __syncthreads();
    }
    float racc = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t row = r0 + ty * 4 + i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t col = c0 + tx * 4 + j;
        if (row < rows && col < Il) {
          const float e = (float)X[row * Il + col] - k[i][j];
          racc = fmaf(e, e, racc);
        }
      }
    }
    acc_tot += (double)racc;
  }
  double tsum = block_sum(acc_tot, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tsum;
}

__global__ void to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

int grid_for(int64_t n, int per) {
  int64_t g = (n + per - 1) / per;
  if (g < 1) g = 1;
  if (g > 152 * 8) g = 152 * 8;
  return (int)g;
}

}  // namespace

template <typename TT, typename TQ, typename TO>
cudaError_t launch_ttm(const TT* T, const TQ* Q, TO* out, int64_t P, int64_t K, int64_t S, int R,
                       cudaStream_t st) {
  if (R < 1 || R > CPQR_MAXR || P < 1 || K < 1 || S < 1) return cudaErrorInvalidValue;
  int64_t tiles = (P * S + BM - 1) / BM;
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  ttm_kernel<TT, TQ, TO><<<(unsigned)tiles, NT, 0, st>>>(T, Q, out, P, K, S, R);
  return cudaGetLastError();
}

template cudaError_t launch_ttm<double, double, double>(const double*, const double*, double*, int64_t, int64_t,
                                                        int64_t, int, cudaStream_t);
template cudaError_t launch_ttm<float, double, double>(const float*, const double*, double*, int64_t, int64_t,
                                                       int64_t, int, cudaStream_t);
template cudaError_t launch_ttm<float, float, float>(const float*, const float*, float*, int64_t, int64_t, int64_t,
                                                     int, cudaStream_t);

cudaError_t launch_ttm_f32_tiled(const float* T, const float* Q, float* out, int64_t P, int64_t K, int64_t S, int R,
                                 cudaStream_t st) {
  if (R < 1 || R > CPQR_MAXR || P < 1 || K < 1 || S < 1) return cudaErrorInvalidValue;
  // float4 accesses: the tensor and the output must be 16-byte aligned
  if ((reinterpret_cast<uintptr_t>(T) & 15) || (reinterpret_cast<uintptr_t>(out) & 15)) return cudaErrorNotSupported;
  if (S == 1) {
    if (K % 4) return cudaErrorNotSupported;
    const int64_t blocks = (P + TBM - 1) / TBM;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    ttm_f32_tiled_kernel<true><<<(unsigned)blocks, TNT, 0, st>>>(T, Q, out, P, K, S, R, 1);
  } else {
    if (S % 4) return cudaErrorNotSupported;
    const int64_t sb = (S + TBM - 1) / TBM;
    const int64_t blocks = P * sb;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    ttm_f32_tiled_kernel<false><<<(unsigned)blocks, TNT, 0, st>>>(T, Q, out, P, K, S, R, sb);
  }
  return cudaGetLastError();
}

int leaf_v_splits(int64_t I, int64_t K) {
  // split K so that the grid covers the GPU about twice (at least one VK chunk per split)
  const int64_t itiles = (I + VI - 1) / VI;
  int64_t want = (2 * 152 + itiles - 1) / itiles;
  const int64_t maxs = (K + VK - 1) / VK;
  if (want > maxs) want = maxs;
  if (want < 1) want = 1;
  return (int)want;
}

template <typename TY, typename TQ>
cudaError_t launch_leaf_v(const TY* Y, int64_t P, int64_t I, int64_t S, const TQ* Q0, const TQ* Q0prev, int R, int C,
                          TQ* work, int* nparts, cudaStream_t st) {
  const int64_t K = P * S;
  if (K > 0x7fffffff || I > 0x7fffffff) return cudaErrorInvalidValue;
  if (C < 1 || C > 2 * 192 || R < 1 || R > 192) return cudaErrorInvalidValue;  // wide-rank path: R <= 192
  const int64_t itiles = (I + VI - 1) / VI;
  const int splits = leaf_v_splits(I, K);
  int64_t kchunk = (K + splits - 1) / splits;
  kchunk = ((kchunk + VK - 1) / VK) * VK;
  if (kchunk < VK) kchunk = VK;
  const int64_t ktiles = (K + kchunk - 1) / kchunk;  // <= splits: fits the work slices
  dim3 grid((unsigned)itiles, (unsigned)ktiles, (unsigned)((C + VC - 1) / VC));
  using TA = typename std::conditional<std::is_same<TY, double>::value, double, float>::type;
  *nparts = (int)ktiles;
  return launch_pdl(leaf_v_kernel<TY, TA, TQ>, grid, dim3(256), 0, st, Y, (int)P, (int)I, (int)S, Q0, Q0prev, R, C,
                    (int)kchunk, work);
}

template cudaError_t launch_leaf_v<double, double>(const double*, int64_t, int64_t, int64_t, const double*,
                                                   const double*, int, int, double*, int*, cudaStream_t);
template cudaError_t launch_leaf_v<float, float>(const float*, int64_t, int64_t, int64_t, const float*, const float*,
                                                 int, int, float*, int*, cudaStream_t);

template <typename TX>
cudaError_t launch_norm2(const TX* X, int64_t n, double* out, double* work, cudaStream_t st) {
  if (!work) return cudaErrorInvalidValue;
  const int g = grid_for(n, 256 * 16);  // <= norm2_work_doubles()
  if constexpr (std::is_same<TX, float>::value) norm2_f32_kernel<<<g, 256, 0, st>>>(X, n, work);
  else norm2_kernel<TX><<<g, 256, 0, st>>>(X, n, work);
  sum_parts_kernel<<<1, 256, 0, st>>>(work, g, out);
  return cudaGetLastError();
}

size_t norm2_work_doubles() { return 152 * 8; }

cudaError_t launch_sum_parts(const double* part, int np, double* out, cudaStream_t st) {
  sum_parts_kernel<<<1, 256, 0, st>>>(part, np, out);
  return cudaGetLastError();
}

constexpr int kResidualParts = 1024;  // partial-sum slots of the residual passes (grids <= 2 x 152 CTAs)
template cudaError_t launch_norm2<float>(const float*, int64_t, double*, double*, cudaStream_t);
template cudaError_t launch_norm2<double>(const double*, int64_t, double*, double*, cudaStream_t);

size_t residual2_work_bytes(int N, const int64_t* d, int R) {
  int64_t total = 0;
  for (int n = 0; n < N; ++n) total += d[n] * R;
  return (size_t)((total + 3) / 4) * 16 + CPQR_MAXN * sizeof(double*) + 64 + kResidualParts * sizeof(double);
}

template <typename TX>
cudaError_t launch_residual2(const TX* X, int N, const int64_t* d, const double* const* A, const double* lambda,
                             int R, double* out, double* work, unsigned int* dev_status, cudaStream_t st, int parts,
                             int reserve_sms) {
  // work: >= sum_n d[n] * R floats + N pointers (device)
  ResParams rp{};
  rp.N = N;
  rp.R = R;
  int64_t rows = 1, total = 0;
  for (int n = 0; n < N; ++n) {
    if (d[n] > 0x7fffffff) return cudaErrorInvalidValue;
    rp.d[n] = (int)d[n];
    if (n < N - 1) rows *= d[n];
    total += d[n] * R;
  }
  if (rows > 0x7fffffff || total > 0x7fffffff) return cudaErrorInvalidValue;
  float* f32 = reinterpret_cast<float*>(work);
  const double** ptrs = reinterpret_cast<const double**>(f32 + ((total + 3) / 4) * 4);
  // per-CTA partial sums after the pointers (8-byte aligned: the float block is a multiple of 16 bytes)
  double* part = reinterpret_cast<double*>(ptrs + CPQR_MAXN) + 8;
  int64_t off = 0;
  for (int n = 0; n < N; ++n) {
    rp.A[n] = f32 + off;
    off += d[n] * R;
  }
  cudaError_t e = cudaSuccess;
  if (parts & RESIDUAL_SNAPSHOT) {
    e = cudaMemcpyAsync(ptrs, A, N * sizeof(double*), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    factors_to_f32_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 512), 256, 0, st>>>(rp, ptrs, lambda, f32,
                                                                                           (int)total);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (!(parts & RESIDUAL_EVALUATE)) return cudaSuccess;
  if (std::is_same<TX, float>::value && residual_tc_supported(N, d, R, X)) {
    int np = 0;
    e = launch_residual_tc(reinterpret_cast<const float*>(X), N, d, rp.A, R, part, kResidualParts, &np, dev_status,
                           st, reserve_sms);
    if (e == cudaSuccess) return launch_sum_parts(part, np, out, st);
    if (e != cudaErrorNotSupported) return e;
  }
  if (R > CPQR_MAXR) {  // the wide-rank path
    const int64_t tiles = ((rows + WRT - 1) / WRT) * ((d[N - 1] + WRT - 1) / WRT);
    const int grid = (int)std::min<int64_t>(tiles, 152 * 4);
    residual_wide_kernel<TX><<<grid, 256, 0, st>>>(X, rp, rows, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_sum_parts(part, grid, out, st);
  }
  // contiguous ranges of (row tile, column chunk) items, two CTAs per SM
  const int64_t items = ((rows + RM - 1) / RM) * ((d[N - 1] + RC - 1) / RC);
  const int grid = (int)std::min<int64_t>(items, 152 * 2);
  residual2_kernel<TX><<<grid, RNT, 0, st>>>(X, rp, (int)rows, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sum_parts(part, grid, out, st);
}
template cudaError_t launch_residual2<float>(const float*, int, const int64_t*, const double* const*, const double*,
                                             int, double*, double*, unsigned int*, cudaStream_t, int, int);
template cudaError_t launch_residual2<double>(const double*, int, const int64_t*, const double* const*,
                                              const double*, int, double*, double*, unsigned int*, cudaStream_t, int,
                                              int);

cudaError_t launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t st) {
  to_f32_kernel<<<grid_for(n, 256 * 4), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

}  // namespace cpqr
