// CUDA-core kernels of the CP-ALS-QR hot path:
//  * the mode-k product T x_k Q^T (Section 2.1) on any node of the dimension
//    tree, FP64 or FP32 (the tensor-core variant for the full tensor lives in
//    ttm_tc.cu);
//  * V = Y_(n) [Q0 | Q0^{k-1}] (Alg. 3 line 7; eq. 19 is applied to V by
//    linearity in the finish kernel);
//  * ||X||^2 and the explicit residual ||X - [[lambda; A]]||^2 (Section 4.1).
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
// V[i, c] = sum_k Y[p, i, s] Qc[k, c], k = p*S + s, Qc = [Q0 | Q0prev].
// CTA tile: 32 rows i x C <= 64 columns x one K chunk; partial sums are added
// to V with FP64 atomics.
// ----------------------------------------------------------------------------
constexpr int VI = 32, VK = 32;

template <typename TY, typename TA>
__global__ void __launch_bounds__(256) leaf_v_kernel(const TY* __restrict__ Y, int64_t P, int64_t I, int64_t S,
                                                     const double* __restrict__ Q0,
                                                     const double* __restrict__ Q0p, int R, int C,
                                                     int64_t kchunk, double* __restrict__ V) {
  __shared__ TA sY[VK][VI + 1];
  __shared__ TA sQ[VK][2 * CPQR_MAXR];
  const int tid = threadIdx.x;
  const int il = tid % VI, cgp = tid / VI;  // row il, columns cgp*8 .. cgp*8+7
  const int64_t i0 = (int64_t)blockIdx.x * VI;
  const int64_t K = P * S;
  const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
  const int64_t kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
  TA acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = TA(0);
  for (int64_t k0 = kbeg; k0 < kend; k0 += VK) {
#pragma unroll
    for (int q = 0; q < (VK * VI) / 256; ++q) {
      int e = tid + 256 * q;
      int kk = e % VK, ii = e / VK;
      int64_t k = k0 + kk, i = i0 + ii;
      TA v = TA(0);
      if (k < kend && i < I) {
        int64_t p = k / S, s = k - p * S;
        v = (TA)Y[(p * I + i) * S + s];
      }
      sY[kk][ii] = v;
    }
#pragma unroll
    for (int q = 0; q < (VK * 2 * CPQR_MAXR) / 256; ++q) {
      int e = tid + 256 * q;
      int kk = e / (2 * CPQR_MAXR), c = e % (2 * CPQR_MAXR);
      int64_t k = k0 + kk;
      TA v = TA(0);
      if (k < kend && c < C) v = (TA)((c < R) ? Q0[k * R + c] : Q0p[k * R + (c - R)]);
      sQ[kk][c] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < VK; ++kk) {
      TA y = sY[kk][il];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += y * sQ[kk][cgp * 8 + j];
    }
    __syncthreads();
  }
  const int64_t i = i0 + il;
  if (i < I) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int c = cgp * 8 + j;
      if (c < C) atomicAdd(&V[i * C + c], (double)acc[j]);
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
__global__ void norm2_kernel(const TX* __restrict__ X, int64_t n, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)X[i];
    acc += v * v;
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) atomicAdd(out, t);
}

// Explicit residual: X viewed as (rows = prod of modes 0..N-2) x (I_last); every
// CTA takes one row, forms w_r = lambda_r prod_{n<N-1} A_n[i_n, r] in FP64 and the
// model entries k = sum_r w_r A_last[l, r] in FP64; (x - k)^2 summed in FP64.
struct ResParams {
  int N, R;
  int64_t d[CPQR_MAXN];
  const double* A[CPQR_MAXN];
  const double* lambda;
};

template <typename TX>
__global__ void residual2_kernel(const TX* __restrict__ X, ResParams rp, int64_t rows, double* __restrict__ out) {
  __shared__ double w[CPQR_MAXR];
  __shared__ double sh[32];
  const int R = rp.R, N = rp.N;
  const int64_t Il = rp.d[N - 1];
  double acc = 0.0;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    if (threadIdx.x < R) {
      double v = rp.lambda[threadIdx.x];
      int64_t x = row;
      for (int n = N - 2; n >= 0; --n) {
        int64_t in = x % rp.d[n];
        x /= rp.d[n];
        v *= rp.A[n][in * R + threadIdx.x];
      }
      w[threadIdx.x] = v;
    }
    __syncthreads();
    for (int64_t l = threadIdx.x; l < Il; l += blockDim.x) {
      double k = 0.0;
      const double* al = rp.A[N - 1] + l * R;
      for (int r = 0; r < R; ++r) k += w[r] * al[r];
      double e = (double)X[row * Il + l] - k;
      acc += e * e;
    }
    __syncthreads();
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) atomicAdd(out, t);
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

template <typename TY>
cudaError_t launch_leaf_v(const TY* Y, int64_t P, int64_t I, int64_t S, const double* Q0, const double* Q0prev,
                          int R, int C, double* V, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(V, 0, sizeof(double) * I * C, st);
  if (e != cudaSuccess) return e;
  const int64_t K = P * S;
  const int64_t itiles = (I + VI - 1) / VI;
  // split K so that the grid covers the GPU about twice
  int64_t want = (2 * 152 + itiles - 1) / itiles;
  int64_t kchunk = (K + want - 1) / want;
  kchunk = ((kchunk + VK - 1) / VK) * VK;
  if (kchunk < VK) kchunk = VK;
  const int64_t ktiles = (K + kchunk - 1) / kchunk;
  dim3 grid((unsigned)itiles, (unsigned)ktiles);
  using TA = typename std::conditional<std::is_same<TY, double>::value, double, float>::type;
  leaf_v_kernel<TY, TA><<<grid, 256, 0, st>>>(Y, P, I, S, Q0, Q0prev, R, C, kchunk, V);
  return cudaGetLastError();
}

template cudaError_t launch_leaf_v<double>(const double*, int64_t, int64_t, int64_t, const double*, const double*,
                                           int, int, double*, cudaStream_t);
template cudaError_t launch_leaf_v<float>(const float*, int64_t, int64_t, int64_t, const double*, const double*,
                                          int, int, double*, cudaStream_t);

template <typename TX>
cudaError_t launch_norm2(const TX* X, int64_t n, double* out, double* /*work*/, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  norm2_kernel<TX><<<grid_for(n, 256 * 16), 256, 0, st>>>(X, n, out);
  return cudaGetLastError();
}
template cudaError_t launch_norm2<float>(const float*, int64_t, double*, double*, cudaStream_t);
template cudaError_t launch_norm2<double>(const double*, int64_t, double*, double*, cudaStream_t);

template <typename TX>
cudaError_t launch_residual2(const TX* X, int N, const int64_t* d, const double* const* A, const double* lambda,
                             int R, double* out, double* /*work*/, cudaStream_t st) {
  ResParams rp{};
  rp.N = N;
  rp.R = R;
  int64_t rows = 1;
  for (int n = 0; n < N; ++n) {
    rp.d[n] = d[n];
    rp.A[n] = A[n];
    if (n < N - 1) rows *= d[n];
  }
  rp.lambda = lambda;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  int grid = (int)((rows < 152 * 16) ? rows : 152 * 16);
  residual2_kernel<TX><<<grid, 256, 0, st>>>(X, rp, rows, out);
  return cudaGetLastError();
}
template cudaError_t launch_residual2<float>(const float*, int, const int64_t*, const double* const*, const double*,
                                             int, double*, double*, cudaStream_t);
template cudaError_t launch_residual2<double>(const double*, int, const int64_t*, const double* const*,
                                              const double*, int, double*, double*, cudaStream_t);

cudaError_t launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t st) {
  to_f32_kernel<<<grid_for(n, 256 * 4), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

}  // namespace cpqr
