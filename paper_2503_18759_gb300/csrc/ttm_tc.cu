// Split-precision staging for the tensor-core TTM of the full tensor.
//
// X (FP32) is stored once as two bf16 arrays, X = hi + lo + O(2^-16 |X|):
// hi = bf16(X), lo = bf16(X - hi).  Each Q_k (FP64) is staged after its QR as
// bf16 hi/lo of Q_k^T, zero-padded to Rp x Kp (the MMA's N x K operand, K
// contiguous).  The product keeps hi*hi + hi*lo + lo*hi and drops lo*lo.
#include "common.cuh"

namespace cpqr {

namespace {

__global__ void split_x_kernel(const float* __restrict__ X, __nv_bfloat16* __restrict__ hi,
                               __nv_bfloat16* __restrict__ lo, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // 4 elements per thread per iteration when aligned
  const int64_t n4 = n / 4;
  const float4* X4 = reinterpret_cast<const float4*>(X);
  for (int64_t q = i; q < n4; q += stride) {
    float4 v = X4[q];
    __nv_bfloat16 h0 = __float2bfloat16_rn(v.x), h1 = __float2bfloat16_rn(v.y);
    __nv_bfloat16 h2 = __float2bfloat16_rn(v.z), h3 = __float2bfloat16_rn(v.w);
    __nv_bfloat16 l0 = __float2bfloat16_rn(v.x - __bfloat162float(h0));
    __nv_bfloat16 l1 = __float2bfloat16_rn(v.y - __bfloat162float(h1));
    __nv_bfloat16 l2 = __float2bfloat16_rn(v.z - __bfloat162float(h2));
    __nv_bfloat16 l3 = __float2bfloat16_rn(v.w - __bfloat162float(h3));
    __nv_bfloat162 a0, a1, b0, b1;
    a0.x = h0; a0.y = h1; a1.x = h2; a1.y = h3;
    b0.x = l0; b0.y = l1; b1.x = l2; b1.y = l3;
    reinterpret_cast<__nv_bfloat162*>(hi)[2 * q] = a0;
    reinterpret_cast<__nv_bfloat162*>(hi)[2 * q + 1] = a1;
    reinterpret_cast<__nv_bfloat162*>(lo)[2 * q] = b0;
    reinterpret_cast<__nv_bfloat162*>(lo)[2 * q + 1] = b1;
  }
  for (int64_t q = 4 * n4 + i; q < n; q += stride) {
    float v = X[q];
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[q] = h;
    lo[q] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// Qt[0][r][i] = hi(Q[i][r]), Qt[1][r][i] = lo(Q[i][r]); zero outside R x K.
__global__ void split_q_kernel(const double* __restrict__ Q, int64_t K, int R, __nv_bfloat16* __restrict__ Qt,
                               int Rp, int64_t Kp) {
  const int64_t total = (int64_t)Rp * Kp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(e / Kp);
    int64_t i = e - (int64_t)r * Kp;
    float q = (r < R && i < K) ? (float)Q[i * R + r] : 0.f;
    __nv_bfloat16 h = __float2bfloat16_rn(q);
    __nv_bfloat16 l = __float2bfloat16_rn(q - __bfloat162float(h));
    Qt[e] = h;
    Qt[total + e] = l;
  }
}

}  // namespace

cudaError_t launch_split_x(const float* X, __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, int64_t n, cudaStream_t st) {
  if (((uintptr_t)X & 15) || ((uintptr_t)Xhi & 15) || ((uintptr_t)Xlo & 15)) {
    // the vector path needs 16-byte alignment; cudaMalloc gives 256
    return cudaErrorMisalignedAddress;
  }
  split_x_kernel<<<152 * 8, 256, 0, st>>>(X, Xhi, Xlo, n);
  return cudaGetLastError();
}

cudaError_t launch_split_q(const double* Q, int64_t K, int R, __nv_bfloat16* Qt, int Rp, int64_t Kp,
                           cudaStream_t st) {
  int64_t total = (int64_t)Rp * Kp;
  int grid = (int)std::min<int64_t>((total + 255) / 256, 1024);
  split_q_kernel<<<grid, 256, 0, st>>>(Q, K, R, Qt, Rp, Kp);
  return cudaGetLastError();
}

bool ttm_tc_supported(int64_t, int64_t, int64_t, int) { return false; }

cudaError_t launch_ttm_tc(const __nv_bfloat16*, const __nv_bfloat16*, const __nv_bfloat16*, int, int64_t, float*,
                          int64_t, int64_t, int64_t, int, unsigned int*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace cpqr
