// Explicit residual ||X - [[lambda; A]]||^2 (Section 4.1's fit without the cancellation of the
// reduced form) on the tensor cores.
//
// X (FP32, C order) is viewed as rows x columns: the columns run over the trailing nt modes, the
// rows over the others (nt = 1 unless the last side is below 128: then trailing modes are folded
// into the columns until they reach 128, so that the weights of a tile serve enough columns).  The
// model block of a tile of 128 rows is K = W B^T with the Khatri-Rao weights W[row, r] =
// prod_{row modes n} A_n[i_n, r] (lambda folded into A_0) and B[c, r] = prod_{column modes n}
// A_n[i_n, r], a 128 x R by R x columns product.  It runs
// as tcgen05 kind::tf32 MMAs with FP32 accumulation in tensor memory, each operand split into a
// TF32 high part and a TF32 remainder, both rounded to nearest: W A^T ~ Wh Ah^T + Wh Al^T +
// Wl Ah^T, relative error ~2^-21 per product, of either sign, against ~1e-3 residuals.  The residual (x - k)^2 is summed in FP32 per 32 columns
// and in FP64 across them.
//
// CTA roles (320 threads, one CTA per SM): warp 0 streams X tiles (128 rows x 32 columns,
// 128-byte swizzle) through a 6-stage TMA ring; warp 1 owns tensor memory and issues the MMAs;
// warps 6-9 build W one tile ahead (one row per thread; their factor loads never stall the
// stream); warps 2-5 read the accumulator (tensor-memory lane = row) and the X ring.  Two W
// buffers and two accumulators of 256 columns let the MMAs of tile t+1 overlap the epilogue of
// tile t.
// Every CTA owns one group of at most 256 columns (A_last^T of the group split into hi / lo
// once, in shared memory) and a contiguous range of row tiles.  All mbarrier waits are bounded
// (CPQR_DEV_TIMEOUT, then every role leaves; in-flight copies are drained and tensor memory is
// freed before the kernel returns).
#include <algorithm>

#include "tc_common.cuh"

namespace cpqr {

namespace {

using namespace tc;

constexpr int RT_THREADS = 320;
constexpr int RT_M = 128;                // rows per tile: MMA M, tensor-memory lanes
constexpr int RT_NXS = 6;                // X ring stages
constexpr int RT_XBOX = RT_M * 128;      // 128 rows x 32 FP32 columns
constexpr int RT_WBYTES = RT_M * 128;    // 128 rows x 32 FP32 weights, one of hi / lo
constexpr int RT_MAXW = 256;             // columns per CTA: one accumulator
constexpr int RT_TMEM_COLS = 2 * RT_MAXW;
constexpr int RT_FOLD = 128;             // a last side below this takes the modes before it into the columns

struct RtParams {
  int N, R;
  int d[CPQR_MAXN];
  const float* A[CPQR_MAXN];  // FP32 factors, lambda folded into A[0]; A[N-1] stored transposed (R x I_last)
  int nt;                     // trailing modes folded into the columns (1 .. N - 1)
  int Ic;                     // columns: prod_{n >= N - nt} d[n]
  int rows;                   // prod_{n < N - nt} d[n] (< 2^31)
  int rtiles;                 // ceil(rows / 128)
  int cpg;                    // CTAs per column group
  int gw;                     // columns per group (multiple of 4); the last group may be narrower
  int ncp;                    // MMA N = gw rounded up to 32
  double* part;  // one partial sum per CTA, added in a fixed order afterwards
  unsigned int* status;
};

struct RtTail {
  unsigned long long xfull[RT_NXS], xempty[RT_NXS];
  unsigned long long wfull[2], mdone[2], tempty[2];
  unsigned long long tdown;
  unsigned int tmem_base;
  int abort_flag;
  int issued[RT_NXS];
  int consumed[RT_NXS];
  double red[4];
};

// Byte offset of 16-byte chunk q of row `row` in a tile of 128-byte rows with the 128-byte
// swizzle (8-row atoms of 1024 bytes): the layout TMA writes and the MMA descriptors read.
__device__ __forceinline__ uint32_t sw128(int row, int q) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((q ^ (row & 7)) << 4));
}

__device__ __forceinline__ float tf32_rna(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// Both parts rounded to the nearest TF32 value: the remainder v - hi - lo and the dropped lo * lo
// term then take either sign.  Clearing the low bits instead (and letting the MMA truncate the
// remainder) makes every split product low by a few 2^-22, which a fit taken away from a
// least-squares optimum (eq. 19's scaled fixed point) sees to first order.
__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
  hi = tf32_rna(v);
  lo = tf32_rna(v - hi);  // v - hi is exact
}

// Lane 0 waits, the warp learns the outcome (keeps .sync.aligned instructions convergent).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, int* abort_flag, unsigned int* status) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag, status) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__global__ void __launch_bounds__(RT_THREADS, 1)
    residual_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ RtParams p) {
  extern __shared__ unsigned char rt_smem_raw[];
  const uint32_t raw = smem_u32(rt_smem_raw);
  unsigned char* base = rt_smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t bbytes = (uint32_t)p.ncp * 128u;  // A_last^T group, one of hi / lo
  unsigned char* gB = base;                         // [hi | lo]
  unsigned char* gW = gB + 2 * bbytes;              // [buf][hi | lo]
  unsigned char* gX = gW + 4 * RT_WBYTES;           // ring
  RtTail* tail = reinterpret_cast<RtTail*>(gX + RT_NXS * RT_XBOX);
  const uint32_t sB = smem_u32(gB), sW = smem_u32(gW), sX = smem_u32(gX);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Il = p.Ic;
  const int cg = blockIdx.x / p.cpg, kq = blockIdx.x % p.cpg;
  const int c0 = cg * p.gw;
  if (c0 >= Il) {  // padding CTA of a clustered launch: no column group, a zero partial
    if (threadIdx.x == 0) p.part[blockIdx.x] = 0.0;
    return;
  }
  const int width = min(p.gw, Il - c0);
  const int t0 = (int)((int64_t)p.rtiles * kq / p.cpg), t1 = (int)((int64_t)p.rtiles * (kq + 1) / p.cpg);
  const int ntl = t1 - t0;
  const int nch = p.ncp / 32;
  int* abort_flag = &tail->abort_flag;

  if (threadIdx.x == 0) {
    for (int i = 0; i < RT_NXS; ++i) {
      mbar_init(smem_u32(&tail->xfull[i]), 1);
      mbar_init(smem_u32(&tail->xempty[i]), 4);
      tail->issued[i] = 0;
      tail->consumed[i] = 0;
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&tail->wfull[i]), 4);
      mbar_init(smem_u32(&tail->mdone[i]), 1);
      mbar_init(smem_u32(&tail->tempty[i]), 4);
    }
    mbar_init(smem_u32(&tail->tdown), 1);
    tail->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&tail->tmem_base), RT_TMEM_COLS);

  // B operand: row c of the group = prod over the column modes of A_n[i_n, 0..31] for column
  // c0 + c (zero past the group or past R; A_last is stored transposed)
  {
    const int Ilast = p.d[p.N - 1];
    const float* AlT = p.A[p.N - 1];
    for (int e = threadIdx.x; e < p.ncp * 8; e += RT_THREADS) {
      const int c = e >> 3, q = e & 7;
      float v4[4] = {0.f, 0.f, 0.f, 0.f};
      if (c < width) {
        const int col = c0 + c;
        int x = col / Ilast;
        const int il = col - x * Ilast;
#pragma unroll
        for (int j = 0; j < 4; ++j) v4[j] = (4 * q + j < p.R) ? AlT[(int64_t)(4 * q + j) * Ilast + il] : 0.f;
        for (int n = p.N - 2; n >= p.N - p.nt; --n) {
          const int qd = x / p.d[n];
          const float* an = p.A[n] + (int64_t)(x - qd * p.d[n]) * p.R;
          x = qd;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (4 * q + j < p.R) v4[j] *= an[4 * q + j];
        }
      }
      float h[4], l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) split_tf32(v4[j], h[j], l[j]);
      *reinterpret_cast<float4*>(gB + sw128(c, q)) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(gB + bbytes + sw128(c, q)) = make_float4(l[0], l[1], l[2], l[3]);
    }
  }
  fence_proxy_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tail->tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- X producer ----------------
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int lt = 0; lt < ntl && ok; ++lt) {
        const int r0 = (t0 + lt) * RT_M;
        for (int j = 0; j < nch; ++j) {
          if (!mbar_wait(smem_u32(&tail->xempty[stage]), phase ^ 1u, abort_flag, p.status)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&tail->xfull[stage]);
          mbar_expect_tx(fb, RT_XBOX);
          tma_load_2d(sX + stage * RT_XBOX, &tmX, c0 + 32 * j, r0, fb);
          tail->issued[stage] += 1;
          if (++stage == RT_NXS) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      // F32 accumulate, TF32 A and B, both K-major, N = ncp, M = 128
      const uint32_t idesc =
          (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(p.ncp >> 3) << 17) | ((uint32_t)(RT_M >> 4) << 24);
      for (int lt = 0; lt < ntl; ++lt) {
        const int b = lt & 1;
        const uint32_t use = (uint32_t)(lt >> 1);
        if (!mbar_wait(smem_u32(&tail->wfull[b]), use & 1u, abort_flag, p.status)) break;
        if (!mbar_wait(smem_u32(&tail->tempty[b]), (use & 1u) ^ 1u, abort_flag, p.status)) break;
        fence_after();
        const uint32_t d = tmem + (uint32_t)(b * RT_MAXW);
        const uint32_t wh = sW + (uint32_t)(2 * b) * RT_WBYTES, wl = wh + RT_WBYTES;
        // K = 32 as four steps of 8 TF32 (32 bytes).  The small correction products go first: the
        // accumulator truncates each sum toward zero relative to its current size, so only the four
        // hi * hi steps at the end truncate at the full size of the model entry
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t ah = smem_desc(wh + ks * 32, 16, 1024), al = smem_desc(wl + ks * 32, 16, 1024);
          const uint64_t bh = smem_desc(sB + ks * 32, 16, 1024), bl = smem_desc(sB + bbytes + ks * 32, 16, 1024);
          mma_tf32(d, ah, bl, idesc, ks > 0 ? 1u : 0u);
          mma_tf32(d, al, bh, idesc, 1u);
        }
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t ah = smem_desc(wh + ks * 32, 16, 1024), bh = smem_desc(sB + ks * 32, 16, 1024);
          mma_tf32(d, ah, bh, idesc, 1u);
        }
        mma_commit(smem_u32(&tail->mdone[b]));
      }
      // every MMA issued above has completed once tdown flips
      mma_commit(smem_u32(&tail->tdown));
      mbar_wait(smem_u32(&tail->tdown), 0, abort_flag, p.status, false);
    }
  } else if (warp >= 6) {
    // ---------------- Khatri-Rao weights: warps 6-9, row m of the tile ----------------
    const int m = (warp - 6) * 32 + lane;
    const bool avec = (p.R & 3) == 0;
    for (int lt = 0; lt < ntl; ++lt) {
      const int b = lt & 1;
      if (lt >= 2) {
        // buffer b was last read by the MMAs of tile lt - 2
        const uint32_t use = (uint32_t)((lt - 2) >> 1);
        if (!warp_wait(smem_u32(&tail->mdone[b]), use & 1u, abort_flag, p.status)) break;
      }
      const int row = (t0 + lt) * RT_M + m;
      float w[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) w[r] = (row < p.rows && r < p.R) ? 1.f : 0.f;
      if (row < p.rows) {
        int x = row;
        for (int n = p.N - 1 - p.nt; n >= 0; --n) {
          int in = x;
          if (n > 0) {
            const int qd = x / p.d[n];
            in = x - qd * p.d[n];
            x = qd;
          }
          const float* an = p.A[n] + (int64_t)in * p.R;
          if (avec) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              if (4 * q < p.R) {
                const float4 u = *reinterpret_cast<const float4*>(an + 4 * q);
                w[4 * q] *= u.x;
                w[4 * q + 1] *= u.y;
                w[4 * q + 2] *= u.z;
                w[4 * q + 3] *= u.w;
              }
            }
          } else {
#pragma unroll
            for (int r = 0; r < 32; ++r)
              if (r < p.R) w[r] *= an[r];
          }
        }
      }
      unsigned char* wh = gW + (2 * b) * RT_WBYTES;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) split_tf32(w[4 * q + j], h[j], l[j]);
        *reinterpret_cast<float4*>(wh + sw128(m, q)) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(wh + RT_WBYTES + sw128(m, q)) = make_float4(l[0], l[1], l[2], l[3]);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tail->wfull[b]));
    }
  } else {
    // ---------------- epilogue: warps 2-5, row m = tensor-memory lane ----------------
    const int m = (warp & 3) * 32 + lane;
    double acc = 0.0;
    int stage = 0;
    uint32_t phase = 0;
    for (int lt = 0; lt < ntl; ++lt) {
      const int b = lt & 1;
      const uint32_t use = (uint32_t)(lt >> 1);
      if (!warp_wait(smem_u32(&tail->mdone[b]), use & 1u, abort_flag, p.status)) break;
      fence_after();
      const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(b * RT_MAXW);
      bool ok = true;
      for (int j = 0; j < nch; ++j) {
        if (!warp_wait(smem_u32(&tail->xfull[stage]), phase, abort_flag, p.status)) {
          ok = false;
          break;
        }
        if (threadIdx.x == 64) tail->consumed[stage] += 1;
        float kv[32];
        tmem_ld32(taddr + 32 * j, kv);
        const unsigned char* xs = gX + stage * RT_XBOX;
        const int nv = min(32, width - 32 * j);  // columns of this chunk inside the group
        float racc = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 x4 = *reinterpret_cast<const float4*>(xs + sw128(m, q));
          const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float dd = (4 * q + e < nv) ? xv[e] - kv[4 * q + e] : 0.f;
            racc = fmaf(dd, dd, racc);
          }
        }
        acc += (double)racc;
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tail->xempty[stage]));
        if (++stage == RT_NXS) {
          stage = 0;
          phase ^= 1u;
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tail->tempty[b]));
      if (!ok) break;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) tail->red[warp - 2] = acc;
  }

  // ---------------- teardown ----------------
  __syncthreads();
  if (threadIdx.x == 64) {
    // copies issued but never consumed (only after an abort): wait for them to land
    for (int st = 0; st < RT_NXS; ++st) {
      if (tail->issued[st] > tail->consumed[st]) {
        const uint32_t par = (uint32_t)((tail->issued[st] - 1) & 1);
        mbar_wait(smem_u32(&tail->xfull[st]), par, abort_flag, p.status, false);
      }
    }
  }
  if (threadIdx.x == 0) p.part[blockIdx.x] = (ntl > 0) ? tail->red[0] + tail->red[1] + tail->red[2] + tail->red[3] : 0.0;
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, RT_TMEM_COLS);
  }
}

}  // namespace

bool residual_tc_supported(int N, const int64_t* d, int R, const void* X) {
  if (N < 2 || N > CPQR_MAXN || R < 1 || R > 32) return false;
  if (reinterpret_cast<uintptr_t>(X) & 15) return false;
  const int64_t Il = d[N - 1];
  if (Il < 4 || (Il % 4) != 0 || Il > (int64_t(1) << 30)) return false;  // TMA row stride: 16-byte multiple
  int64_t rows = 1;
  for (int n = 0; n < N - 1; ++n) {
    if (d[n] < 1) return false;
    rows *= d[n];
    if (rows > 0x7fff0000) return false;
  }
  return true;
}

size_t residual_tc_smem_bytes(int ncp) {
  return 1024 + (size_t)2 * ncp * 128 + (size_t)4 * RT_WBYTES + (size_t)RT_NXS * RT_XBOX + sizeof(RtTail);
}

cudaError_t launch_residual_tc(const float* X, int N, const int64_t* d, const float* const* Af, int R, double* part,
                               int max_parts, int* nparts, unsigned int* dev_status, cudaStream_t st,
                               int reserve_sms) {
  if (!residual_tc_supported(N, d, R, X)) return cudaErrorNotSupported;
  tc::EncodeTiledFn enc = tc::encode_tiled_fn();
  if (!enc) return cudaErrorNotSupported;
  RtParams p{};
  p.N = N;
  p.R = R;
  for (int n = 0; n < N; ++n) {
    p.d[n] = (int)d[n];
    p.A[n] = Af[n];
  }
  // columns: the last mode, with the modes before it folded in while the columns are fewer than
  // RT_FOLD (a short last side leaves the weights and the hand-offs of a tile serving few bytes of
  // X; 128 columns, 64 KB a tile, already keep a CTA's share of the bandwidth busy, and folding
  // them would leave fewer row tiles than CTAs per column group)
  int nt = 1;
  int64_t Ic = d[N - 1];
  while (Ic < RT_FOLD && nt < N - 1 && Ic * d[N - 1 - nt] <= (int64_t(1) << 30)) Ic *= d[N - 1 - nt++];
  int64_t rows = 1;
  for (int n = 0; n < N - nt; ++n) rows *= d[n];
  const int Il = (int)Ic;
  p.nt = nt;
  p.Ic = Il;
  p.rows = (int)rows;
  p.rtiles = (int)((rows + RT_M - 1) / RT_M);
  const int ncg = (Il + RT_MAXW - 1) / RT_MAXW;
  p.gw = (((Il + ncg - 1) / ncg) + 3) & ~3;
  p.ncp = (p.gw + 31) & ~31;
  if (p.ncp > RT_MAXW) return cudaErrorNotSupported;
  p.cpg = std::max(1, std::min(p.rtiles, tc::num_sms() / ncg));
  p.part = part;
  p.status = dev_status;
  CUtensorMap tm;
  {
    cuuint64_t dims[2] = {(cuuint64_t)Il, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Il * 4};
    cuuint32_t box[2] = {32, (cuuint32_t)RT_M};
    cuuint32_t es[2] = {1, 1};
    if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)X, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  const size_t smem = residual_tc_smem_bytes(p.ncp);
  static size_t smem_set = 0;  // the attribute is raised once to the largest size used
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(residual_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)residual_tc_smem_bytes(RT_MAXW));
    if (e != cudaSuccess) return e;
    smem_set = residual_tc_smem_bytes(RT_MAXW);
  }
  if (reserve_sms > 0) {
    // Beside a cluster QR (reserve_sms CTAs in one GPC): clusters of the same size, one fewer than
    // fit, leave a GPC free for it (the CTAs never synchronise as a cluster).  CTAs past
    // ncg * cpg have no work and return at once.
    const int cl = reserve_sms;
    cudaError_t e = cudaFuncSetAttribute(residual_tc_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(RT_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)cl, 1, 1);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, residual_tc_kernel, &cfg) == cudaSuccess && nclusters >= 2) {
      const int ctas = (nclusters - 1) * cl;
      p.cpg = std::max(1, std::min(p.rtiles, ctas / ncg));
      cfg.gridDim = dim3((unsigned)ctas, 1, 1);
      if (ctas > max_parts) return cudaErrorInvalidValue;
      *nparts = ncg * p.cpg;  // the CTAs with work; the padding CTAs after them only write zeros
      e = cudaLaunchKernelEx(&cfg, residual_tc_kernel, tm, p);
      if (e == cudaSuccess) return cudaSuccess;
    }
    cudaGetLastError();
    p.cpg = std::max(1, std::min(p.rtiles, (tc::num_sms() - reserve_sms) / ncg));
  }
  if (ncg * p.cpg > max_parts) return cudaErrorInvalidValue;
  *nparts = ncg * p.cpg;
  residual_tc_kernel<<<(unsigned)(ncg * p.cpg), RT_THREADS, smem, st>>>(tm, p);
  return cudaGetLastError();
}

}  // namespace cpqr
