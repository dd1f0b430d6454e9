// Split-precision staging for the tensor-core TTM of the full tensor.
//
// X (FP32) is stored once as two bf16 arrays, X = hi + lo + O(2^-16 |X|):
// hi = bf16(X), lo = bf16(X - hi).  Each Q_k (FP64) is staged after its QR as
// bf16 hi/lo of Q_k^T, zero-padded to Rp x Kp (the MMA's N x K operand, K
// contiguous).  The product keeps all four terms hi*hi + hi*lo + lo*hi + lo*lo.
#include <algorithm>

#include "tc_common.cuh"

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

// Rows of ld elements: hi / lo of X's row (last elements), zero in the padding.
__global__ void split_x_padded_kernel(const float* __restrict__ X, __nv_bfloat16* __restrict__ hi,
                                      __nv_bfloat16* __restrict__ lo, int64_t rows, int64_t last, int64_t ld) {
  const int64_t total = rows * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ld, c = e - r * ld;
    const float v = (c < last) ? X[r * last + c] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
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

cudaError_t launch_split_x_padded(const float* X, __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, int64_t rows, int64_t last,
                                  int64_t ld, cudaStream_t st) {
  if (last < 1 || ld < last || (ld % 8) != 0 || rows < 1) return cudaErrorInvalidValue;
  split_x_padded_kernel<<<152 * 8, 256, 0, st>>>(X, Xhi, Xlo, rows, last, ld);
  return cudaGetLastError();
}

TtmView ttm_view(int64_t K, int64_t S, SplitLayout lay) {
  TtmView v{};
  v.ok = true;
  if (lay.ld == 0) {  // dense
    v.Sit = S;
    v.So = S;
    v.rowS = S;
    v.ldK = K;
    return v;
  }
  if (lay.last < 1 || lay.ld < lay.last || (lay.ld % 8) != 0) {
    v.ok = false;
    return v;
  }
  if (S == 1) {  // the contracted mode is the padded last one
    v.ok = (K == lay.last);
    v.Sit = v.So = v.rowS = 1;
    v.ldK = lay.ld;
    return v;
  }
  if (S % lay.last != 0) {
    v.ok = false;
    return v;
  }
  const int64_t q = S / lay.last;
  v.So = S;
  v.ldK = K;
  if (q == 1) {  // S is the padded last dimension itself: its extent with the padded stride
    v.Sit = S;
    v.rowS = lay.ld;
  } else {  // S spans rows of it: iterate over the padded rows, skip the padding in the epilogue
    v.Sit = q * lay.ld;
    v.rowS = v.Sit;
    v.s_last = lay.last;
    v.s_pad = lay.ld;
  }
  return v;
}

cudaError_t launch_split_q(const double* Q, int64_t K, int R, __nv_bfloat16* Qt, int Rp, int64_t Kp,
                           cudaStream_t st) {
  int64_t total = (int64_t)Rp * Kp;
  int grid = (int)std::min<int64_t>((total + 255) / 256, 1024);
  split_q_kernel<<<grid, 256, 0, st>>>(Q, K, R, Qt, Rp, Kp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tensor-core TTM (tcgen05, sm_103a) of the full tensor and of the tree's
// intermediates, from operands split into bf16 hi/lo.
//
// out[p, r, s] = sum_i X[p, i, s] Q[i, r].
//  * S a multiple of 8 (MN-major A): viewed per p, D (S x R) = X_p^T (S x K,
//    s contiguous) * Q (K x R).  A 128-row MMA tile is two 64-row "half tiles"
//    (p, block of 64 s) taken in (p, s-block) order, each loaded by TMA as a
//    64 (s) x 64 (i) bf16 box with 128-byte swizzle.
//  * S == 1 (K-major A, the contracted mode is the contiguous one): D (P x R) =
//    X (P x K, i contiguous) * Q; a tile is 128 rows p, loaded as one 64 (i) x
//    128 (p) box per 64-deep K block.
// Rows beyond S or P are zero-filled by TMA and masked in the epilogue.  Q^T
// (bf16 hi/lo, K-major, zero padded to Rp x Kp) stays resident in shared
// memory.  Per 16-deep K step four MMAs accumulate hi*hi + hi*lo + lo*hi + lo*lo
// into FP32 accumulators in tensor memory (M = 128, N = Rp; hi*hi of even and odd K
// blocks and the corrections apart, see TC_NACC): the products are exact, so the
// error is that of the operands' two-term bf16 representations (~2^-17 each) plus
// the accumulators' truncation; the tensor pipe is far from busy at these ranks.  The epilogue writes
// the FP32 result and, when asked, its own bf16 hi/lo split for the next TTM.
//
// Warp roles (192 threads): warps 0-3 epilogue (tensor-memory lanes 32w..32w+31),
// warp 4 TMA producer + tensor-memory allocation, warp 5 MMA issuer.  Stages of
// A are guarded by full/empty mbarriers, the two accumulators by tfull/tempty.
// Every mbarrier wait gives up after ~2 s, sets CPQR_DEV_TIMEOUT and makes every
// role leave its loop; the kernel then drains in-flight copies and MMAs (again
// bounded) and frees tensor memory before returning.
// ---------------------------------------------------------------------------

namespace {

constexpr int TC_THREADS = 192;
constexpr int TC_NST = 4;                   // A pipeline stages
constexpr int TC_HALF_BYTES = 64 * 64 * 2;  // one 64 x 64 bf16 box
constexpr int TC_STAGE_BYTES = 4 * TC_HALF_BYTES;  // hi h0, hi h1, lo h0, lo h1
constexpr int TC_MAX_KB = 8;                // K <= 512
// Tensor-core FP32 accumulation truncates toward zero: every MMA into an accumulator lowers it by
// ~2^-26 relative on average (measured on GB300: mean relative error -1.3e-6 at K = 400 with one
// accumulator for all four products).  So each tile has three accumulators of 32 columns: hi*hi of
// the even and of the odd 64-deep K blocks, and the three small correction products; the epilogue
// adds them in FP32 with rounding to nearest.  A main accumulator then takes an eighth of the MMAs,
// and the corrections' truncation is relative to their own ~2^-8 smaller size.
constexpr int TC_NACC = 3;
constexpr int TC_ACC_COLS = TC_NACC * 32;   // per tile buffer
constexpr int TC_TMEM_COLS = 256;           // two tile buffers (192 columns), rounded to a power of 2

struct TcParams {
  int64_t P, K, S;  // S: iteration extent of the S dimension (see ttm_view)
  int64_t So, s_last, s_pad;  // dense output extent; remap of padded S rows (s_pad = 0: none)
  int R, Rp, nkb;
  int64_t nsb;  // 64-wide s blocks per p (MN-major)
  int64_t H;    // half tiles = P * nsb (MN-major)
  int64_t T;    // tiles: ceil(H / 2) (MN-major), ceil(P / 128) (K-major)
  float* out;             // FP32 result (may be null when only the split is wanted)
  __nv_bfloat16* out_hi;  // optional split copy of out (hi + lo = out to ~2^-16)
  __nv_bfloat16* out_lo;
  int64_t oh_last, oh_ld;  // the split copy's rows: last dimension padded to oh_ld (0: dense)
  int pair_ok;             // out 8-byte and out_hi / out_lo 4-byte aligned: column pairs stored together
  unsigned int* status;
  unsigned long long wait_ns;  // limit of the pipeline waits (drain waits keep kTimeoutNs)
  int skip_x_loads;            // failure-detection test: issue no tile loads, so the MMA wait runs out
};

struct TcSmemTail {
  unsigned long long full[TC_NST];
  unsigned long long empty[TC_NST];
  unsigned long long tfull[2];
  unsigned long long tempty[2];
  unsigned long long bfull;
  unsigned long long tdown;
  unsigned int tmem_base;
  int abort_flag;
  int issued[TC_NST];
  int consumed[TC_NST];
};

using namespace tc;

// out[idx] and, if asked, the split copy at si (idx, or its place in the padded rows)
__device__ __forceinline__ void store_out(const TcParams& p, int64_t idx, int64_t si, float v) {
  if (p.out) p.out[idx] = v;
  if (p.out_hi) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    p.out_hi[si] = h;
    p.out_lo[si] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// The MN-major epilogue's stores of one row s: out[o + r So] for r < R, FP32 and / or the split
// copy (hi and lo of a pair of columns converted together; each is rounded on its own, so the
// pair conversion equals two single ones).  Base pointers advance by So per column, so a column
// costs its conversion and stores only.
template <int RPT>
__device__ __forceinline__ void store_row_mn(const TcParams& p, int64_t o, const float* v) {
  const int64_t So = p.So;
  const int R = p.R;
  if (p.out_hi) {
    __nv_bfloat16* dh = p.out_hi + o;
    __nv_bfloat16* dl = p.out_lo + o;
#pragma unroll
    for (int r = 0; r < RPT; r += 2) {
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[r], v[r + 1]);
      const float2 hf = __bfloat1622float2(h2);
      const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[r] - hf.x, v[r + 1] - hf.y);
      if (r < R) {
        dh[0] = h2.x;
        dl[0] = l2.x;
      }
      if (r + 1 < R) {
        dh[So] = h2.y;
        dl[So] = l2.y;
      }
      dh += 2 * So;
      dl += 2 * So;
    }
  }
  if (p.out) {
    float* df = p.out + o;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (r < R) *df = v[r];
      df += So;
    }
  }
}

// PO: the split copy of the output goes to padded rows (a dense output compiles without it);
// RPT: accumulator columns read back per part (Rp, 16 or 32)
template <bool KM, bool PO, int RPT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    ttm_tc_kernel(const __grid_constant__ CUtensorMap tmXhi, const __grid_constant__ CUtensorMap tmXlo,
                  const __grid_constant__ CUtensorMap tmQ, TcParams p) {
  extern __shared__ unsigned char tc_smem_raw[];
  // 1024-byte aligned base for the swizzled operand buffers
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
  unsigned char* base = tc_smem_raw + pad;
  const uint32_t sA = smem_u32(base);                            // TC_NST stages
  const uint32_t sB = sA + TC_NST * TC_STAGE_BYTES;              // nkb x {hi, lo} x (Rp x 128 B)
  const uint32_t bsub = (uint32_t)p.Rp * 128u;
  TcSmemTail* tail = reinterpret_cast<TcSmemTail*>(base + TC_NST * TC_STAGE_BYTES + (size_t)p.nkb * 2 * bsub);
  // K-major epilogue: each warp's 32 rows x R results pass through shared memory so that the
  // rows (R contiguous floats each) are written with coalesced stores
  float* epi = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(tail) + ((sizeof(TcSmemTail) + 15) / 16) * 16);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < TC_NST; ++i) {
      mbar_init(smem_u32(&tail->full[i]), 1);
      mbar_init(smem_u32(&tail->empty[i]), 1);
      tail->issued[i] = 0;
      tail->consumed[i] = 0;
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&tail->tfull[i]), 1);
      mbar_init(smem_u32(&tail->tempty[i]), 4);
    }
    mbar_init(smem_u32(&tail->bfull), 1);
    mbar_init(smem_u32(&tail->tdown), 1);
    tail->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tail->tmem_base)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tail->tmem_base;
  // launched as a programmatic dependent: the set-up above overlapped the previous kernel's tail;
  // nothing in global memory is read or written before that kernel has finished
  pdl_wait();

  const int64_t ntile_local = (p.T > (int64_t)blockIdx.x) ? (p.T - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp == 4) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      const uint32_t bbytes = (uint32_t)p.nkb * 2u * bsub;
      mbar_expect_tx(smem_u32(&tail->bfull), bbytes);
      for (int kb = 0; kb < p.nkb; ++kb) {
        tma_load_2d(sB + (2 * kb) * bsub, &tmQ, kb * 64, 0, smem_u32(&tail->bfull));
        tma_load_2d(sB + (2 * kb + 1) * bsub, &tmQ, kb * 64, p.Rp, smem_u32(&tail->bfull));
      }
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t lt = 0; lt < ntile_local && ok; ++lt) {
        const int64_t tile = blockIdx.x + lt * gridDim.x;
        const int64_t h0 = 2 * tile, h1 = 2 * tile + 1;
        int p0 = 0, sb0 = 0, p1 = (int)p.P, sb1 = 0;  // past the last half tile: an all-out-of-bounds box
        if (!KM) {
          p0 = (int)(h0 / p.nsb);
          sb0 = (int)(h0 % p.nsb);
          if (h1 < p.H) {
            p1 = (int)(h1 / p.nsb);
            sb1 = (int)(h1 % p.nsb);
          }
        }
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!mbar_wait(smem_u32(&tail->empty[stage]), phase ^ 1u, &tail->abort_flag, p.status, true, p.wait_ns)) {
            ok = false;
            break;
          }
          if (p.skip_x_loads) {  // nothing arrives on full[stage]: the MMA issuer's wait runs out
            if (++stage == TC_NST) {
              stage = 0;
              phase ^= 1u;
            }
            continue;
          }
          const uint32_t fb = smem_u32(&tail->full[stage]);
          const uint32_t dst = sA + stage * TC_STAGE_BYTES;
          mbar_expect_tx(fb, TC_STAGE_BYTES);
          if (KM) {
            // 128 rows p x 64 i of hi, then of lo
            tma_load_2d(dst, &tmXhi, kb * 64, (int)(tile * 128), fb);
            tma_load_2d(dst + 2 * TC_HALF_BYTES, &tmXlo, kb * 64, (int)(tile * 128), fb);
          } else {
            tma_load_3d(dst, &tmXhi, sb0 * 64, kb * 64, p0, fb);
            tma_load_3d(dst + TC_HALF_BYTES, &tmXhi, sb1 * 64, kb * 64, p1, fb);
            tma_load_3d(dst + 2 * TC_HALF_BYTES, &tmXlo, sb0 * 64, kb * 64, p0, fb);
            tma_load_3d(dst + 3 * TC_HALF_BYTES, &tmXlo, sb1 * 64, kb * 64, p1, fb);
          }
          tail->issued[stage] += 1;
          if (++stage == TC_NST) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      // F32 accumulate, bf16 A and B, B K-major, A MN-major (bit 15) or K-major
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (KM ? 0u : (1u << 15)) |
                             ((uint32_t)(p.Rp >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      bool ok = mbar_wait(smem_u32(&tail->bfull), 0, &tail->abort_flag, p.status, true, p.wait_ns);
      fence_after();
      int stage = 0;
      uint32_t phase = 0;
      for (int64_t lt = 0; lt < ntile_local && ok; ++lt) {
        const int acc = (int)(lt & 1);
        const uint32_t use = (uint32_t)(lt >> 1);
        if (!mbar_wait(smem_u32(&tail->tempty[acc]), (use & 1u) ^ 1u, &tail->abort_flag, p.status, true, p.wait_ns))
          break;
        fence_after();
        const uint32_t d0 = tmem + (uint32_t)(acc * TC_ACC_COLS);
        const uint32_t dc = d0 + 64;  // correction products
        for (int kb = 0; kb < p.nkb; ++kb) {
          const uint32_t dm = d0 + (uint32_t)((kb & 1) * 32);  // hi * hi of even / odd K blocks
          if (!mbar_wait(smem_u32(&tail->full[stage]), phase, &tail->abort_flag, p.status, true, p.wait_ns)) {
            ok = false;
            break;
          }
          tail->consumed[stage] += 1;
          fence_after();
          const uint32_t a_hi = sA + stage * TC_STAGE_BYTES;
          const uint32_t a_lo = a_hi + 2 * TC_HALF_BYTES;
          const uint32_t b_hi = sB + (2 * kb) * bsub, b_lo = b_hi + bsub;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            // MN-major: 16 i-rows of 128 bytes per K step, the two 64-row halves TC_HALF_BYTES apart;
            // K-major: 32 bytes (16 bf16) along each 128-byte row, 8-row groups 1024 bytes apart
            const uint64_t ah = KM ? smem_desc(a_hi + ks * 32, 16, 1024) : smem_desc(a_hi + ks * 2048, TC_HALF_BYTES, 1024);
            const uint64_t al = KM ? smem_desc(a_lo + ks * 32, 16, 1024) : smem_desc(a_lo + ks * 2048, TC_HALF_BYTES, 1024);
            const uint64_t bh = smem_desc(b_hi + ks * 32, 16, 1024);
            const uint64_t bl = smem_desc(b_lo + ks * 32, 16, 1024);
            mma_bf16(dm, ah, bh, idesc, (kb >= 2 || ks != 0) ? 1u : 0u);
            mma_bf16(dc, ah, bl, idesc, (kb | ks) != 0 ? 1u : 0u);
            mma_bf16(dc, al, bh, idesc, 1u);
            mma_bf16(dc, al, bl, idesc, 1u);
          }
          mma_commit(smem_u32(&tail->empty[stage]));
          if (++stage == TC_NST) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(smem_u32(&tail->tfull[acc]));
      }
      // every MMA issued above has completed once tdown flips
      mma_commit(smem_u32(&tail->tdown));
      mbar_wait(smem_u32(&tail->tdown), 0, &tail->abort_flag, p.status, false);
    }
  } else {
    // ---------------- epilogue: warps 0-3, tensor-memory lanes 32w .. 32w+31 ----------------
    const int m = warp * 32 + lane;
    // K-major: element e = lane + 32 j of the warp's rows x R block is (row, r); both advance by
    // 32 / R rows and 32 % R columns per step
    const int km_dq = 32 / p.R, km_dr = 32 - km_dq * p.R;
    for (int64_t lt = 0; lt < ntile_local; ++lt) {
      const int acc = (int)(lt & 1);
      const uint32_t use = (uint32_t)(lt >> 1);
      if (!mbar_wait(smem_u32(&tail->tfull[acc]), use & 1u, &tail->abort_flag, p.status, true, p.wait_ns)) break;
      fence_after();
      // (even + odd) + corrections, each add rounded to nearest; a K of one block has no odd part.
      // The parts are loaded together, with one wait.
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * TC_ACC_COLS);
      float v[RPT];
      uint32_t raw[3 * RPT];
      if (p.nkb > 1) {
        if (RPT == 32) tmem_ld32x3(taddr, taddr + 32, taddr + 64, raw);
        else tmem_ld16x3(taddr, taddr + 32, taddr + 64, raw);
#pragma unroll
        for (int r = 0; r < RPT; ++r)
          v[r] = (__uint_as_float(raw[r]) + __uint_as_float(raw[RPT + r])) + __uint_as_float(raw[2 * RPT + r]);
      } else {
        if (RPT == 32) tmem_ld32x2(taddr, taddr + 64, raw);
        else tmem_ld16x2(taddr, taddr + 64, raw);
#pragma unroll
        for (int r = 0; r < RPT; ++r) v[r] = __uint_as_float(raw[r]) + __uint_as_float(raw[RPT + r]);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tail->tempty[acc]));
      const int64_t tile = blockIdx.x + lt * gridDim.x;
      if (KM) {
        float* stg = epi + warp * (32 * 33);
#pragma unroll
        for (int r = 0; r < RPT; ++r) stg[lane * 33 + r] = v[r];
        __syncwarp();
        const int64_t p0 = tile * 128 + warp * 32;  // this warp's rows, contiguous in out
        const int nrows = (int)std::min<int64_t>(32, p.P - p0);
        if (!(PO && p.oh_ld) && (p.R & 1) == 0 && p.pair_ok) {
          // dense rows of even R: a lane stores a pair of adjacent columns (float2, bf16x2)
          const int half = p.R >> 1;
          const int dq = 32 / half, dc = 32 - dq * half;
          int row = lane / half, c = lane - row * half;
          for (int e = lane; e < nrows * half; e += 32) {
            const float a = stg[row * 33 + 2 * c], b = stg[row * 33 + 2 * c + 1];
            const int64_t idx = p0 * p.R + 2 * e;  // = (p0 + row) R + 2 c
            if (p.out) *reinterpret_cast<float2*>(p.out + idx) = make_float2(a, b);
            if (p.out_hi) {
              const __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
              const float2 hf = __bfloat1622float2(h2);
              *reinterpret_cast<__nv_bfloat162*>(p.out_hi + idx) = h2;
              *reinterpret_cast<__nv_bfloat162*>(p.out_lo + idx) = __floats2bfloat162_rn(a - hf.x, b - hf.y);
            }
            row += dq;
            c += dc;
            if (c >= half) {
              c -= half;
              ++row;
            }
          }
          __syncwarp();
          continue;
        }
        int row = lane / p.R, r = lane - row * p.R;
        for (int e = lane; e < nrows * p.R; e += 32) {
          // K-major output: rows of R (the split copy's rows padded to oh_ld when R is not a multiple of 8)
          const int64_t idx = p0 * p.R + e;
          store_out(p, idx, (PO && p.oh_ld) ? (p0 + row) * p.oh_ld + r : idx, stg[row * 33 + r]);
          row += km_dq;
          r += km_dr;
          if (r >= p.R) {
            r -= p.R;
            ++row;
          }
        }
        __syncwarp();
      } else {
        const int64_t h = 2 * tile + (m >> 6);
        if (h < p.H) {
          int64_t pp, sb;
          if (p.H <= 0x7fffffffLL) {  // the common case: a 32-bit division
            const uint32_t q = (uint32_t)h / (uint32_t)p.nsb;
            pp = q;
            sb = (int64_t)((uint32_t)h - q * (uint32_t)p.nsb);
          } else {
            pp = h / p.nsb;
            sb = h - pp * p.nsb;
          }
          const int64_t sidx = sb * 64 + (m & 63);
          bool live = sidx < p.S;
          int64_t so = sidx;
          if (p.s_pad) {  // a padded source: skip the padding of its last dimension
            const int64_t qd = sidx / p.s_pad, i2 = sidx - qd * p.s_pad;
            live = live && i2 < p.s_last;
            so = qd * p.s_last + i2;
          }
          if (live) {
            const int64_t o = (pp * p.R) * p.So + so;
            if (PO && p.oh_ld) {
              // the split copy in padded rows of the output's last dimension: one division here,
              // element (pp, r, so) then at row (pp R + r) q + so / last, column so % last
              const int64_t q = p.So / p.oh_last;
              const int64_t sq = so / p.oh_last;
              const int64_t srow = pp * p.R * q + sq;
              const int64_t scol = so - sq * p.oh_last;
#pragma unroll
              for (int r = 0; r < RPT; ++r)
                if (r < p.R) {
                  const int64_t idx = o + (int64_t)r * p.So;
                  store_out(p, idx, (srow + (int64_t)r * q) * p.oh_ld + scol, v[r]);
                }
            } else {
              store_row_mn<RPT>(p, o, v);
            }
          }
        }
      }
    }
  }

  // ---------------- teardown ----------------
  __syncthreads();
  if (threadIdx.x == 4 * 32) {
    // copies issued but never consumed (only after an abort): wait for them to land
    for (int st = 0; st < TC_NST; ++st) {
      const int pending = tail->issued[st] - tail->consumed[st];
      if (pending > 0) {
        const uint32_t par = (uint32_t)((tail->issued[st] - 1) & 1);
        mbar_wait(smem_u32(&tail->full[st]), par, &tail->abort_flag, p.status, false);
      }
    }
  }
  __syncthreads();
  if (warp == 4) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

}  // namespace

bool ttm_tc_supported(int64_t P, int64_t K, int64_t S, int R, SplitLayout lay) {
  if (R < 1 || R > 32 || K < 1 || K > 64 * TC_MAX_KB || P < 1 || P > 0x7fffffff || S > 0x7fffffff) return false;
  const TtmView v = ttm_view(K, S, lay);
  if (!v.ok || v.Sit > 0x7fffffff) return false;
  if (S == 1) return (v.ldK % 8) == 0 && (P + 127) / 128 < (int64_t(1) << 31);  // K-major: 16-byte row stride
  if (v.rowS < 8 || (v.rowS % 8) != 0) return false;                          // MN-major: 16-byte row stride
  const int64_t nsb = (v.Sit + 63) / 64;
  if (P * nsb > (int64_t(1) << 40)) return false;
  return true;
}

cudaError_t launch_ttm_tc(const __nv_bfloat16* Xhi, const __nv_bfloat16* Xlo, const __nv_bfloat16* Qt, int Rp,
                          int64_t Kp, float* out, int64_t P, int64_t K, int64_t S, int R, unsigned int* dev_status,
                          cudaStream_t st, int reserve_sms, __nv_bfloat16* out_hi, __nv_bfloat16* out_lo,
                          unsigned long long wait_ns, int skip_x_loads, SplitLayout lay, SplitLayout out_lay) {
  if (!ttm_tc_supported(P, K, S, R, lay) || (Rp != 16 && Rp != 32) || Rp < R || Kp < K || (Kp % 64) != 0)
    return cudaErrorNotSupported;
  const TtmView view = ttm_view(K, S, lay);
  if (((uintptr_t)Xhi & 15) || ((uintptr_t)Xlo & 15) || ((uintptr_t)Qt & 15)) return cudaErrorMisalignedAddress;
  if ((out_hi == nullptr) != (out_lo == nullptr)) return cudaErrorInvalidValue;
  const bool km = (S == 1);
  tc::EncodeTiledFn enc = tc::encode_tiled_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tmh, tml, tmq;
  if (km) {
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)P};
    cuuint64_t strides[1] = {(cuuint64_t)view.ldK * 2};
    cuuint32_t box[2] = {64, 128};
    cuuint32_t es[2] = {1, 1};
    if (enc(&tmh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)Xhi, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
    if (enc(&tml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)Xlo, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  } else {
    cuuint64_t dims[3] = {(cuuint64_t)view.Sit, (cuuint64_t)K, (cuuint64_t)P};
    cuuint64_t strides[2] = {(cuuint64_t)view.rowS * 2, (cuuint64_t)view.rowS * K * 2};
    cuuint32_t box[3] = {64, 64, 1};
    cuuint32_t es[3] = {1, 1, 1};
    if (enc(&tmh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)Xhi, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
    if (enc(&tml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)Xlo, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)(2 * Rp)};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)Rp};
    cuuint32_t es[2] = {1, 1};
    if (enc(&tmq, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)Qt, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  TcParams prm;
  prm.P = P;
  prm.K = K;
  prm.R = R;
  prm.Rp = Rp;
  prm.nkb = (int)((K + 63) / 64);
  prm.S = view.Sit;
  prm.So = view.So;
  prm.s_last = view.s_last;
  prm.s_pad = view.s_pad;
  prm.nsb = km ? 1 : (view.Sit + 63) / 64;
  prm.H = P * prm.nsb;
  prm.T = km ? (P + 127) / 128 : (prm.H + 1) / 2;
  prm.out = out;
  prm.out_hi = out_hi;
  prm.out_lo = out_lo;
  prm.oh_last = out_lay.ld ? out_lay.last : 0;
  prm.oh_ld = out_lay.ld;
  prm.pair_ok = ((uintptr_t)out & 7) == 0 && ((uintptr_t)out_hi & 3) == 0 && ((uintptr_t)out_lo & 3) == 0;
  prm.status = dev_status;
  prm.wait_ns = wait_ns ? wait_ns : tc::kTimeoutNs;
  prm.skip_x_loads = skip_x_loads;
  if (prm.nkb * 64 > Kp) return cudaErrorInvalidValue;
  const size_t smem = 1024 + (size_t)TC_NST * TC_STAGE_BYTES + (size_t)prm.nkb * 2 * Rp * 128 +
                      ((sizeof(TcSmemTail) + 15) / 16) * 16 + (km ? 4 * 32 * 33 * sizeof(float) : 0);
  const bool po = out_hi && out_lay.ld;
  auto kern = (Rp == 16)
                  ? (km ? (po ? ttm_tc_kernel<true, true, 16> : ttm_tc_kernel<true, false, 16>)
                        : (po ? ttm_tc_kernel<false, true, 16> : ttm_tc_kernel<false, false, 16>))
                  : (km ? (po ? ttm_tc_kernel<true, true, 32> : ttm_tc_kernel<true, false, 32>)
                        : (po ? ttm_tc_kernel<false, true, 32> : ttm_tc_kernel<false, false, 32>));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (reserve_sms > 0) {
    // A cluster QR (reserve_sms CTAs in one cluster, hence in one GPC) runs beside this grid.
    // Spare SMs scattered over the GPCs would not let it start, so the persistent grid is
    // launched as clusters of the same size, one fewer than fit on the device: each of them
    // takes a GPC of its own and one GPC's worth stays free whatever is placed first.  The
    // CTAs never synchronise as a cluster; the clustering only steers placement.
    const int cl = reserve_sms;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
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
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 2) {
      const int64_t want = (prm.T + cl - 1) / cl;  // clusters with at least one tile each
      const int64_t ncl = std::min<int64_t>(want, nclusters - 1);
      cfg.gridDim = dim3((unsigned)(ncl * cl), 1, 1);
      e = cudaLaunchKernelEx(&cfg, kern, tmh, tml, tmq, prm);
      if (e == cudaSuccess) return cudaSuccess;
    }
    cudaGetLastError();  // fall back to a plain grid that leaves reserve_sms SMs idle
  }
  const int64_t grid = std::min<int64_t>(prm.T, std::max(1, tc::num_sms() - std::max(0, reserve_sms)));
  return launch_pdl(kern, dim3((unsigned)grid), dim3(TC_THREADS), smem, st, tmh, tml, tmq, prm);
}

namespace tc {

EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

}  // namespace tc

}  // namespace cpqr
