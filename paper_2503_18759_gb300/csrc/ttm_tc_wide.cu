// Tensor-core TTM for ranks 33..192 (the wide-rank path; the high-rank regime of Section 4.2).
//
// out[p, r, s] = sum_i X[p, i, s] Q[i, r] from bf16 hi/lo operands, like ttm_tc.cu, with the MMA's
// N = Rp (R rounded up to 16) up to 192 columns.  Differences from the narrow kernel:
//  * Q^T no longer fits in shared memory for the whole K: every pipeline stage carries the 64-deep
//    K block of Q^T (hi and lo, Rp rows of 128 bytes each) beside the X tile, loaded by the same
//    TMA transaction (Q^T is small and stays in L2);
//  * two accumulators per tile, hi*hi and the three correction products (hi*lo, lo*hi, lo*lo),
//    each Rp rounded up to 32 tensor-memory columns; double-buffered while that fits 512 columns
//    (Rp <= 128), else one buffer;
//  * the epilogue reads the accumulators in 32-column chunks.
// At these ranks the contraction reaches the tensor cores' ridge: per element of X (4 bytes of
// bf16 hi + lo) the four products issue 8 Rp flops.
#include <algorithm>

#include "tc_common.cuh"

namespace cpqr {

namespace {

using namespace tc;

constexpr int TW_THREADS = 192;
constexpr int TW_A_BYTES = 4 * 64 * 64 * 2;  // X tile: hi h0, hi h1, lo h0, lo h1 (or 128-row hi, lo)
constexpr int TW_HALF = 64 * 64 * 2;
constexpr int TW_MAXST = 3;
constexpr int TW_SMEM_LIMIT = 227 * 1024;

struct TwParams {
  int64_t P, K, S;  // S: iteration extent of the S dimension (see ttm_view)
  int64_t So, s_last, s_pad;  // dense output extent; remap of padded S rows (s_pad = 0: none)
  int R, Rp, nkb, nst, nbuf;
  uint32_t stage_bytes, tmem_cols;
  int64_t nsb, H, T;
  float* out;
  __nv_bfloat16* out_hi;
  __nv_bfloat16* out_lo;
  int64_t oh_last, oh_ld;  // the split copy's rows: last dimension padded to oh_ld (0: dense)
  unsigned int* status;
};

struct TwTail {
  unsigned long long full[TW_MAXST];
  unsigned long long empty[TW_MAXST];
  unsigned long long tfull[2];
  unsigned long long tempty[2];
  unsigned long long tdown;
  unsigned int tmem_base;
  int abort_flag;
  int issued[TW_MAXST];
  int consumed[TW_MAXST];
};

// out[idx] and, if asked, the split copy at si (idx, or its place in the padded rows)
__device__ __forceinline__ void store_w(const TwParams& p, int64_t idx, int64_t si, float v) {
  if (p.out) p.out[idx] = v;
  if (p.out_hi) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    p.out_hi[si] = h;
    p.out_lo[si] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// The MN-major stores of one row s for the nc columns of a chunk: out[o + r So], r < nc (o at
// the chunk's first column), FP32 and / or the split copy (pair conversion as in ttm_tc.cu);
// base pointers advance by So per column.
__device__ __forceinline__ void store_chunk_mn(const TwParams& p, int64_t o, const float* v, int nc) {
  const int64_t So = p.So;
  if (p.out_hi) {
    __nv_bfloat16* dh = p.out_hi + o;
    __nv_bfloat16* dl = p.out_lo + o;
#pragma unroll
    for (int r = 0; r < 32; r += 2) {
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[r], v[r + 1]);
      const float2 hf = __bfloat1622float2(h2);
      const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[r] - hf.x, v[r + 1] - hf.y);
      if (r < nc) {
        dh[0] = h2.x;
        dl[0] = l2.x;
      }
      if (r + 1 < nc) {
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
    for (int r = 0; r < 32; ++r) {
      if (r < nc) *df = v[r];
      df += So;
    }
  }
}

// PO: the split copy of the output goes to padded rows (a dense output compiles without it)
template <bool KM, bool PO>
__global__ void __launch_bounds__(TW_THREADS, 1)
    ttm_tc_wide_kernel(const __grid_constant__ CUtensorMap tmXhi, const __grid_constant__ CUtensorMap tmXlo,
                       const __grid_constant__ CUtensorMap tmQ, TwParams p) {
  extern __shared__ unsigned char tw_smem_raw[];
  const uint32_t raw = smem_u32(tw_smem_raw);
  const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
  unsigned char* base = tw_smem_raw + pad;
  const uint32_t sS = smem_u32(base);  // stages: [A tile | Q^T hi (Rp x 128 B) | Q^T lo]
  const uint32_t bsub = (uint32_t)p.Rp * 128u;
  TwTail* tail = reinterpret_cast<TwTail*>(base + (size_t)p.nst * p.stage_bytes);
  float* epi = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(tail) + ((sizeof(TwTail) + 15) / 16) * 16);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < p.nst; ++i) {
      mbar_init(smem_u32(&tail->full[i]), 1);
      mbar_init(smem_u32(&tail->empty[i]), 1);
      tail->issued[i] = 0;
      tail->consumed[i] = 0;
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&tail->tfull[i]), 1);
      mbar_init(smem_u32(&tail->tempty[i]), 4);
    }
    mbar_init(smem_u32(&tail->tdown), 1);
    tail->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 4) tmem_alloc(smem_u32(&tail->tmem_base), p.tmem_cols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tail->tmem_base;
  const int64_t ntile_local = (p.T > (int64_t)blockIdx.x) ? (p.T - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  // [hi*hi | corrections] of one tile, each starting on a 32-column boundary
  const uint32_t rpa = ((uint32_t)p.Rp + 31u) & ~31u;
  const uint32_t acc_cols = 2u * rpa;

  if (warp == 4) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
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
          if (!mbar_wait(smem_u32(&tail->empty[stage]), phase ^ 1u, &tail->abort_flag, p.status)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&tail->full[stage]);
          const uint32_t dst = sS + (uint32_t)stage * p.stage_bytes;
          mbar_expect_tx(fb, p.stage_bytes);
          if (KM) {
            tma_load_2d(dst, &tmXhi, kb * 64, (int)(tile * 128), fb);
            tma_load_2d(dst + 2 * TW_HALF, &tmXlo, kb * 64, (int)(tile * 128), fb);
          } else {
            tma_load_3d(dst, &tmXhi, sb0 * 64, kb * 64, p0, fb);
            tma_load_3d(dst + TW_HALF, &tmXhi, sb1 * 64, kb * 64, p1, fb);
            tma_load_3d(dst + 2 * TW_HALF, &tmXlo, sb0 * 64, kb * 64, p0, fb);
            tma_load_3d(dst + 3 * TW_HALF, &tmXlo, sb1 * 64, kb * 64, p1, fb);
          }
          tma_load_2d(dst + TW_A_BYTES, &tmQ, kb * 64, 0, fb);             // Q^T hi, Rp rows
          tma_load_2d(dst + TW_A_BYTES + bsub, &tmQ, kb * 64, p.Rp, fb);   // Q^T lo
          tail->issued[stage] += 1;
          if (++stage == p.nst) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (KM ? 0u : (1u << 15)) |
                             ((uint32_t)(p.Rp >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t lt = 0; lt < ntile_local && ok; ++lt) {
        const int acc = (p.nbuf == 2) ? (int)(lt & 1) : 0;
        const uint32_t use = (p.nbuf == 2) ? (uint32_t)(lt >> 1) : (uint32_t)lt;
        if (!mbar_wait(smem_u32(&tail->tempty[acc]), (use & 1u) ^ 1u, &tail->abort_flag, p.status)) break;
        fence_after();
        const uint32_t dm = tmem + (uint32_t)acc * acc_cols, dc = dm + rpa;
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!mbar_wait(smem_u32(&tail->full[stage]), phase, &tail->abort_flag, p.status)) {
            ok = false;
            break;
          }
          tail->consumed[stage] += 1;
          fence_after();
          const uint32_t a_hi = sS + (uint32_t)stage * p.stage_bytes;
          const uint32_t a_lo = a_hi + 2 * TW_HALF;
          const uint32_t b_hi = a_hi + TW_A_BYTES, b_lo = b_hi + bsub;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t ah = KM ? smem_desc(a_hi + ks * 32, 16, 1024) : smem_desc(a_hi + ks * 2048, TW_HALF, 1024);
            const uint64_t al = KM ? smem_desc(a_lo + ks * 32, 16, 1024) : smem_desc(a_lo + ks * 2048, TW_HALF, 1024);
            const uint64_t bh = smem_desc(b_hi + ks * 32, 16, 1024);
            const uint64_t bl = smem_desc(b_lo + ks * 32, 16, 1024);
            const uint32_t first = (kb | ks) != 0 ? 1u : 0u;
            mma_bf16(dm, ah, bh, idesc, first);
            mma_bf16(dc, ah, bl, idesc, first);
            mma_bf16(dc, al, bh, idesc, 1u);
            mma_bf16(dc, al, bl, idesc, 1u);
          }
          mma_commit(smem_u32(&tail->empty[stage]));
          if (++stage == p.nst) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(smem_u32(&tail->tfull[acc]));
      }
      mma_commit(smem_u32(&tail->tdown));
      mbar_wait(smem_u32(&tail->tdown), 0, &tail->abort_flag, p.status, false);
    }
  } else {
    // ---------------- epilogue: warps 0-3, tensor-memory lanes 32w .. 32w+31 ----------------
    const int m = warp * 32 + lane;
    for (int64_t lt = 0; lt < ntile_local; ++lt) {
      const int acc = (p.nbuf == 2) ? (int)(lt & 1) : 0;
      const uint32_t use = (p.nbuf == 2) ? (uint32_t)(lt >> 1) : (uint32_t)lt;
      if (!mbar_wait(smem_u32(&tail->tfull[acc]), use & 1u, &tail->abort_flag, p.status)) break;
      fence_after();
      const int64_t tile = blockIdx.x + lt * gridDim.x;
      const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)acc * acc_cols;
      // MN-major: this thread's row s of the tile (a 32-bit division in the common case)
      int64_t o_row = -1, po_q = 0, po_srow = 0, po_scol = 0;
      if (!KM) {
        const int64_t h = 2 * tile + (m >> 6);
        if (h < p.H) {
          int64_t pp, sb;
          if (p.H <= 0x7fffffffLL) {
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
            o_row = (pp * p.R) * p.So + so;
            if (PO && p.oh_ld) {
              // the split copy in padded rows of the output's last dimension (see ttm_tc.cu)
              po_q = p.So / p.oh_last;
              const int64_t sq = so / p.oh_last;
              po_srow = pp * p.R * po_q + sq;
              po_scol = so - sq * p.oh_last;
            }
          }
        }
      }
      for (int c0 = 0; c0 < p.Rp; c0 += 32) {
        const int w = (p.Rp - c0 >= 32) ? 32 : 16;
        // hi*hi and the corrections of the chunk, loaded with one wait
        float v[32];
        uint32_t raw[64];
        if (w == 32) {
          tmem_ld32x2(tbase + (uint32_t)c0, tbase + rpa + (uint32_t)c0, raw);
#pragma unroll
          for (int r = 0; r < 32; ++r) v[r] = __uint_as_float(raw[r]) + __uint_as_float(raw[32 + r]);
        } else {
          tmem_ld16x2(tbase + (uint32_t)c0, tbase + rpa + (uint32_t)c0, raw);
#pragma unroll
          for (int r = 0; r < 16; ++r) v[r] = __uint_as_float(raw[r]) + __uint_as_float(raw[16 + r]);
#pragma unroll
          for (int r = 16; r < 32; ++r) v[r] = 0.f;
        }
        if (KM) {
          float* stg = epi + warp * (32 * 33);
#pragma unroll
          for (int r = 0; r < 32; ++r) stg[lane * 33 + r] = v[r];
          __syncwarp();
          const int64_t r0 = tile * 128 + warp * 32;  // this warp's rows
          const int nrows = (int)std::min<int64_t>(32, p.P - r0);
          const int wc = std::min(w, p.R - c0);    // valid columns of the chunk
          const int dq = 32 / wc, dr = 32 - dq * wc;
          int row = lane / wc, rr = lane - row * wc;
          for (int e = lane; e < nrows * wc; e += 32) {
            const int64_t idx = (r0 + row) * p.R + c0 + rr;
            store_w(p, idx, (PO && p.oh_ld) ? (r0 + row) * p.oh_ld + c0 + rr : idx, stg[row * 33 + rr]);
            row += dq;
            rr += dr;
            if (rr >= wc) {
              rr -= wc;
              ++row;
            }
          }
          __syncwarp();
        } else if (o_row >= 0) {
          const int nc = std::min(w, p.R - c0);
          if (PO && p.oh_ld) {
#pragma unroll
            for (int r = 0; r < 32; ++r)
              if (r < nc) {
                const int64_t idx = o_row + (int64_t)(c0 + r) * p.So;
                store_w(p, idx, (po_srow + (int64_t)(c0 + r) * po_q) * p.oh_ld + po_scol, v[r]);
              }
          } else {
            store_chunk_mn(p, o_row + (int64_t)c0 * p.So, v, nc);
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tail->tempty[acc]));
    }
  }

  // ---------------- teardown ----------------
  __syncthreads();
  if (threadIdx.x == 4 * 32) {
    for (int st = 0; st < p.nst; ++st) {
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
    tmem_dealloc(tmem, p.tmem_cols);
  }
}

size_t tw_tail_bytes(bool km) { return ((sizeof(TwTail) + 15) / 16) * 16 + (km ? 4 * 32 * 33 * sizeof(float) : 0); }

}  // namespace

bool ttm_tc_wide_supported(int64_t P, int64_t K, int64_t S, int R, SplitLayout lay) {
  if (R <= 32 || R > 192 || K < 1 || P < 1 || P > 0x7fffffff || S > 0x7fffffff) return false;
  if (K > 0x3fffffff) return false;
  const TtmView v = ttm_view(K, S, lay);
  if (!v.ok || v.Sit > 0x7fffffff) return false;
  if (S == 1) return (v.ldK % 8) == 0 && (P + 127) / 128 < (int64_t(1) << 31);
  if (v.rowS < 8 || (v.rowS % 8) != 0) return false;
  const int64_t nsb = (v.Sit + 63) / 64;
  return P * nsb <= (int64_t(1) << 40);
}

cudaError_t launch_ttm_tc_wide(const __nv_bfloat16* Xhi, const __nv_bfloat16* Xlo, const __nv_bfloat16* Qt, int Rp,
                               int64_t Kp, float* out, int64_t P, int64_t K, int64_t S, int R,
                               unsigned int* dev_status, cudaStream_t st, __nv_bfloat16* out_hi,
                               __nv_bfloat16* out_lo, SplitLayout lay, SplitLayout out_lay) {
  if (!ttm_tc_wide_supported(P, K, S, R, lay) || Rp % 16 || Rp < R || Rp > 192 || Kp < K || (Kp % 64) != 0)
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
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&tml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)Xlo, dims, strides, box, es,
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
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&tml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)Xlo, dims, strides, box, es,
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
  TwParams prm{};
  prm.P = P;
  prm.K = K;
  prm.S = view.Sit;
  prm.So = view.So;
  prm.s_last = view.s_last;
  prm.s_pad = view.s_pad;
  prm.R = R;
  prm.Rp = Rp;
  prm.nkb = (int)((K + 63) / 64);
  prm.nsb = km ? 1 : (view.Sit + 63) / 64;
  prm.H = P * prm.nsb;
  prm.T = km ? (P + 127) / 128 : (prm.H + 1) / 2;
  prm.out = out;
  prm.out_hi = out_hi;
  prm.out_lo = out_lo;
  prm.oh_last = out_lay.ld ? out_lay.last : 0;
  prm.oh_ld = out_lay.ld;
  prm.status = dev_status;
  if ((int64_t)prm.nkb * 64 > Kp) return cudaErrorInvalidValue;
  prm.stage_bytes = (uint32_t)(TW_A_BYTES + 2 * Rp * 128);
  const int rpa = (Rp + 31) & ~31;
  prm.nbuf = (4 * rpa <= 512) ? 2 : 1;
  const uint32_t need = (uint32_t)(prm.nbuf * 2 * rpa);
  uint32_t cols = 32;
  while (cols < need) cols <<= 1;
  prm.tmem_cols = cols;  // <= 512
  const size_t fixed = 1024 + tw_tail_bytes(km);
  int nst = TW_MAXST;
  while (nst > 2 && fixed + (size_t)nst * prm.stage_bytes > (size_t)TW_SMEM_LIMIT) --nst;
  if (fixed + (size_t)nst * prm.stage_bytes > (size_t)TW_SMEM_LIMIT) return cudaErrorNotSupported;
  prm.nst = nst;
  const size_t smem = fixed + (size_t)nst * prm.stage_bytes;
  const bool po = out_hi && out_lay.ld;
  auto kern = km ? (po ? ttm_tc_wide_kernel<true, true> : ttm_tc_wide_kernel<true, false>)
                  : (po ? ttm_tc_wide_kernel<false, true> : ttm_tc_wide_kernel<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>(prm.T, tc::num_sms());
  kern<<<(unsigned)grid, TW_THREADS, smem, st>>>(tmh, tml, tmq, prm);
  return cudaGetLastError();
}

}  // namespace cpqr
