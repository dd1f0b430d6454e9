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
// round-robin.  Each Householder column costs one cluster barrier: every CTA
// reduces [x^T a_c (c >= j), pivot row] over its rows and pushes the sums into
// every peer's shared memory before the barrier, so after it the reduction is
// local; every CTA then applies the reflector to its rows.  Q is formed with
// the compact-WY (UT) representation: Q = E - V T V_top^T with
// T^{-1} = striu(V^T V) + diag(V^T V)/2 (reduce-scatter + all-gather of V^T V
// over the cluster, two more barriers).
//
// Khatri-Rao rows are processed sorted by the largest index among their
// digits: a row whose digits are <= m is zero in columns < m because every
// R_k is upper triangular, so column j's reflector only touches the first
// (j+1)^m sorted rows and no fill-in escapes that staircase.
#include <cooperative_groups.h>

#include <cstdlib>

#include "common.cuh"

namespace cg = cooperative_groups;

#ifdef CPQR_QR_PHASES
__device__ unsigned long long g_qr_phase[8];
#define QR_PHASE(i)                                                              \
  do {                                                                           \
    if (threadIdx.x == 0 && cluster.block_rank() == 0) {                         \
      unsigned long long t_;                                                     \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                     \
      g_qr_phase[i] = t_;                                                        \
    }                                                                            \
  } while (0)
#else
#define QR_PHASE(i) \
  do {              \
  } while (0)
#endif

namespace cpqr {

namespace {

constexpr int NT = kQrThreads;
constexpr int NW = NT / 32;
constexpr int MAXCL = 16;
constexpr int PSLOT = 2 * CPQR_MAXR + 2;  // partial-sum slots per step
constexpr int RR = CPQR_MAXR * CPQR_MAXR;

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
  const double* V;
  int C;
  const double* R0;
  double beta, alpha;
  FinishOut fin;
  // outputs
  double* Q;
  double* Rout;
  unsigned int* status;
};

struct SmemLayout {
  double inbox[2][MAXCL][PSLOT];  // partial sums pushed by every CTA of the cluster (double buffered)
  double pivbox[2][CPQR_MAXR];    // pivot row of the current column, pushed by its owner CTA
  double pivloc[CPQR_MAXR];       // pivot row as seen by the owning warp
  double dvec[CPQR_MAXR];         // cluster-wide x^T a_c of the current column
  double red[NW][PSLOT];          // per-warp partial sums
  double bcw[CPQR_MAXR];          // broadcast w_c of the current step
  double alpha[CPQR_MAXR];
  double tau[CPQR_MAXR];
  double vpiv[CPQR_MAXR];
  double spart[RR];               // this CTA's partial V^T V (upper entries), then scratch
  double sinbox[MAXCL][RR / 8];   // reduce-scatter inbox: entries i with i % CL == rank
  double Ssum[RR];                // total V^T V
  double vtop[RR];                // v_a[t] for t < R (row-major [t][a]) of the whole cluster
  double W2[RR];
  double R0[RR];                  // finish: R0
  double rdiag[CPQR_MAXR];
};

// Row t's lowest column with a nonzero reflector entry (staircase) for KRP mode.
__device__ __forceinline__ int row_alo(const QrParams& p, int t) {
  if (p.mode != MODE_KRP) return 0;
  int a = 0;
  while (a < p.R - 1 && p.act[a] <= t) ++a;
  return a;
}

__device__ __forceinline__ double krp_value(const QrParams& p, int orig, int c) {
  // orig = digits (r_1 .. r_m) base R, r_m fastest
  double v = 1.0;
  int x = orig;
  for (int k = p.krp_m - 1; k >= 0; --k) {
    int r = x % p.R;
    x /= p.R;
    v *= p.tri.p[k][r * p.R + c];
  }
  return v;
}

__device__ __forceinline__ double tree8(const double* v, int stride) {
  return ((v[0] + v[stride]) + (v[2 * stride] + v[3 * stride])) +
         ((v[4 * stride] + v[5 * stride]) + (v[6 * stride] + v[7 * stride]));
}

template <int CL>
__global__ void __launch_bounds__(NT, 1) qr_cluster_kernel(QrParams p) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = p.R;
  const int M = p.M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemLayout& sm = *reinterpret_cast<SmemLayout*>(smem_raw);
  double* rows_smem = reinterpret_cast<double*>(smem_raw + ((sizeof(SmemLayout) + 15) / 16) * 16);

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

  // Warp 0 sums the per-warp vectors red[*][0..n) and pushes the CTA total into
  // inbox[buf][rank] of every CTA of the cluster.
  auto push_partials = [&](int buf, int n0, int n1) {
    __syncthreads();
    if (warp == 0) {
      for (int i = n0 + lane; i < n1; i += 32) {
        double v = tree8(&sm.red[0][i], PSLOT);
        for (int r = 0; r < CL; ++r) cluster.map_shared_rank(&sm.inbox[buf][rank][0], r)[i] = v;
      }
    }
    cluster.sync();
  };
  auto inbox_sum = [&](int buf, int i) -> double {
    double s[MAXCL / 2];
#pragma unroll
    for (int h = 0; h < CL / 2; ++h) s[h] = sm.inbox[buf][2 * h][i] + sm.inbox[buf][2 * h + 1][i];
#pragma unroll
    for (int w = CL / 4; w >= 1; w >>= 1)
#pragma unroll
      for (int h = 0; h < w; ++h) s[h] += s[h + w];
    return s[0];
  };

  QR_PHASE(0);
  // ---------------- prologue: fill the local rows ----------------
  if (p.mode == MODE_PLAIN) {
    for (int u = warp; u < L; u += NW)
      if (lane < R) W(u)[lane] = p.A_in[(size_t)grow(u) * R + lane];
  } else if (p.mode == MODE_KRP) {
    for (int u = warp; u < L; u += NW)
      if (lane < R) W(u)[lane] = krp_value(p, p.perm[grow(u)], lane);
  } else {
    // MODE_FINISH: V^ per row, back substitution A^ R0^T = V^, column norms.
    for (int i = tid; i < R * R; i += NT) sm.R0[(i / R) * CPQR_MAXR + i % R] = p.R0[i];
    __syncthreads();
    if (tid < R) {
      double d = sm.R0[tid * CPQR_MAXR + tid];
      sm.rdiag[tid] = (d != 0.0) ? 1.0 / d : 0.0;
      if (d == 0.0 && rank == 0) atomicOr(p.status, CPQR_DEV_SINGULAR);
    }
    __syncthreads();
    const bool ext = (p.C == 2 * R);
    const double c0 = 1.0 + p.beta, c1 = -p.alpha * p.beta;
    double nrm = 0.0, f_in = 0.0, f_nn = 0.0;
    for (int u = warp; u < L; u += NW) {
      const size_t t = (size_t)grow(u);
      double v0 = 0.0, vh = 0.0;
      if (lane < R) {
        v0 = p.V[t * p.C + lane];
        vh = ext ? (c0 * v0 + c1 * p.V[t * p.C + R + lane]) : v0;
      }
      f_in += v0 * vh;
      f_nn += vh * vh;
      double res = vh, ahat = 0.0;
      for (int c = R - 1; c >= 0; --c) {
        double a_c = __shfl_sync(0xffffffffu, res, c) * sm.rdiag[c];
        if (lane == c) ahat = a_c;
        if (lane < c) res -= sm.R0[lane * CPQR_MAXR + c] * a_c;
      }
      if (lane < R) W(u)[lane] = ahat;
      nrm += ahat * ahat;
    }
    for (int o = 16; o > 0; o >>= 1) {
      f_in += __shfl_xor_sync(0xffffffffu, f_in, o);
      f_nn += __shfl_xor_sync(0xffffffffu, f_nn, o);
    }
    sm.red[warp][lane] = nrm;
    if (lane == 0) {
      sm.red[warp][2 * CPQR_MAXR] = f_in;
      sm.red[warp][2 * CPQR_MAXR + 1] = f_nn;
    }
    push_partials(1, 0, PSLOT);
    if (warp == 0) {
      double lam = sqrt(inbox_sum(1, lane));
      if (lane < R) {
        sm.bcw[lane] = (lam > 0.0) ? 1.0 / lam : 0.0;
        if (lam == 0.0 && rank == 0) atomicOr(p.status, CPQR_DEV_SINGULAR);
        if (rank == 0) p.fin.lambda[lane] = lam;
      }
      if (lane == 0 && rank == 0) {
        p.fin.fit_terms[0] = inbox_sum(1, 2 * CPQR_MAXR);
        p.fin.fit_terms[1] = inbox_sum(1, 2 * CPQR_MAXR + 1);
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
  __syncwarp();
  QR_PHASE(1);

  // ---------------- Householder steps: one cluster barrier per column ----------------
  // FP64 instructions cost ~64 cycles per warp on GB300, so the reductions are
  // split over warps 0..3 (one per SM sub-partition) and the pivot row, owned by
  // a single CTA, is pushed instead of reduced.
  constexpr int IPG = CL / 4;  // inboxes summed by each of the 4 lane groups
  for (int j = 0; j < R; ++j) {
    const int buf = j & 1;
    const int actj = p.act[j];
    const int u0 = (j <= rank) ? 0 : (j - rank + CL - 1) / CL;
    const int u1 = (actj > rank) ? (actj - rank + CL - 1) / CL : 0;
    const int us = u0 + ((warp - (u0 % NW)) + NW) % NW;
    double acc = 0.0;
    for (int u = us; u < u1; u += NW) {
      const double* w = W(u);
      double x = w[j];
      double a = (lane < R) ? w[lane] : 0.0;
      if (lane >= j) acc += x * a;
      if (grow(u) == j) sm.pivloc[lane] = a;
    }
    sm.red[warp][lane] = acc;
    __syncthreads();
    if (warp < 4) {
      const int slot = 8 * warp + (lane & 7), g = lane >> 3;
      double v = sm.red[2 * g][slot] + sm.red[2 * g + 1][slot];
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      for (int r = g; r < CL; r += 4) cluster.map_shared_rank(&sm.inbox[buf][rank][0], r)[slot] = v;
    } else if (warp == 4 && rank == j % CL) {
      const double pvv = sm.pivloc[lane];
      for (int r = 0; r < CL; ++r) cluster.map_shared_rank(&sm.pivbox[buf][0], r)[lane] = pvv;
    }
    cluster.sync();
    if (warp < 4) {
      const int slot = 8 * warp + (lane & 7), g = lane >> 3;
      double v = sm.inbox[buf][g * IPG][slot];
#pragma unroll
      for (int q = 1; q < IPG; ++q) v += sm.inbox[buf][g * IPG + q][slot];
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      if (g == 0) sm.dvec[slot] = v;
    }
    __syncthreads();
    if (warp == 0) {
      const double s = sm.dvec[j], xj = sm.pivbox[buf][j];
      double alpha = 0.0, tau = 0.0, vp = 0.0;
      if (s > 0.0) {
        double nx = sqrt(s);
        alpha = (xj >= 0.0) ? -nx : nx;
        vp = xj - alpha;
        tau = 1.0 / (s - alpha * xj);  // 2 / ||v||^2 with ||v||^2 = 2 (s - alpha xj)
      }
      sm.bcw[lane] = (lane > j && lane < R) ? tau * (sm.dvec[lane] - alpha * sm.pivbox[buf][lane]) : 0.0;
      if (lane == 0 && rank == 0 && !(s > 0.0)) atomicOr(p.status, CPQR_DEV_SINGULAR);
      if (lane == 0) {
        sm.alpha[j] = alpha;
        sm.tau[j] = tau;
        sm.vpiv[j] = vp;
      }
    }
    __syncthreads();
    {
      const double tw = sm.bcw[lane], vp = sm.vpiv[j], al = sm.alpha[j];
      for (int u = us; u < u1; u += NW) {
        double* w = W(u);
        const bool pivrow = (grow(u) == j);
        double v = pivrow ? vp : w[j];
        if (lane > j && lane < R) w[lane] -= tw * v;
        __syncwarp();
        if (pivrow && lane == j) w[j] = al;
      }
    }
    __syncwarp();
  }

  // reflector entry v_a[t] of local row u (t = grow(u))
  auto vref = [&](int u, int t, int a) -> double {
    if (t < a || t >= p.act[a]) return 0.0;
    if (t == a) return sm.vpiv[a];
    return W(u)[a];
  };

  // ---------------- R factor (positive diagonal) ----------------
  __syncthreads();
  QR_PHASE(2);
  for (int u = warp; u < L; u += NW) {
    int t = grow(u);
    if (t >= R) break;
    if (lane < R) {
      double sg = (sm.alpha[t] < 0.0) ? -1.0 : 1.0;
      double v = (lane < t) ? 0.0 : (lane == t ? sm.alpha[t] : W(u)[lane]);
      p.Rout[t * R + lane] = sg * v;
    }
  }

  // ---------------- compact WY: S = V^T V (reduce-scatter, then all-gather) ----------------
  // upper entries (a, b), a <= b < R, packed densely over the threads
  for (int e = tid; e < RR; e += NT) sm.spart[e] = 0.0;
  __syncthreads();
  {
    const int nup = R * (R + 1) / 2;
    for (int k = tid; k < nup; k += NT) {
      // k -> (a, b): rows a have R - a entries
      int a = 0, rem = k;
      while (rem >= R - a) {
        rem -= R - a;
        ++a;
      }
      const int b = a + rem;
      double acc = 0.0;
      // v_a[t] is nonzero only for a <= t < act[a]; v_b[t] needs t >= b
      const int ulo = (b <= rank) ? 0 : (b - rank + CL - 1) / CL;
      const int uhi = (p.act[a] > rank) ? (p.act[a] - rank + CL - 1) / CL : 0;
      for (int u = ulo; u < uhi; ++u) {
        const int t = grow(u);
        acc += vref(u, t, a) * vref(u, t, b);
      }
      sm.spart[a * CPQR_MAXR + b] = acc;
    }
  }
  // vtop rows owned here, zero elsewhere (summed over the cluster below)
  __syncthreads();
  QR_PHASE(3);
  for (int e = tid; e < RR; e += NT) {
    const int r = e % CL, k = e / CL;
    cluster.map_shared_rank(&sm.sinbox[rank][0], r)[k] = sm.spart[e];
  }
  cluster.sync();
  for (int k = tid; k < RR / CL; k += NT) {
    const int e = k * CL + rank;
    double v = 0.0;
    for (int r = 0; r < CL; ++r) v += sm.sinbox[r][k];
    for (int r = 0; r < CL; ++r) cluster.map_shared_rank(&sm.Ssum[0], r)[e] = v;
  }
  for (int u = warp; u < L; u += NW) {
    int t = grow(u);
    if (t >= R) break;
    double v = (lane < R) ? vref(u, t, lane) : 0.0;
    for (int r = 0; r < CL; ++r) cluster.map_shared_rank(&sm.vtop[0], r)[t * CPQR_MAXR + lane] = v;
  }
  cluster.sync();  // every remote write is done: no DSMEM access after this point
  QR_PHASE(4);
  // W2 = T V_top^T, i.e. solve Tinv W2 = V_top^T, Tinv = striu(S) + diag(S)/2 (upper),
  // blocked by 8 rows: off-block products on all warps, 8 x 8 diagonal solves on warp 0.
  if (warp == 0) {
    const int c = lane;
    double dg = (c < R) ? 0.5 * sm.Ssum[c * CPQR_MAXR + c] : 0.0;
    sm.rdiag[c] = (dg > 0.0) ? 1.0 / dg : 0.0;
  }
  for (int e = tid; e < RR; e += NT) sm.W2[e] = 0.0;
  __syncthreads();
  for (int kb = (R - 1) / 8; kb >= 0; --kb) {
    const int a0 = kb * 8, a1 = (a0 + 8 < R) ? a0 + 8 : R;
    {
      const int a = a0 + warp, c = lane;  // one row of the block per warp
      if (a < a1 && c < R) {
        double rhs = (c >= a) ? sm.vtop[c * CPQR_MAXR + a] : 0.0;  // V_top^T[a][c] = v_a[c]
        for (int b = a1; b < R; ++b) rhs -= sm.Ssum[a * CPQR_MAXR + b] * sm.W2[b * CPQR_MAXR + c];
        sm.spart[a * CPQR_MAXR + c] = rhs;
      }
    }
    __syncthreads();
    if (warp == 0 && lane < R) {
      const int c = lane;
      for (int a = a1 - 1; a >= a0; --a) {
        double rhs = sm.spart[a * CPQR_MAXR + c];
        for (int b = a + 1; b < a1; ++b) rhs -= sm.Ssum[a * CPQR_MAXR + b] * sm.W2[b * CPQR_MAXR + c];
        sm.W2[a * CPQR_MAXR + c] = rhs * sm.rdiag[a];
      }
    }
    __syncthreads();
  }
  QR_PHASE(5);

  // ---------------- Q rows: Q[t, c] = sign_c (delta_tc - sum_a v_a[t] W2[a][c]) ----------------
  for (int u = warp; u < L; u += NW) {
    const int t = grow(u);
    if (lane >= R) continue;
    const int c = lane;
    const int alo = row_alo(p, t);
    const int ahi = (t < c) ? t : c;
    double q = (t == c) ? 1.0 : 0.0;
    for (int a = alo; a <= ahi; ++a) q -= vref(u, t, a) * sm.W2[a * CPQR_MAXR + c];
    q *= (sm.alpha[c] < 0.0) ? -1.0 : 1.0;
    const size_t orow = (p.mode == MODE_KRP) ? (size_t)p.perm[t] : (size_t)t;
    p.Q[orow * R + c] = q;
    if (p.mode == MODE_FINISH && p.fin.Qf) p.fin.Qf[orow * R + c] = (float)q;
  }
  __syncthreads();
  QR_PHASE(6);
}

size_t smem_bytes(int M, int R, int CL, bool use_smem) {
  size_t base = ((sizeof(SmemLayout) + 15) / 16) * 16;
  if (!use_smem) return base;
  size_t L = (size_t)(M + CL - 1) / CL;
  return base + L * R * sizeof(double);
}

constexpr size_t kSmemMax = 227 * 1024;

int g_cluster = 0;  // cluster size in use (16 if the device allows it, else 8)

template <int CL>
cudaError_t launch_cl(QrParams& p, cudaStream_t st) {
  size_t base = smem_bytes(p.M, p.R, CL, false);
  size_t full = smem_bytes(p.M, p.R, CL, true);
  p.use_smem = (full <= kSmemMax) ? 1 : 0;
  if (!p.use_smem && p.work == nullptr) return cudaErrorInvalidValue;
  size_t sm = p.use_smem ? full : base;
  cudaError_t e = cudaFuncSetAttribute(qr_cluster_kernel<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  if (CL > 8) {
    e = cudaFuncSetAttribute(qr_cluster_kernel<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = sm;
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

#ifdef CPQR_QR_PHASES
// Profiling build only: %globaltimer stamps of the last cluster-QR launch (rank 0).
extern "C" void cpqr_debug_qr_phases(unsigned long long* out) {
  cudaMemcpyFromSymbol(out, g_qr_phase, sizeof(g_qr_phase));
}
#endif

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
                          unsigned int* dev_status, cudaStream_t st) {
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
  p.Rout = R0;
  p.status = dev_status;
  return run(p, st);
}

cudaError_t launch_mode_finish(const double* V, int C, const double* R0, double beta, double alpha,
                               int64_t I, int R, FinishOut out, double* work, unsigned int* dev_status,
                               cudaStream_t st) {
  QrParams p{};
  p.mode = MODE_FINISH;
  if (I > (int64_t(1) << 30)) return cudaErrorInvalidValue;
  p.M = (int)I;
  p.R = R;
  p.work = work;
  for (int j = 0; j < CPQR_MAXR; ++j) p.act[j] = (int32_t)I;
  p.V = V;
  p.C = C;
  p.R0 = R0;
  p.beta = beta;
  p.alpha = alpha;
  p.fin = out;
  p.Q = out.Q;
  p.Rout = out.Rn;
  p.status = dev_status;
  return run(p, st);
}

}  // namespace cpqr
