// FP64 Householder QRs of tall, skinny matrices (R <= 32 columns) on one
// thread-block cluster, for the three QRs of a CP-ALS-QR mode update:
//  * the factor QR A^(n) = Q_n R_n (Alg. 2 line 10), preceded by the
//    extrapolated right-hand side V^ = (1+beta) V0 - alpha beta V1 (eq. 19),
//    the solve A^ R0^T = V^ (line 8) and the column normalisation (line 9);
//  * the QR of the Khatri-Rao product Z_n = R_{k1} (.) ... (.) R_{km} of the
//    other factors' triangles (lines 3-4);
//  * a plain QR (initial factors).
//
// GB300 has ~8 GFLOP/s of FP64 per SM, so these run on a cluster of
// kQrCluster CTAs that own the rows round-robin.  Each Householder column
// costs one cluster barrier: every CTA reduces [x^T x, x^T a_c (c > j), pivot
// row] over its rows, the partial sums are read through distributed shared
// memory, and every CTA applies the reflector to its rows.  Q is formed with
// the compact-WY (UT) representation: Q = E - V T V_top^T with
// T^{-1} = striu(V^T V) + diag(V^T V)/2, one more cluster reduction.
//
// Khatri-Rao rows are processed sorted by the largest index among their
// digits: a row whose digits are <= m is zero in columns < m because every
// R_k is upper triangular, so column j's reflector only touches the first
// (j+1)^m sorted rows and no fill-in escapes that staircase.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace cpqr {

namespace {

constexpr int CL = kQrCluster;
constexpr int NT = kQrThreads;
constexpr int NW = NT / 32;
constexpr int PSLOT = 2 * CPQR_MAXR + 2;  // partial-sum slots per step

enum { MODE_PLAIN = 0, MODE_KRP = 1, MODE_FINISH = 2 };

struct QrParams {
  int mode;
  int64_t M;
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
  double part[2][PSLOT];     // cluster-visible partial sums (double buffered)
  double red[NW][PSLOT];     // per-warp partial sums
  double bcw[CPQR_MAXR];     // broadcast w_c of the current step
  double alpha[CPQR_MAXR];
  double tau[CPQR_MAXR];
  double vpiv[CPQR_MAXR];
  double vtop[CPQR_MAXR][CPQR_MAXR];  // cluster-visible: v_a[t] for rows t < R owned here
  double S[CPQR_MAXR][CPQR_MAXR];     // cluster-visible partial V^T V, then the total
  double W2[CPQR_MAXR][CPQR_MAXR];
  double Ssum[CPQR_MAXR][CPQR_MAXR];
  double R0[CPQR_MAXR][CPQR_MAXR];    // finish: R0; reused as scratch
  double rdiag[CPQR_MAXR];
  double sred[NW][8][CPQR_MAXR];      // S cross-warp reduction, 8 rows of a at a time
  int pad;
};

__device__ __forceinline__ int64_t first_local(int64_t t0, int rank) {
  // smallest local index u with rank + CL*u >= t0
  if (t0 <= rank) return 0;
  return (t0 - rank + CL - 1) / CL;
}

// Row t's lowest column with a nonzero reflector entry (staircase) for KRP mode.
__device__ __forceinline__ int row_alo(const QrParams& p, int64_t t) {
  if (p.mode != MODE_KRP) return 0;
  int a = 0;
  while (a < p.R - 1 && (int64_t)p.act[a] <= t) ++a;
  return a;
}

__device__ __forceinline__ double krp_value(const QrParams& p, int64_t orig, int c) {
  // orig = digits (r_1 .. r_m) base R, r_m fastest
  double v = 1.0;
  int64_t x = orig;
  for (int k = p.krp_m - 1; k >= 0; --k) {
    int r = (int)(x % p.R);
    x /= p.R;
    v *= p.tri.p[k][r * p.R + c];
  }
  return v;
}

__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT, 1) qr_cluster_kernel(QrParams p) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = p.R;
  const int64_t M = p.M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemLayout& sm = *reinterpret_cast<SmemLayout*>(smem_raw);
  double* rows_smem = reinterpret_cast<double*>(smem_raw + ((sizeof(SmemLayout) + 15) / 16) * 16);

  const int64_t L = (M > rank) ? (M - rank + CL - 1) / CL : 0;  // local rows
  double* Wb;
  int64_t ldw;
  if (p.use_smem) {
    Wb = rows_smem;
    ldw = R;
  } else {
    Wb = p.work + (int64_t)rank * R;
    ldw = (int64_t)CL * R;
  }
  auto W = [&](int64_t u) -> double* { return Wb + u * ldw; };
  auto grow = [&](int64_t u) -> int64_t { return rank + (int64_t)CL * u; };

  // ---------------- prologue: fill the local rows ----------------
  if (p.mode == MODE_PLAIN) {
    for (int64_t u = warp; u < L; u += NW)
      if (lane < R) W(u)[lane] = p.A_in[grow(u) * R + lane];
  } else if (p.mode == MODE_KRP) {
    for (int64_t u = warp; u < L; u += NW) {
      int64_t t = grow(u);
      if (lane < R) W(u)[lane] = krp_value(p, (int64_t)p.perm[t], lane);
    }
  } else {
    // MODE_FINISH: V^ per row, back substitution A^ R0^T = V^, column norms.
    for (int i = tid; i < R * R; i += NT) sm.R0[i / R][i % R] = p.R0[i];
    __syncthreads();
    if (tid < R) {
      double d = sm.R0[tid][tid];
      sm.rdiag[tid] = (d != 0.0) ? 1.0 / d : 0.0;
      if (d == 0.0 && rank == 0) atomicOr(p.status, CPQR_DEV_SINGULAR);
    }
    __syncthreads();
    const bool ext = (p.C == 2 * R);
    const double c0 = 1.0 + p.beta, c1 = -p.alpha * p.beta;
    double nrm = 0.0, f_in = 0.0, f_nn = 0.0;
    for (int64_t u = warp; u < L; u += NW) {
      int64_t t = grow(u);
      double v0 = 0.0, vh = 0.0;
      if (lane < R) {
        v0 = p.V[t * p.C + lane];
        vh = ext ? (c0 * v0 + c1 * p.V[t * p.C + R + lane]) : v0;
      }
      f_in += v0 * vh;
      f_nn += vh * vh;
      // back substitution, lanes hold the residual of their column
      double res = vh, ahat = 0.0;
      for (int c = R - 1; c >= 0; --c) {
        double a_c = __shfl_sync(0xffffffffu, res, c) * sm.rdiag[c];
        if (lane == c) ahat = a_c;
        if (lane < c) res -= sm.R0[lane][c] * a_c;
      }
      if (lane < R) W(u)[lane] = ahat;
      nrm += ahat * ahat;
    }
    // reduce: slots 0..R-1 column norms, 2R: <V0, V^>, 2R+1: ||V^||^2
    for (int o = 16; o > 0; o >>= 1) {
      f_in += __shfl_xor_sync(0xffffffffu, f_in, o);
      f_nn += __shfl_xor_sync(0xffffffffu, f_nn, o);
    }
    sm.red[warp][lane] = nrm;
    if (lane == 0) {
      sm.red[warp][2 * CPQR_MAXR] = f_in;
      sm.red[warp][2 * CPQR_MAXR + 1] = f_nn;
    }
    __syncthreads();
    if (warp == 0) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int w = 0; w < NW; ++w) {
        a += sm.red[w][lane];
        if (lane == 0) {
          b += sm.red[w][2 * CPQR_MAXR];
          c += sm.red[w][2 * CPQR_MAXR + 1];
        }
      }
      sm.part[1][lane] = a;
      if (lane == 0) {
        sm.part[1][2 * CPQR_MAXR] = b;
        sm.part[1][2 * CPQR_MAXR + 1] = c;
      }
    }
    cluster.sync();
    if (warp == 0) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int r = 0; r < CL; ++r) {
        const double* rp = cluster.map_shared_rank(&sm.part[1][0], r);
        a += rp[lane];
        if (lane == 0) {
          b += rp[2 * CPQR_MAXR];
          c += rp[2 * CPQR_MAXR + 1];
        }
      }
      double lam = sqrt(a);
      if (lane < R) {
        sm.bcw[lane] = (lam > 0.0) ? 1.0 / lam : 0.0;
        if (lam == 0.0 && rank == 0) atomicOr(p.status, CPQR_DEV_SINGULAR);
        if (rank == 0) p.fin.lambda[lane] = lam;
      }
      if (lane == 0 && rank == 0) {
        p.fin.fit_terms[0] = b;
        p.fin.fit_terms[1] = c;
      }
    }
    __syncthreads();
    for (int64_t u = warp; u < L; u += NW) {
      if (lane < R) {
        double a = W(u)[lane] * sm.bcw[lane];
        W(u)[lane] = a;
        p.fin.A[grow(u) * R + lane] = a;
      }
    }
  }
  __syncthreads();

  // ---------------- Householder steps ----------------
  for (int j = 0; j < R; ++j) {
    const int buf = j & 1;
    const int64_t actj = p.act[j];
    const int64_t u0 = first_local(j, rank);
    const int64_t u1 = (actj > rank) ? (actj - rank + CL - 1) / CL : 0;
    int64_t us = u0 + (((warp - u0) % NW) + NW) % NW;
    double acc = 0.0, piv = 0.0;
    for (int64_t u = us; u < u1; u += NW) {
      const double* w = W(u);
      double x = w[j];
      double a = (lane < R) ? w[lane] : 0.0;
      if (lane >= j) acc += x * a;
      if (grow(u) == j) piv = a;
    }
    sm.red[warp][lane] = acc;
    sm.red[warp][CPQR_MAXR + lane] = piv;
    __syncthreads();
    if (warp == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < NW; ++w) {
        a += sm.red[w][lane];
        b += sm.red[w][CPQR_MAXR + lane];
      }
      sm.part[buf][lane] = a;
      sm.part[buf][CPQR_MAXR + lane] = b;
    }
    cluster.sync();
    if (warp == 0) {
      double d = 0.0, pv = 0.0;
      for (int r = 0; r < CL; ++r) {
        const double* rp = cluster.map_shared_rank(&sm.part[buf][0], r);
        d += rp[lane];
        pv += rp[CPQR_MAXR + lane];
      }
      double s = __shfl_sync(0xffffffffu, d, j);
      double xj = __shfl_sync(0xffffffffu, pv, j);
      double alpha = 0.0, tau = 0.0, vp = 0.0;
      if (s > 0.0) {
        double nx = sqrt(s);
        alpha = (xj >= 0.0) ? -nx : nx;
        vp = xj - alpha;
        tau = 1.0 / (s - alpha * xj);  // 2 / ||v||^2 with ||v||^2 = 2 (s - alpha xj)
      }
      sm.bcw[lane] = (lane > j && lane < R) ? (d - alpha * pv) : 0.0;
      if (lane == 0 && rank == 0 && !(s > 0.0)) atomicOr(p.status, CPQR_DEV_SINGULAR);
      if (lane == 0) {
        sm.alpha[j] = alpha;
        sm.tau[j] = tau;
        sm.vpiv[j] = vp;
      }
    }
    __syncthreads();
    if (lane > j && lane < R) {
      const double tau = sm.tau[j], wc = sm.bcw[lane], vp = sm.vpiv[j];
      const double tw = tau * wc;
      for (int64_t u = us; u < u1; u += NW) {
        double* w = W(u);
        double v = (grow(u) == j) ? vp : w[j];
        w[lane] -= tw * v;
      }
    }
    __syncwarp();
    if (lane == j) {
      for (int64_t u = us; u < u1; u += NW)
        if (grow(u) == j) W(u)[j] = sm.alpha[j];
    }
    __syncthreads();
  }

  // reflector entry v_a[t] of local row u (t = grow(u))
  auto vref = [&](int64_t u, int64_t t, int a) -> double {
    if (t < a || t >= (int64_t)p.act[a]) return 0.0;
    if (t == a) return sm.vpiv[a];
    return W(u)[a];
  };

  // ---------------- R factor (positive diagonal) ----------------
  for (int64_t u = warp; u < L; u += NW) {
    int64_t t = grow(u);
    if (t >= R) break;
    if (lane < R) {
      double sg = (sm.alpha[t] < 0.0) ? -1.0 : 1.0;
      double v = (lane < t) ? 0.0 : (lane == t ? sm.alpha[t] : W(u)[lane]);
      p.Rout[t * R + lane] = sg * v;
    }
  }

  // ---------------- compact WY: S = V^T V ----------------
  // vtop rows (t < R) for every CTA
  for (int i = tid; i < CPQR_MAXR * CPQR_MAXR; i += NT) (&sm.vtop[0][0])[i] = 0.0;
  __syncthreads();
  for (int64_t u = warp; u < L; u += NW) {
    int64_t t = grow(u);
    if (t >= R) break;
    if (lane < R) sm.vtop[t][lane] = vref(u, t, lane);
  }
  {
    double acc[CPQR_MAXR];
#pragma unroll
    for (int a = 0; a < CPQR_MAXR; ++a) acc[a] = 0.0;
    if (lane < R) {
      const int b = lane;
      for (int64_t u = warp; u < L; u += NW) {
        int64_t t = grow(u);
        double vb = vref(u, t, b);
        if (vb == 0.0) continue;
        int alo = row_alo(p, t);
#pragma unroll
        for (int a = 0; a < CPQR_MAXR; ++a)
          if (a >= alo && a <= b) acc[a] += vref(u, t, a) * vb;
      }
    }
#pragma unroll
    for (int a0 = 0; a0 < CPQR_MAXR; a0 += 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q) sm.sred[warp][q][lane] = acc[a0 + q];
      __syncthreads();
      {
        int q = tid >> 5, b = tid & 31;  // 8 x 32 entries, one per thread
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += sm.sred[w][q][b];
        sm.S[a0 + q][b] = s;
      }
      __syncthreads();
    }
  }
  cluster.sync();
  for (int i = tid; i < CPQR_MAXR * CPQR_MAXR; i += NT) {
    double s = 0.0, vt = 0.0;
    for (int r = 0; r < CL; ++r) {
      s += cluster.map_shared_rank(&sm.S[0][0], r)[i];
      vt += cluster.map_shared_rank(&sm.vtop[0][0], r)[i];
    }
    (&sm.Ssum[0][0])[i] = s;
    (&sm.R0[0][0])[i] = vt;  // all rows t < R of V: R0[t][a] = v_a[t]
  }
  cluster.sync();  // remote reads done before anyone moves on / exits
  // W2 = T V_top^T, i.e. solve Tinv W2 = V_top^T, Tinv = striu(S) + diag(S)/2 (upper).
  if (warp == 0 && lane < R) {
    const int c = lane;
    for (int a = R - 1; a >= 0; --a) {
      double rhs = (c >= a) ? sm.R0[c][a] : 0.0;  // V_top^T[a][c] = v_a[c]
      for (int b = a + 1; b < R; ++b) rhs -= sm.Ssum[a][b] * sm.W2[b][c];
      double dg = 0.5 * sm.Ssum[a][a];
      sm.W2[a][c] = (dg > 0.0) ? rhs / dg : 0.0;
    }
  }
  __syncthreads();

  // ---------------- Q rows ----------------
  for (int64_t u = warp; u < L; u += NW) {
    int64_t t = grow(u);
    if (lane >= R) continue;
    const int c = lane;
    int alo = row_alo(p, t);
    int ahi = (int)((t < c) ? t : c);
    double q = (t == c) ? 1.0 : 0.0;
    for (int a = alo; a <= ahi; ++a) q -= vref(u, t, a) * sm.W2[a][c];
    q *= (sm.alpha[c] < 0.0) ? -1.0 : 1.0;
    int64_t orow = (p.mode == MODE_KRP) ? (int64_t)p.perm[t] : t;
    p.Q[orow * R + c] = q;
    if (p.mode == MODE_FINISH && p.fin.Qf) p.fin.Qf[orow * R + c] = (float)q;
  }
}

size_t smem_bytes(int64_t M, int R, bool use_smem) {
  size_t base = ((sizeof(SmemLayout) + 15) / 16) * 16;
  if (!use_smem) return base;
  int64_t L = (M + CL - 1) / CL;
  return base + (size_t)L * R * sizeof(double);
}

constexpr size_t kSmemRowBudget = 160 * 1024;

cudaError_t run(QrParams& p, cudaStream_t st) {
  int64_t L = (p.M + CL - 1) / CL;
  p.use_smem = ((size_t)L * p.R * sizeof(double) <= kSmemRowBudget) ? 1 : 0;
  if (!p.use_smem && p.work == nullptr) return cudaErrorInvalidValue;
  size_t sm = smem_bytes(p.M, p.R, p.use_smem);
  cudaError_t e = cudaFuncSetAttribute(qr_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  qr_cluster_kernel<<<CL, NT, sm, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

size_t house_qr_work_doubles(int64_t M, int R) { return (size_t)M * R; }
size_t krp_qr_work_doubles(const ZPlan& plan) { return (size_t)plan.M * plan.R; }

cudaError_t launch_house_qr(const double* A, int64_t M, int R, double* Q, double* Rout, double* work,
                            unsigned int* dev_status, cudaStream_t st) {
  if (R < 1 || R > CPQR_MAXR || M < R) return cudaErrorInvalidValue;
  QrParams p{};
  p.mode = MODE_PLAIN;
  p.M = M;
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
  p.M = plan.M;
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
  p.M = I;
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
