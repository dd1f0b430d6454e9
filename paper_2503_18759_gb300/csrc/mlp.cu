// Learned extrapolation proposer: a multilayer perceptron with three hidden
// layers of 128 units (ReLU) mapping the features of the last sweeps to logits
// over CPQR_MLP_CLASSES candidate values of beta (eq. 19).  Weights and
// activations are stored in bf16, every product is accumulated in FP32; master
// weights and Adam moments are FP32.
//
// Parameter vector (FP32), layer l = 0..3 with (in, out) = (F,H), (H,H), (H,H), (H,C):
//   [W_l (out x in, row-major), b_l (out)] concatenated.
#include "../../include/cpqr.h"
#include "common.cuh"

namespace cpqr {

namespace {

constexpr int F = CPQR_MLP_FEATURES;
constexpr int H = CPQR_MLP_HIDDEN;
constexpr int NC = CPQR_MLP_CLASSES;
constexpr int NL = 4;

__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? F : H; }
__host__ __device__ constexpr int layer_out(int l) { return l == NL - 1 ? NC : H; }
__host__ __device__ constexpr int layer_off(int l) {
  return l == 0 ? 0 : layer_off(l - 1) + layer_in(l - 1) * layer_out(l - 1) + layer_out(l - 1);
}
static_assert(layer_off(NL) == CPQR_MLP_NPARAMS, "parameter count");

__global__ void to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// Y[b, o] = act(sum_i X[b, i] W[o, i] + bias[o]), X and W bf16, FP32 accumulate, Y bf16
// (hidden layers, ReLU) or FP32 logits (last layer, no activation).
__global__ void fwd_layer_kernel(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ Wb,
                                 const float* __restrict__ bias_f32, int B, int in, int out, int relu,
                                 __nv_bfloat16* __restrict__ Yb, float* __restrict__ Yf) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (o >= out || b >= B) return;
  const __nv_bfloat16* x = X + (size_t)b * in;
  const __nv_bfloat16* w = Wb + (size_t)o * in;
  float acc = bias_f32[o];
  for (int i = 0; i < in; ++i) acc += __bfloat162float(x[i]) * __bfloat162float(w[i]);
  if (relu) acc = acc > 0.f ? acc : 0.f;
  if (Yb) Yb[(size_t)b * out + o] = __float2bfloat16_rn(acc);
  if (Yf) Yf[(size_t)b * out + o] = acc;
}

// Mean softmax cross-entropy; dlogits = (softmax - onehot) / B.
__global__ void softmax_xent_kernel(const float* __restrict__ logits, const int32_t* __restrict__ y, int B,
                                    float* __restrict__ dlogits, float* __restrict__ loss) {
  __shared__ float sl[256];
  float l = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float* z = logits + (size_t)b * NC;
    float mx = z[0];
    for (int c = 1; c < NC; ++c) mx = fmaxf(mx, z[c]);
    float s = 0.f;
    for (int c = 0; c < NC; ++c) s += __expf(z[c] - mx);
    const int t = y[b];
    for (int c = 0; c < NC; ++c) {
      float p = __expf(z[c] - mx) / s;
      dlogits[(size_t)b * NC + c] = (p - (c == t ? 1.f : 0.f)) / (float)B;
    }
    l += (mx + __logf(s)) - z[t];
  }
  sl[threadIdx.x] = l;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sl[threadIdx.x] += sl[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sl[0] / (float)B;
}

// dZ[b, o] = dY[b, o] * relu'(Y[b, o]) (hidden layers; the last layer passes dY through).
// dX[b, i] = sum_o dZ[b, o] W[o, i]   (bf16 W, FP32 accumulate)
__global__ void bwd_dx_kernel(const float* __restrict__ dZ, const __nv_bfloat16* __restrict__ Wb, int B, int in,
                              int out, const __nv_bfloat16* __restrict__ Xprev_act, float* __restrict__ dX) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= in || b >= B) return;
  float acc = 0.f;
  for (int o = 0; o < out; ++o) acc += dZ[(size_t)b * out + o] * __bfloat162float(Wb[(size_t)o * in + i]);
  // the input of this layer is the previous layer's ReLU output: mask by it
  if (Xprev_act && !(__bfloat162float(Xprev_act[(size_t)b * in + i]) > 0.f)) acc = 0.f;
  dX[(size_t)b * in + i] = acc;
}

// dW[o, i] = sum_b dZ[b, o] X[b, i]; db[o] = sum_b dZ[b, o]
__global__ void bwd_dw_kernel(const float* __restrict__ dZ, const __nv_bfloat16* __restrict__ X, int B, int in,
                              int out, float* __restrict__ gW, float* __restrict__ gb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y;
  if (o >= out) return;
  if (i < in) {
    float acc = 0.f;
    for (int b = 0; b < B; ++b) acc += dZ[(size_t)b * out + o] * __bfloat162float(X[(size_t)b * in + i]);
    gW[(size_t)o * in + i] = acc;
  }
  if (i == in) {
    float acc = 0.f;
    for (int b = 0; b < B; ++b) acc += dZ[(size_t)b * out + o];
    gb[o] = acc;
  }
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// bf16 copy of the weights, each layer transposed to (in x out) so that the threads of a layer
// (one output each) read consecutive addresses.
__global__ void prepare_weights_kernel(const float* __restrict__ params, __nv_bfloat16* __restrict__ wt) {
  for (int l = 0; l < NL; ++l) {
    const int in = layer_in(l), out = layer_out(l);
    const float* W = params + layer_off(l);
    __nv_bfloat16* T = wt + layer_off(l);  // same offsets; the bias slots stay unused
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < in * out; e += gridDim.x * blockDim.x) {
      const int o = e / in, i = e - o * in;
      T[i * out + o] = __float2bfloat16_rn(W[e]);
    }
  }
}

__device__ double beta_band_dev(double fit) {
  if (fit > 0.95) return 1.0 / 20000.0;
  if (fit > 0.90) return 1.0 / 2000.0;
  if (fit > 0.70) return 1.0 / 500.0;
  return 1.0 / 250.0;
}

// One block of H threads after a sweep: the sweep's fit from its raw terms, the fit / beta history,
// the Section 4.2 rule's state, the features (same definition as cpqr_mlp_features), the network
// (bf16 weights and activations, FP32 accumulation in the order of fwd_layer_kernel) and the
// proposal for the next sweep (arg max of the logits, first maximum).
__global__ void __launch_bounds__(H) mlp_propose_kernel(const __nv_bfloat16* __restrict__ wt,
                                                         const float* __restrict__ params, MlpState* __restrict__ st,
                                                         MlpFitSource src, double beta_used) {
  __shared__ float x0[H], x1[H];
  const int o = threadIdx.x;
  if (o == 0) {
    const double r2 = src.r2 ? src.r2[0] : src.normX2 - 2.0 * src.terms[0] + src.terms[1];
    const double fit = 1.0 - sqrt(fmax(r2, 0.0)) / sqrt(src.normX2);
    for (int j = 0; j < MLP_RING; ++j) st->fit[j] = st->fit[j + 1];
    st->fit[MLP_RING] = fit;
    for (int j = 0; j + 1 < MLP_RING; ++j) st->beta[j] = st->beta[j + 1];
    st->beta[MLP_RING - 1] = beta_used;
    const int n = ++st->n;
    if (!st->activated && n >= 2 && fabs(st->fit[MLP_RING] - st->fit[MLP_RING - 1]) < 0.03) {
      st->rule_beta = beta_band_dev(fit);
      st->activated = 1;
    }
    float f[F];
    for (int i = 0; i < F; ++i) f[i] = 0.f;
    for (int j = 0; j < 8 && n - 1 - j >= 0; ++j) {
      const int k = n - 1 - j;  // sweep index (0-based) j sweeps back
      const double fk = st->fit[MLP_RING - j];
      f[3 * j] = (float)(log10(fmax(1.0 - fk, 1e-12)) / 12.0);
      if (k >= 1) {
        const double d = fk - st->fit[MLP_RING - j - 1];
        const double m = (log10(fmax(fabs(d), 1e-14)) + 14.0) / 14.0;
        f[3 * j + 1] = (float)(d >= 0 ? m : -m);
      }
      f[3 * j + 2] = (float)(log10(st->beta[MLP_RING - 1 - j] + 1e-8) / 8.0);
    }
    f[24] = (float)(log10((double)n + 1.0) / 3.0);
    f[25] = (float)(log10(st->rule_beta + 1e-8) / 8.0);
    f[26] = st->activated ? 1.f : 0.f;
    for (int i = 0; i < F; ++i) {
      st->feat[i] = f[i];
      x0[i] = __bfloat162float(__float2bfloat16_rn(f[i]));
    }
  }
  __syncthreads();
  float* in_act = x0;
  float* out_act = x1;
  for (int l = 0; l < NL; ++l) {
    const int in = layer_in(l), out = layer_out(l);
    const __nv_bfloat16* T = wt + layer_off(l);
    if (o < out) {
      float acc = params[layer_off(l) + in * out + o];
      for (int i = 0; i < in; ++i) acc += in_act[i] * __bfloat162float(T[i * out + o]);
      if (l < NL - 1) {
        acc = acc > 0.f ? acc : 0.f;
        out_act[o] = __bfloat162float(__float2bfloat16_rn(acc));
      } else {
        st->logits[o] = acc;
      }
    }
    __syncthreads();
    float* t = in_act;
    in_act = out_act;
    out_act = t;
  }
  if (o == 0) {
    int best = 0;
    for (int c = 1; c < NC; ++c)
      if (st->logits[c] > st->logits[best]) best = c;
    st->cls = best;
  }
}

}  // namespace

cudaError_t mlp_prepare_weights(const float* params, __nv_bfloat16* wt, cudaStream_t st) {
  prepare_weights_kernel<<<64, 256, 0, st>>>(params, wt);
  return cudaGetLastError();
}

cudaError_t mlp_propose(const __nv_bfloat16* wt, const float* params, MlpState* state, MlpFitSource src,
                        double beta_used, cudaStream_t st) {
  mlp_propose_kernel<<<1, H, 0, st>>>(wt, params, state, src, beta_used);
  return cudaGetLastError();
}

// Workspace (device, floats): bf16 weight copy + activations + gradients of activations.
struct MlpWork {
  __nv_bfloat16* wb;       // NPARAMS bf16
  __nv_bfloat16* act[NL];  // act[0] = input (B x F); act[l] = output of layer l-1 (B x H)
  float* logits;           // B x NC
  float* dz;               // B x H scratch
  float* dz2;              // B x H scratch
};

size_t mlp_work_bytes(int B) {
  size_t s = (size_t)CPQR_MLP_NPARAMS * 2 + 256;
  s += ((size_t)B * F * 2 + 256) + (size_t)(NL - 1) * ((size_t)B * H * 2 + 256);
  s += (size_t)B * NC * 4 + 256 + 2 * ((size_t)B * H * 4 + 256);
  return s;
}

static MlpWork carve(void* work, int B) {
  unsigned char* p = static_cast<unsigned char*>(work);
  auto take = [&](size_t bytes) {
    void* r = p;
    p += (bytes + 255) / 256 * 256;
    return r;
  };
  MlpWork w;
  w.wb = (__nv_bfloat16*)take((size_t)CPQR_MLP_NPARAMS * 2);
  w.act[0] = (__nv_bfloat16*)take((size_t)B * F * 2);
  for (int l = 1; l < NL; ++l) w.act[l] = (__nv_bfloat16*)take((size_t)B * H * 2);
  w.logits = (float*)take((size_t)B * NC * 4);
  w.dz = (float*)take((size_t)B * H * 4);
  w.dz2 = (float*)take((size_t)B * H * 4);
  return w;
}

static cudaError_t forward(const float* params, const float* X, int B, MlpWork& w, cudaStream_t st) {
  to_bf16_kernel<<<(CPQR_MLP_NPARAMS + 255) / 256, 256, 0, st>>>(params, w.wb, CPQR_MLP_NPARAMS);
  to_bf16_kernel<<<(B * F + 255) / 256, 256, 0, st>>>(X, w.act[0], B * F);
  for (int l = 0; l < NL; ++l) {
    const int in = layer_in(l), out = layer_out(l);
    const __nv_bfloat16* Wl = w.wb + layer_off(l);
    const float* bl = params + layer_off(l) + in * out;
    dim3 grid((out + 127) / 128, B);
    const bool last = (l == NL - 1);
    fwd_layer_kernel<<<grid, 128, 0, st>>>(w.act[l], Wl, bl, B, in, out, last ? 0 : 1,
                                           last ? nullptr : w.act[l + 1], last ? w.logits : nullptr);
  }
  return cudaGetLastError();
}

cudaError_t mlp_forward(const float* params, const float* X, int B, float* logits, void* work, cudaStream_t st) {
  MlpWork w = carve(work, B);
  cudaError_t e = forward(params, X, B, w, st);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(logits, w.logits, (size_t)B * NC * 4, cudaMemcpyDeviceToDevice, st);
}

cudaError_t mlp_grad(const float* params, const float* X, const int32_t* y, int B, float* grad, float* loss,
                     void* work, cudaStream_t st) {
  MlpWork w = carve(work, B);
  cudaError_t e = forward(params, X, B, w, st);
  if (e != cudaSuccess) return e;
  softmax_xent_kernel<<<1, 256, 0, st>>>(w.logits, y, B, w.dz, loss);
  // dz holds dZ of the current layer (B x out)
  float* dz = w.dz;
  float* dx = w.dz2;
  for (int l = NL - 1; l >= 0; --l) {
    const int in = layer_in(l), out = layer_out(l);
    const __nv_bfloat16* Wl = w.wb + layer_off(l);
    float* gW = grad + layer_off(l);
    float* gb = gW + in * out;
    bwd_dw_kernel<<<dim3((in + 1 + 127) / 128, out), 128, 0, st>>>(dz, w.act[l], B, in, out, gW, gb);
    if (l > 0) {
      bwd_dx_kernel<<<dim3((in + 127) / 128, B), 128, 0, st>>>(dz, Wl, B, in, out, w.act[l], dx);
      float* t = dz;
      dz = dx;
      dx = t;
    }
  }
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* params, float* m, float* v, const float* grad, float lr, int step, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(CPQR_MLP_NPARAMS + 255) / 256, 256, 0, st>>>(params, m, v, grad, CPQR_MLP_NPARAMS, lr, b1, b2, eps,
                                                              c1, c2);
  return cudaGetLastError();
}

}  // namespace cpqr
