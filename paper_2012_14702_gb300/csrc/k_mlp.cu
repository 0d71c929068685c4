// The learned-acceleration models: NI -> 64 -> 64 -> NO MLPs (tanh, tanh) with
// FP16 parameters and FP32 arithmetic, and their training kernels
// (mean-squared-error gradient, Adam step).
//   damping model  NI = 6, NO = 1: alpha = 2 sigmoid(y0)
//   mixing model   NI = 7, NO = 2: alpha = 2 sigmoid(y0), gamma = 2 tanh(y1)
//
// Parameter layout (FP16, packed, row-major): W1[NI][64], b1[64], W2[64][64],
// b2[64], W3[64][NO], b3[NO].  Samples are rows of X [B x NI]; outputs and
// targets rows of [B x NO].
//
// Forward: one thread per sample, the parameters in shared memory as FP32.
// Gradient: a block of 64 samples recomputes the forward pass, keeps h1 and
// the back-propagated da2 of its samples in shared memory, forms its share
// of every weight gradient as a small product over the samples (dW2 = h1^T
// da2 ...) and adds it to the FP32 gradient with one atomic per parameter.
#include <cuda_fp16.h>

#include "ipt_internal.cuh"

namespace ipt {

namespace {

constexpr int NH = kMlpHidden;
constexpr int GB = 64;  // samples per gradient block

template <int NI, int NO>
struct Mlp {
  static constexpr int O_W1 = 0, O_B1 = O_W1 + NI * NH, O_W2 = O_B1 + NH,
                       O_B2 = O_W2 + NH * NH, O_W3 = O_B2 + NH, O_B3 = O_W3 + NH * NO,
                       NP = O_B3 + NO;
};
static_assert(Mlp<kMlpInputs, 1>::NP == kMlpParams, "damping parameter count");
static_assert(Mlp<kMixInputs, 2>::NP == kMixParams, "mixing parameter count");

__device__ __forceinline__ float sigmoidf_(float y) { return 1.f / (1.f + __expf(-y)); }

template <int NP>
__device__ __forceinline__ void load_params(const __half* __restrict__ p, float* w) {
  for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = __half2float(p[i]);
}

// h1, h2 (registers) and y[NO] for one sample
template <int NI, int NO>
__device__ __forceinline__ void mlp_row(const float* w, const float* x, float* h1, float* h2,
                                        float* y) {
  using L = Mlp<NI, NO>;
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    float a = w[L::O_B1 + j];
#pragma unroll
    for (int f = 0; f < NI; ++f) a = fmaf(x[f], w[L::O_W1 + f * NH + j], a);
    h1[j] = tanhf(a);
  }
#pragma unroll 4
  for (int j = 0; j < NH; ++j) {
    float a = w[L::O_B2 + j];
#pragma unroll
    for (int i = 0; i < NH; ++i) a = fmaf(h1[i], w[L::O_W2 + i * NH + j], a);
    h2[j] = tanhf(a);
  }
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    float a = w[L::O_B3 + o];
#pragma unroll
    for (int j = 0; j < NH; ++j) a = fmaf(h2[j], w[L::O_W3 + j * NO + o], a);
    y[o] = a;
  }
}

// The outputs from y: alpha = 2 sigmoid(y0); gamma = 2 tanh(y1)
__device__ __forceinline__ float model_output(int o, float y) {
  return o == 0 ? 2.f * sigmoidf_(y) : 2.f * tanhf(y);
}
// d output / d y
__device__ __forceinline__ float model_output_slope(int o, float y) {
  if (o == 0) {
    const float s = sigmoidf_(y);
    return 2.f * s * (1.f - s);
  }
  const float t = tanhf(y);
  return 2.f * (1.f - t * t);
}

template <int NI, int NO>
__global__ void __launch_bounds__(128)
    k_mlp_forward(const __half* __restrict__ p, const float* __restrict__ X, int B,
                  float* __restrict__ out) {
  __shared__ float w[Mlp<NI, NO>::NP];
  load_params<Mlp<NI, NO>::NP>(p, w);
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float x[NI], h1[NH], h2[NH], y[NO];
#pragma unroll
  for (int f = 0; f < NI; ++f) x[f] = X[(int64_t)b * NI + f];
  mlp_row<NI, NO>(w, x, h1, h2, y);
#pragma unroll
  for (int o = 0; o < NO; ++o) out[(int64_t)b * NO + o] = model_output(o, y[o]);
}

// grad += d/dparams of mean_b sum_o (out_bo - target_bo)^2 over all B samples
// (the 1/B is applied here); loss += the mean.
template <int NI, int NO>
__global__ void __launch_bounds__(GB)
    k_mlp_grad(const __half* __restrict__ p, const float* __restrict__ X,
               const float* __restrict__ target, int B, float* __restrict__ grad,
               double* __restrict__ loss) {
  using L = Mlp<NI, NO>;
  extern __shared__ float sm[];
  float* w = sm;                    // NP
  float* H1 = w + L::NP;            // GB x (NH + 1)
  float* DA2 = H1 + GB * (NH + 1);  // GB x (NH + 1)
  float* DA1 = DA2 + GB * (NH + 1); // GB x (NH + 1)
  float* XS = DA1 + GB * (NH + 1);  // GB x NI
  load_params<L::NP>(p, w);
  __syncthreads();
  const int t = threadIdx.x;
  const int b = blockIdx.x * GB + t;
  const bool live = b < B;
  float x[NI], h1[NH], h2[NH], y[NO], dy[NO];
#pragma unroll
  for (int f = 0; f < NI; ++f) x[f] = live ? X[(int64_t)b * NI + f] : 0.f;
  mlp_row<NI, NO>(w, x, h1, h2, y);
  float lv = 0.f;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    const float r = live ? model_output(o, y[o]) - target[(int64_t)b * NO + o] : 0.f;
    dy[o] = live ? (2.f / (float)B) * r * model_output_slope(o, y[o]) : 0.f;
    lv += r * r / (float)B;
  }
  // da2 = (W3 dy) (1 - h2^2); da1 = (W2 da2) (1 - h1^2)
  float da2[NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    float a = 0.f;
#pragma unroll
    for (int o = 0; o < NO; ++o) a = fmaf(dy[o], w[L::O_W3 + j * NO + o], a);
    da2[j] = a * (1.f - h2[j] * h2[j]);
  }
#pragma unroll 4
  for (int i = 0; i < NH; ++i) {
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < NH; ++j) a = fmaf(w[L::O_W2 + i * NH + j], da2[j], a);
    DA1[t * (NH + 1) + i] = a * (1.f - h1[i] * h1[i]);
  }
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    H1[t * (NH + 1) + j] = h1[j];
    DA2[t * (NH + 1) + j] = da2[j];
  }
#pragma unroll
  for (int f = 0; f < NI; ++f) XS[t * NI + f] = x[f];
  // the W3 / b3 gradients need h2: reduce them now
  __shared__ float red[NH * NO + NO];
  for (int i = t; i < NH * NO + NO; i += GB) red[i] = 0.f;
  __shared__ float lred;
  if (t == 0) lred = 0.f;
  __syncthreads();
#pragma unroll
  for (int o = 0; o < NO; ++o) {
#pragma unroll
    for (int j = 0; j < NH; ++j) atomicAdd(&red[j * NO + o], dy[o] * h2[j]);
    atomicAdd(&red[NH * NO + o], dy[o]);
  }
  atomicAdd(&lred, lv);
  __syncthreads();
  for (int i = t; i < NH * NO; i += GB) atomicAdd(&grad[L::O_W3 + i], red[i]);
  if (t < NO) atomicAdd(&grad[L::O_B3 + t], red[NH * NO + t]);
  if (t == 0) atomicAdd(loss, (double)lred);
  // dW2[i][j] = sum_b h1[b][i] da2[b][j]; thread t owns row i = t, all j
  for (int i = t; i < NH; i += GB) {
    float acc[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) acc[j] = 0.f;
    for (int bb = 0; bb < GB; ++bb) {
      const float hv = H1[bb * (NH + 1) + i];
#pragma unroll
      for (int j = 0; j < NH; ++j) acc[j] = fmaf(hv, DA2[bb * (NH + 1) + j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < NH; ++j) atomicAdd(&grad[L::O_W2 + i * NH + j], acc[j]);
  }
  // db2[j] = sum_b da2[b][j]; db1[j] = sum_b da1[b][j]; dW1[f][j] = sum_b x[b][f] da1[b][j]
  if (t < NH) {
    float a2 = 0.f, a1 = 0.f, wf[NI];
#pragma unroll
    for (int f = 0; f < NI; ++f) wf[f] = 0.f;
    for (int bb = 0; bb < GB; ++bb) {
      a2 += DA2[bb * (NH + 1) + t];
      const float d1 = DA1[bb * (NH + 1) + t];
      a1 += d1;
#pragma unroll
      for (int f = 0; f < NI; ++f) wf[f] = fmaf(XS[bb * NI + f], d1, wf[f]);
    }
    atomicAdd(&grad[L::O_B2 + t], a2);
    atomicAdd(&grad[L::O_B1 + t], a1);
#pragma unroll
    for (int f = 0; f < NI; ++f) atomicAdd(&grad[L::O_W1 + f * NH + t], wf[f]);
  }
}

// Adam (Kingma & Ba) on FP32 master parameters; writes the FP16 copy and
// clears the gradient.
__global__ void k_mlp_adam(float* __restrict__ master, __half* __restrict__ p,
                           float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
                           int np, float lr, float b1, float b2, float eps, int step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)step));
  const float vh = vi / (1.f - powf(b2, (float)step));
  const float x = master[i] - lr * mh / (sqrtf(vh) + eps);
  master[i] = x;
  p[i] = __float2half_rn(x);
  grad[i] = 0.f;
}

template <int NI, int NO>
constexpr size_t grad_smem() {
  return sizeof(float) * (Mlp<NI, NO>::NP + 3 * GB * (NH + 1) + GB * NI);
}

template <int NI, int NO>
cudaError_t forward_impl(const void* params, const float* X, int B, float* out, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_mlp_forward<NI, NO><<<(B + 127) / 128, 128, 0, s>>>(static_cast<const __half*>(params), X,
                                                        B, out);
  return cudaGetLastError();
}

template <int NI, int NO>
cudaError_t grad_impl(const void* params, const float* X, const float* target, int B,
                      float* grad, double* loss, cudaStream_t s) {
  static int configured = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured != dev) {
    e = cudaFuncSetAttribute(k_mlp_grad<NI, NO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)grad_smem<NI, NO>());
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  if (B <= 0) return cudaSuccess;
  k_mlp_grad<NI, NO><<<(B + GB - 1) / GB, GB, grad_smem<NI, NO>(), s>>>(
      static_cast<const __half*>(params), X, target, B, grad, loss);
  return cudaGetLastError();
}

cudaError_t adam_impl(int np, float* master, void* params, float* grad, float* m, float* v,
                      float lr, float b1, float b2, float eps, int step, cudaStream_t s) {
  k_mlp_adam<<<(np + 255) / 256, 256, 0, s>>>(master, static_cast<__half*>(params), grad, m, v,
                                              np, lr, b1, b2, eps, step);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mlp_forward(const void* params, const float* X, int B, float* alpha,
                               cudaStream_t s) {
  return forward_impl<kMlpInputs, 1>(params, X, B, alpha, s);
}

cudaError_t launch_mlp_grad(const void* params, const float* X, const float* target, int B,
                            float* grad, double* loss, cudaStream_t s) {
  return grad_impl<kMlpInputs, 1>(params, X, target, B, grad, loss, s);
}

cudaError_t launch_mlp_adam(float* master, void* params, float* grad, float* m, float* v,
                            float lr, float b1, float b2, float eps, int step, cudaStream_t s) {
  return adam_impl(kMlpParams, master, params, grad, m, v, lr, b1, b2, eps, step, s);
}

cudaError_t launch_mix_forward(const void* params, const float* X, int B, float* out,
                               cudaStream_t s) {
  return forward_impl<kMixInputs, 2>(params, X, B, out, s);
}

cudaError_t launch_mix_grad(const void* params, const float* X, const float* target, int B,
                            float* grad, double* loss, cudaStream_t s) {
  return grad_impl<kMixInputs, 2>(params, X, target, B, grad, loss, s);
}

cudaError_t launch_mix_adam(float* master, void* params, float* grad, float* m, float* v,
                            float lr, float b1, float b2, float eps, int step, cudaStream_t s) {
  return adam_impl(kMixParams, master, params, grad, m, v, lr, b1, b2, eps, step, s);
}

}  // namespace ipt
