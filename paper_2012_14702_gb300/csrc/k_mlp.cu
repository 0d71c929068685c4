// The learned-damping model: a 6 -> 64 -> 64 -> 1 MLP (tanh, tanh, output
// alpha = 2 sigmoid(y)) with FP16 parameters and FP32 arithmetic, and its
// training kernels (mean-squared-error gradient, Adam step).
//
// Parameter layout (FP16, packed, row-major): W1[6][64], b1[64], W2[64][64],
// b2[64], W3[64][1], b3[1]  (4673 values).  Samples are rows of X [B x 6].
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

constexpr int NI = kMlpInputs, NH = kMlpHidden;
constexpr int O_W1 = 0, O_B1 = O_W1 + NI * NH, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
              O_W3 = O_B2 + NH, O_B3 = O_W3 + NH, NP = O_B3 + 1;
static_assert(NP == kMlpParams, "parameter count");
constexpr int GB = 64;  // samples per gradient block

__device__ __forceinline__ float sigmoidf_(float y) { return 1.f / (1.f + __expf(-y)); }

__device__ __forceinline__ void load_params(const __half* __restrict__ p, float* w) {
  for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = __half2float(p[i]);
}

// h1, h2 (registers) and y for one sample
__device__ __forceinline__ float mlp_row(const float* w, const float* x, float* h1, float* h2) {
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    float a = w[O_B1 + j];
#pragma unroll
    for (int f = 0; f < NI; ++f) a = fmaf(x[f], w[O_W1 + f * NH + j], a);
    h1[j] = tanhf(a);
  }
#pragma unroll 4
  for (int j = 0; j < NH; ++j) {
    float a = w[O_B2 + j];
#pragma unroll
    for (int i = 0; i < NH; ++i) a = fmaf(h1[i], w[O_W2 + i * NH + j], a);
    h2[j] = tanhf(a);
  }
  float y = w[O_B3];
#pragma unroll
  for (int j = 0; j < NH; ++j) y = fmaf(h2[j], w[O_W3 + j], y);
  return y;
}

__global__ void __launch_bounds__(128)
    k_mlp_forward(const __half* __restrict__ p, const float* __restrict__ X, int B,
                  float* __restrict__ alpha) {
  __shared__ float w[NP];
  load_params(p, w);
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float x[NI], h1[NH], h2[NH];
#pragma unroll
  for (int f = 0; f < NI; ++f) x[f] = X[(int64_t)b * NI + f];
  alpha[b] = 2.f * sigmoidf_(mlp_row(w, x, h1, h2));
}

// grad += d/dparams of mean_b (alpha_b - target_b)^2 over all B samples (the
// 1/B is applied here); loss += the mean.
__global__ void __launch_bounds__(GB)
    k_mlp_grad(const __half* __restrict__ p, const float* __restrict__ X,
               const float* __restrict__ target, int B, float* __restrict__ grad,
               double* __restrict__ loss) {
  extern __shared__ float sm[];
  float* w = sm;                    // NP
  float* H1 = w + NP;               // GB x (NH + 1)
  float* DA2 = H1 + GB * (NH + 1);  // GB x (NH + 1)
  float* DA1 = DA2 + GB * (NH + 1); // GB x (NH + 1)
  float* XS = DA1 + GB * (NH + 1);  // GB x NI
  float* DY = XS + GB * NI;         // GB
  load_params(p, w);
  __syncthreads();
  const int t = threadIdx.x;
  const int b = blockIdx.x * GB + t;
  const bool live = b < B;
  float x[NI], h1[NH], h2[NH];
#pragma unroll
  for (int f = 0; f < NI; ++f) x[f] = live ? X[(int64_t)b * NI + f] : 0.f;
  const float y = mlp_row(w, x, h1, h2);
  const float s = sigmoidf_(y);
  const float r = live ? 2.f * s - target[b] : 0.f;
  const float dy = live ? (2.f / (float)B) * r * 2.f * s * (1.f - s) : 0.f;
  // da2 = dy W3 (1 - h2^2); da1 = (W2 da2) (1 - h1^2)
  float da2[NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) da2[j] = dy * w[O_W3 + j] * (1.f - h2[j] * h2[j]);
#pragma unroll 4
  for (int i = 0; i < NH; ++i) {
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < NH; ++j) a = fmaf(w[O_W2 + i * NH + j], da2[j], a);
    DA1[t * (NH + 1) + i] = a * (1.f - h1[i] * h1[i]);
  }
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    H1[t * (NH + 1) + j] = h1[j];
    DA2[t * (NH + 1) + j] = da2[j];
  }
#pragma unroll
  for (int f = 0; f < NI; ++f) XS[t * NI + f] = x[f];
  DY[t] = dy;
  // the W3 / b3 gradients need h2: reduce them now
  __shared__ float red[NH + 1];
  for (int i = t; i < NH + 1; i += GB) red[i] = 0.f;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NH; ++j) atomicAdd(&red[j], dy * h2[j]);
  atomicAdd(&red[NH], dy);
  const float lv = r * r / (float)B;
  __shared__ float lred;
  if (t == 0) lred = 0.f;
  __syncthreads();
  atomicAdd(&lred, lv);
  __syncthreads();
  if (t < NH) atomicAdd(&grad[O_W3 + t], red[t]);
  if (t == 0) {
    atomicAdd(&grad[O_B3], red[NH]);
    atomicAdd(loss, (double)lred);
  }
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
    for (int j = 0; j < NH; ++j) atomicAdd(&grad[O_W2 + i * NH + j], acc[j]);
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
    atomicAdd(&grad[O_B2 + t], a2);
    atomicAdd(&grad[O_B1 + t], a1);
#pragma unroll
    for (int f = 0; f < NI; ++f) atomicAdd(&grad[O_W1 + f * NH + t], wf[f]);
  }
}

// Adam (Kingma & Ba) on FP32 master parameters; writes the FP16 copy and
// clears the gradient.
__global__ void k_mlp_adam(float* __restrict__ master, __half* __restrict__ p,
                           float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
                           float lr, float b1, float b2, float eps, int step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
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

constexpr size_t grad_smem() {
  return sizeof(float) * (NP + 3 * GB * (NH + 1) + GB * NI + GB);
}

}  // namespace

cudaError_t launch_mlp_forward(const void* params, const float* X, int B, float* alpha,
                               cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_mlp_forward<<<(B + 127) / 128, 128, 0, s>>>(static_cast<const __half*>(params), X, B, alpha);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const void* params, const float* X, const float* target, int B,
                            float* grad, double* loss, cudaStream_t s) {
  static int configured = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured != dev) {
    e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)grad_smem());
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  if (B <= 0) return cudaSuccess;
  k_mlp_grad<<<(B + GB - 1) / GB, GB, grad_smem(), s>>>(static_cast<const __half*>(params), X,
                                                       target, B, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* master, void* params, float* grad, float* m, float* v,
                            float lr, float b1, float b2, float eps, int step, cudaStream_t s) {
  k_mlp_adam<<<(NP + 255) / 256, 256, 0, s>>>(master, static_cast<__half*>(params), grad, m, v,
                                              lr, b1, b2, eps, step);
  return cudaGetLastError();
}

}  // namespace ipt
