// Training and evaluation kernels of the ghost-rejection network.
//
// The network is trained on the GPU by these kernels (float32): one thread
// per sample runs the forward pass and back-propagates the binary
// cross-entropy of sigmoid(logit) to per-sample deltas; one thread per weight
// then sums its gradient over the batch in sample order (deterministic, no
// floating-point atomics); Adam updates the weights.  Inference for
// evaluation runs either the reconstruction's bfloat16 tensor-core routine or
// a float32 CUDA-core reference.
#include <cuda_runtime.h>

#include <cmath>

#include "velo_internal.cuh"
#include "velo_mlp.cuh"

namespace velo {

namespace {

constexpr int kW1 = 0;                     // W1[32][12]
constexpr int kB1 = kW1 + kHid * kFeat;    // b1[32]
constexpr int kW2 = kB1 + kHid;            // W2[32][32]
constexpr int kB2 = kW2 + kHid * kHid;     // b2[32]
constexpr int kW3 = kB2 + kHid;            // W3[32]
constexpr int kB3 = kW3 + kHid;            // b3
static_assert(kB3 + 1 == VELO_MLP_WEIGHTS, "weight layout");


struct SampleBufs {
  float* h1;    // [n][32]
  float* h2;    // [n][32]
  float* d1;    // [n][32]  dL/da1
  float* d2;    // [n][32]  dL/da2
  float* dz;    // [n]      dL/dz
  float* loss;  // [n]      per-sample loss
};

__global__ void __launch_bounds__(128) k_mlp_samples(const float* __restrict__ x, const float* __restrict__ y,
                                                      uint64_t n, const float* __restrict__ w, SampleBufs B) {
  __shared__ float sw[VELO_MLP_WEIGHTS];
  for (int i = threadIdx.x; i < VELO_MLP_WEIGHTS; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float xi[kFeat], a1[kHid], a2[kHid];
  for (int k = 0; k < kFeat; ++k) xi[k] = x[s * kFeat + k];
  for (int j = 0; j < kHid; ++j) {
    float a = sw[kB1 + j];
    for (int k = 0; k < kFeat; ++k) a += sw[kW1 + j * kFeat + k] * xi[k];
    a1[j] = a;
    B.h1[s * kHid + j] = a > 0.0f ? a : 0.0f;
  }
  for (int j = 0; j < kHid; ++j) {
    float a = sw[kB2 + j];
    for (int k = 0; k < kHid; ++k) a += sw[kW2 + j * kHid + k] * (a1[k] > 0.0f ? a1[k] : 0.0f);
    a2[j] = a;
    B.h2[s * kHid + j] = a > 0.0f ? a : 0.0f;
  }
  float z = sw[kB3];
  for (int j = 0; j < kHid; ++j) z += sw[kW3 + j] * (a2[j] > 0.0f ? a2[j] : 0.0f);
  const float yy = y[s];
  const float inv_n = 1.0f / (float)n;
  B.loss[s] = fmaxf(z, 0.0f) - z * yy + log1pf(expf(-fabsf(z)));
  const float dz = (1.0f / (1.0f + expf(-z)) - yy) * inv_n;
  B.dz[s] = dz;
  float d2[kHid];
  for (int j = 0; j < kHid; ++j) {
    d2[j] = a2[j] > 0.0f ? dz * sw[kW3 + j] : 0.0f;
    B.d2[s * kHid + j] = d2[j];
  }
  for (int k = 0; k < kHid; ++k) {
    float d = 0.0f;
    for (int j = 0; j < kHid; ++j) d += d2[j] * sw[kW2 + j * kHid + k];
    B.d1[s * kHid + k] = a1[k] > 0.0f ? d : 0.0f;
  }
}

// one thread per trainable weight (and one for the loss): sums over samples in order
__global__ void __launch_bounds__(256) k_mlp_grads(const float* __restrict__ x, uint64_t n, SampleBufs B,
                                                    float* grad, float* loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > VELO_MLP_WEIGHTS) return;
  float g = 0.0f;
  if (i == VELO_MLP_WEIGHTS) {
    for (uint64_t s = 0; s < n; ++s) g += B.loss[s];
    *loss = g / (float)n;
    return;
  }
  if (i < kB1) {
    const int j = i / kFeat, k = i % kFeat;
    for (uint64_t s = 0; s < n; ++s) g += B.d1[s * kHid + j] * x[s * kFeat + k];
  } else if (i < kW2) {
    const int j = i - kB1;
    for (uint64_t s = 0; s < n; ++s) g += B.d1[s * kHid + j];
  } else if (i < kB2) {
    const int j = (i - kW2) / kHid, k = (i - kW2) % kHid;
    for (uint64_t s = 0; s < n; ++s) g += B.d2[s * kHid + j] * B.h1[s * kHid + k];
  } else if (i < kW3) {
    const int j = i - kB2;
    for (uint64_t s = 0; s < n; ++s) g += B.d2[s * kHid + j];
  } else if (i < kB3) {
    const int j = i - kW3;
    for (uint64_t s = 0; s < n; ++s) g += B.dz[s] * B.h2[s * kHid + j];
  } else {
    for (uint64_t s = 0; s < n; ++s) g += B.dz[s];
  }
  grad[i] = g;
}

__global__ void k_mlp_adam(float* w, const float* g, float* m, float* v, uint32_t nw, float lr, float b1, float b2,
                           float eps, float c1, float c2) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// bfloat16 tensor-core inference, one warp per 32 candidates
__global__ void __launch_bounds__(256) k_mlp_infer_bf16(const float* __restrict__ f, uint64_t n, const float* blob,
                                                         float* logits) {
  __shared__ MlpWeights W;
  __shared__ MlpTiles T[8];
  mlp_load(blob, W, threadIdx.x, blockDim.x);
  __syncthreads();
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float fi[kFeat];
  for (int k = 0; k < kFeat; ++k) fi[k] = s < n ? f[s * kFeat + k] : 0.0f;
  const float z = mlp_logit_warp(fi, W, T[threadIdx.x >> 5]);
  if (s < n) logits[s] = z;
}

// float32 reference on CUDA cores (normalisation as in the blob, no bf16 rounding)
__global__ void __launch_bounds__(128) k_mlp_infer_f32(const float* __restrict__ f, uint64_t n, const float* blob,
                                                        float* logits) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float* w = blob + 2 * kFeat;
  float xi[kFeat], h1[kHid];
  for (int k = 0; k < kFeat; ++k) xi[k] = (f[s * kFeat + k] - blob[k]) * blob[kFeat + k];
  for (int j = 0; j < kHid; ++j) {
    float a = w[kB1 + j];
    for (int k = 0; k < kFeat; ++k) a += w[kW1 + j * kFeat + k] * xi[k];
    h1[j] = a > 0.0f ? a : 0.0f;
  }
  float z = w[kB3];
  for (int j = 0; j < kHid; ++j) {
    float a = w[kB2 + j];
    for (int k = 0; k < kHid; ++k) a += w[kW2 + j * kHid + k] * h1[k];
    z += w[kW3 + j] * (a > 0.0f ? a : 0.0f);
  }
  logits[s] = z;
}

uint64_t mlp_workspace_bytes(uint64_t n) { return (4 * (uint64_t)kHid + 2) * n * sizeof(float) + 1024; }

}  // namespace

}  // namespace velo

using namespace velo;

extern "C" {

int velo_mlp_infer(const float* features, uint64_t n, const float* mlp, float* logits, int mode, void* stream) {
  if ((n && (!features || !logits)) || !mlp || (mode != 0 && mode != 1)) return VELO_EINVAL;
  if (n == 0) return VELO_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (mode == 0) k_mlp_infer_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(features, n, mlp, logits);
  else k_mlp_infer_f32<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(features, n, mlp, logits);
  return cudaGetLastError() == cudaSuccess ? VELO_OK : VELO_ECUDA;
}

int velo_mlp_workspace_size(uint64_t n, uint64_t* bytes) {
  if (!bytes) return VELO_EINVAL;
  *bytes = mlp_workspace_bytes(n);
  return VELO_OK;
}

int velo_mlp_loss_grad(const float* x, const float* y, uint64_t n, const float* w, float* grad, float* loss,
                       void* workspace, uint64_t workspace_bytes, void* stream) {
  if (n == 0 || !x || !y || !w || !grad || !loss || !workspace) return VELO_EINVAL;
  if (workspace_bytes < mlp_workspace_bytes(n) || (reinterpret_cast<uintptr_t>(workspace) & 15u)) return VELO_ECAPACITY;
  float* base = reinterpret_cast<float*>(workspace);
  SampleBufs B;
  B.h1 = base;
  B.h2 = B.h1 + (uint64_t)kHid * n;
  B.d1 = B.h2 + (uint64_t)kHid * n;
  B.d2 = B.d1 + (uint64_t)kHid * n;
  B.dz = B.d2 + (uint64_t)kHid * n;
  B.loss = B.dz + n;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_mlp_samples<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(x, y, n, w, B);
  k_mlp_grads<<<(VELO_MLP_WEIGHTS + 1 + 255) / 256, 256, 0, s>>>(x, n, B, grad, loss);
  return cudaGetLastError() == cudaSuccess ? VELO_OK : VELO_ECUDA;
}

int velo_mlp_adam_step(float* w, const float* grad, float* m, float* v, uint32_t n_weights, float lr, float beta1,
                       float beta2, float eps, uint32_t step, void* stream) {
  if (!w || !grad || !m || !v || step == 0 || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f))
    return VELO_EINVAL;
  const float c1 = 1.0f - (float)std::pow((double)beta1, (double)step);
  const float c2 = 1.0f - (float)std::pow((double)beta2, (double)step);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_mlp_adam<<<(n_weights + 255) / 256, 256, 0, s>>>(w, grad, m, v, n_weights, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? VELO_OK : VELO_ECUDA;
}

}  // extern "C"
