// Learned weights: the FP32 MLP (4 -> 64 -> 64 -> 2, ReLU) that maps features
// of an interface line to its weight parameters (s, kt), with forward,
// backward and Adam kernels (training on the GPU).
//
// Parameter layout (4610 floats): W1 (64x4), b1 (64), W2 (64x64), b2 (64),
// W3 (2x64), b3 (2), row-major.  Loss L = (1/2N) sum (o - t)^2.
// One CTA handles a tile of 64 samples with the whole parameter vector in
// shared memory; the backward kernel writes one partial gradient per CTA and
// a second kernel sums them in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "sem_schwarz.h"

namespace sem {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int NI = 4, NH = 64, NO = 2, TS = 64;  // inputs, hidden, outputs, samples per CTA
constexpr int OW1 = 0, OB1 = OW1 + NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NO * NH, NP = OB3 + NO;
static_assert(NP == SEM_MLP_PARAMS, "parameter count");

struct Tile {
  float w[NP];
  float x[TS][NI];
  float z1[TS][NH + 1];
  float z2[TS][NH + 1];
  float o[TS][NO];
};

// forward pass of the CTA's samples into shared memory (pre-activations kept)
__device__ void forward_tile(Tile& t, const float* __restrict__ params, const float* __restrict__ X, int n, int s0) {
  for (int i = threadIdx.x; i < NP; i += blockDim.x) t.w[i] = params[i];
  for (int i = threadIdx.x; i < TS * NI; i += blockDim.x) {
    const int s = i / NI, k = i - s * NI;
    t.x[s][k] = (s0 + s < n) ? X[(long)(s0 + s) * NI + k] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TS * NH; i += blockDim.x) {
    const int s = i / NH, u = i - s * NH;
    float a = t.w[OB1 + u];
#pragma unroll
    for (int k = 0; k < NI; ++k) a += t.w[OW1 + u * NI + k] * t.x[s][k];
    t.z1[s][u] = a;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TS * NH; i += blockDim.x) {
    const int s = i / NH, u = i - s * NH;
    float a = t.w[OB2 + u];
#pragma unroll 8
    for (int k = 0; k < NH; ++k) a += t.w[OW2 + u * NH + k] * fmaxf(t.z1[s][k], 0.f);
    t.z2[s][u] = a;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TS * NO; i += blockDim.x) {
    const int s = i / NO, j = i - s * NO;
    float a = t.w[OB3 + j];
#pragma unroll 8
    for (int k = 0; k < NH; ++k) a += t.w[OW3 + j * NH + k] * fmaxf(t.z2[s][k], 0.f);
    t.o[s][j] = a;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_mlp_forward(const float* __restrict__ params, const float* __restrict__ X,
                                                     int n, float* __restrict__ Y, int transform) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tile& t = *reinterpret_cast<Tile*>(smem_raw);
  const int s0 = blockIdx.x * TS;
  forward_tile(t, params, X, n, s0);
  for (int i = threadIdx.x; i < TS * NO; i += blockDim.x) {
    const int s = i / NO, j = i - s * NO;
    if (s0 + s >= n) continue;
    float v = t.o[s][j];
    if (transform) {
      const float sg = 1.f / (1.f + expf(-v));
      v = j == 0 ? 0.25f + 0.75f * sg : 1.f + 6.f * sg;
    }
    Y[(long)(s0 + s) * NO + j] = v;
  }
}

// per-CTA partial gradient (NP floats) and partial loss (1 float)
__global__ void __launch_bounds__(256) k_mlp_backward(const float* __restrict__ params, const float* __restrict__ X,
                                                      const float* __restrict__ T, int n, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tile& t = *reinterpret_cast<Tile*>(smem_raw);
  __shared__ float d[TS][NO];
  __shared__ float dh[TS][NH + 1];
  __shared__ float red[256];
  const int s0 = blockIdx.x * TS;
  forward_tile(t, params, X, n, s0);
  float* g = part + (long)blockIdx.x * (NP + 1);
  const float inv_n = 1.f / (float)n;
  float lacc = 0.f;
  for (int i = threadIdx.x; i < TS * NO; i += blockDim.x) {
    const int s = i / NO, j = i - s * NO;
    float v = 0.f;
    if (s0 + s < n) {
      const float e = t.o[s][j] - T[(long)(s0 + s) * NO + j];
      v = e * inv_n;
      lacc += 0.5f * e * e * inv_n;
    }
    d[s][j] = v;
  }
  red[threadIdx.x] = lacc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) g[NP] = red[0];
  // layer 3
  for (int i = threadIdx.x; i < NO * NH + NO; i += blockDim.x) {
    float a = 0.f;
    if (i < NO * NH) {
      const int j = i / NH, k = i - j * NH;
      for (int s = 0; s < TS; ++s) a += d[s][j] * fmaxf(t.z2[s][k], 0.f);
      g[OW3 + i] = a;
    } else {
      const int j = i - NO * NH;
      for (int s = 0; s < TS; ++s) a += d[s][j];
      g[OB3 + j] = a;
    }
  }
  for (int i = threadIdx.x; i < TS * NH; i += blockDim.x) {
    const int s = i / NH, k = i - s * NH;
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < NO; ++j) a += d[s][j] * t.w[OW3 + j * NH + k];
    dh[s][k] = t.z2[s][k] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // layer 2
  for (int i = threadIdx.x; i < NH * NH + NH; i += blockDim.x) {
    float a = 0.f;
    if (i < NH * NH) {
      const int u = i / NH, k = i - u * NH;
      for (int s = 0; s < TS; ++s) a += dh[s][u] * fmaxf(t.z1[s][k], 0.f);
      g[OW2 + i] = a;
    } else {
      const int u = i - NH * NH;
      for (int s = 0; s < TS; ++s) a += dh[s][u];
      g[OB2 + u] = a;
    }
  }
  // dh1 (into z2's storage: z2 is no longer needed)
  for (int i = threadIdx.x; i < TS * NH; i += blockDim.x) {
    const int s = i / NH, k = i - s * NH;
    float a = 0.f;
    for (int u = 0; u < NH; ++u) a += dh[s][u] * t.w[OW2 + u * NH + k];
    t.z2[s][k] = t.z1[s][k] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // layer 1
  for (int i = threadIdx.x; i < NH * NI + NH; i += blockDim.x) {
    float a = 0.f;
    if (i < NH * NI) {
      const int u = i / NI, k = i - u * NI;
      for (int s = 0; s < TS; ++s) a += t.z2[s][u] * t.x[s][k];
      g[OW1 + i] = a;
    } else {
      const int u = i - NH * NI;
      for (int s = 0; s < TS; ++s) a += t.z2[s][u];
      g[OB1 + u] = a;
    }
  }
}

// grad[i] = sum over CTAs of the partials, fixed order; loss likewise
__global__ void __launch_bounds__(256) k_mlp_reduce(const float* __restrict__ part, int nblk, float* __restrict__ grad,
                                                    float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > NP) return;
  float a = 0.f;
  for (int b = 0; b < nblk; ++b) a += part[(long)b * (NP + 1) + i];
  if (i < NP) grad[i] = a;
  else if (loss) *loss = a;
}

// Adam (Kingma & Ba 2015) with bias correction at step t
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ params, const float* __restrict__ grad,
                                              float* __restrict__ m, float* __restrict__ v, float lr, int t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gi = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)t)), vh = vi / (1.f - powf(b2, (float)t));
  params[i] -= lr * mh / (sqrtf(vh) + eps);
}

int fail(int code, const std::string& m) {
  sem::set_last_error(m);
  return code;
}

int nblocks(int n) { return (n + TS - 1) / TS; }

cudaError_t allow() {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Tile));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Tile));
  return e;
}

}  // namespace

extern "C" {

int64_t sem_mlp_workspace_bytes(int32_t n) {
  if (n < 1) return 0;
  return (int64_t)sizeof(float) * ((int64_t)nblocks(n) * (NP + 1) + NP);
}

int sem_mlp_forward(const float* params, const float* X, int32_t n, float* Y, int32_t transform, void* stream) {
  if (!params || !X || !Y || n < 1) return fail(SEM_BAD_ARG, "sem_mlp_forward: invalid argument");
  cudaError_t e = allow();
  if (e == cudaSuccess) {
    k_mlp_forward<<<nblocks(n), 256, sizeof(Tile), static_cast<cudaStream_t>(stream)>>>(params, X, n, Y, transform);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? SEM_OK : fail(SEM_CUDA_ERROR, cudaGetErrorString(e));
}

int sem_mlp_loss_grad(const float* params, const float* X, const float* T, int32_t n, float* grad, float* loss,
                      void* workspace, void* stream) {
  if (!params || !X || !T || !grad || !workspace || n < 1) return fail(SEM_BAD_ARG, "sem_mlp_loss_grad: invalid argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = static_cast<float*>(workspace);
  cudaError_t e = allow();
  if (e == cudaSuccess) {
    k_mlp_backward<<<nblocks(n), 256, sizeof(Tile), s>>>(params, X, T, n, part);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_mlp_reduce<<<(NP + 1 + 255) / 256, 256, 0, s>>>(part, nblocks(n), grad, loss);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? SEM_OK : fail(SEM_CUDA_ERROR, cudaGetErrorString(e));
}

int sem_mlp_train(float* params, float* adam_m, float* adam_v, const float* X, const float* T, int32_t n,
                  int32_t steps, float lr, int32_t step0, float* loss_hist, void* workspace, void* stream) {
  if (!params || !adam_m || !adam_v || !X || !T || !workspace || n < 1 || steps < 0 || step0 < 0 || !(lr > 0.f))
    return fail(SEM_BAD_ARG, "sem_mlp_train: invalid argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = static_cast<float*>(workspace);
  float* grad = part + (size_t)nblocks(n) * (NP + 1);
  cudaError_t e = allow();
  for (int k = 0; k < steps && e == cudaSuccess; ++k) {
    k_mlp_backward<<<nblocks(n), 256, sizeof(Tile), s>>>(params, X, T, n, part);
    k_mlp_reduce<<<(NP + 1 + 255) / 256, 256, 0, s>>>(part, nblocks(n), grad, loss_hist ? loss_hist + k : nullptr);
    k_adam<<<(NP + 255) / 256, 256, 0, s>>>(params, grad, adam_m, adam_v, lr, step0 + k + 1);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? SEM_OK : fail(SEM_CUDA_ERROR, cudaGetErrorString(e));
}

}  // extern "C"
