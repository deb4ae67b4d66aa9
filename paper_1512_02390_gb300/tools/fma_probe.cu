// FMA throughput probe for the ALU rooflines of this library: each thread runs
// 8 independent FMA chains; no memory traffic except one in-bounds store per thread.
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_chain(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <typename T>
double run(int blocks, int threads, int iters) {
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  fma_chain<T><<<blocks, threads>>>(out, 16, (T)0.999, (T)0.001);
  cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    fma_chain<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
  }
  cudaFree(out);
  double flops = 2.0 * 8 * (double)iters * blocks * threads;
  return flops / (best * 1e-3) / 1e12;
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  printf("device %s SMs %d L2 %d MB smem/block optin %zu KB\n", p.name, p.multiProcessorCount, p.l2CacheSize >> 20, p.sharedMemPerBlockOptin >> 10);
  int sms = p.multiProcessorCount;
  printf("fp64 TFLOP/s %.3f\n", run<double>(sms * 8, 256, 2048));
  printf("fp32 TFLOP/s %.3f\n", run<float>(sms * 8, 256, 8192));
  cudaError_t e = cudaGetLastError(); printf("status %s\n", cudaGetErrorString(e));
  return e != cudaSuccess;
}
