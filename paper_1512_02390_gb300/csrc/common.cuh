// Device-side views shared by the kernels of the Schwarz/multigrid solver.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>
#include <utility>

namespace sem {

// One direction of one multigrid level, as the kernels see it.
template <typename T>
struct DirView {
  int p;          // polynomial order of the level
  int n;          // elements
  int N;          // global nodes (periodic: n p; Dirichlet: n p + 1)
  int periodic;   // 1 periodic, 0 Dirichlet walls
  int n_o, m;     // overlap layers, window size p + 1 + 2 n_o
  int segN;       // > 0: Dirichlet wall every segN nodes (independent problems stacked)
  const T* Le;    // n x (p+1)^2 element stiffness
  const T* Mg;    // N assembled mass diagonal
  const int* tab; // n subdomain table ids
  const T* S;     // tables x m x m eigenvectors (padded)
  const T* lam;   // tables x m eigenvalues (padded with 1)
  const T* w;     // tables x m weights (padded with 0)
};

// wrap/validate a global node index of a direction; returns -1 if the node
// does not exist or is a Dirichlet wall node (value 0 there).  segN > 0 adds
// internal walls every segN nodes (problems stacked along the direction).
__device__ __forceinline__ int node_or_wall(int g, int N, int periodic, int segN = 0) {
  if (periodic) {
    g %= N;
    return g < 0 ? g + N : g;
  }
  if (!(g > 0 && g < N - 1)) return -1;
  return (segN > 0 && g % segN == 0) ? -1 : g;
}

// is node g of a direction a Dirichlet wall node?
__device__ __forceinline__ bool wall_node(int g, int N, int periodic, int segN = 0) {
  if (periodic) return false;
  return g == 0 || g == N - 1 || (segN > 0 && g % segN == 0);
}

constexpr int kRedThreads = 256;

// Deterministic block sum of one double per thread (fixed tree order).
__device__ __forceinline__ double block_sum(double v, double* sbuf) {
  // fixed-order tree: butterfly within each warp (lane 0's result is used),
  // then warp 0 over the warp totals; blockDim.x a multiple of 32, sbuf >= 33
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sbuf[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double r = lane < nw ? sbuf[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) sbuf[32] = r;
  }
  __syncthreads();
  const double r = sbuf[32];
  __syncthreads();
  return r;
}

// The same sum with its FP64 adds in one warp, for kernels bound by the
// narrow FP64 pipe (a butterfly in every warp issues nw times the adds): lane
// l of warp 0 adds the values of threads l, l + 32, l + 64, ... in that
// order, then a butterfly over the 32 lane sums.  sbuf: blockDim.x doubles
// (a multiple of 32).
__device__ __forceinline__ double block_sum_w0(double v, double* sbuf) {
  __shared__ double s_total;
  sbuf[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = sbuf[threadIdx.x];
    for (int i = threadIdx.x + 32; i < (int)blockDim.x; i += 32) r += sbuf[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (threadIdx.x == 0) s_total = r;
  }
  __syncthreads();
  return s_total;
}

// Sum of n partials written by other CTAs of the same launch (read through
// L2, fixed order): used by the last CTA of a launch.
__device__ __forceinline__ double sum_partials_cg(const double* part, int n, double* sbuf) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(part + i);
  return block_sum_w0(v, sbuf);
}

// Sum of n partials in a fixed order, identical in every block that calls it.
__device__ __forceinline__ double sum_partials(const double* part, int n, double* sbuf) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  return block_sum_w0(v, sbuf);
}

}  // namespace sem

namespace sem {

// floor(a / b) for b > 0 and any sign of a
__device__ __forceinline__ int floordiv(int a, int b) {
  int q = a / b;
  return (q * b > a) ? q - 1 : q;
}

// one-time opt-in to more than 48 KB of dynamic shared memory
template <typename K>
inline cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace sem

namespace sem {

// Sum of the weighted Schwarz corrections at node (gj, gi): the R_s^T sum of
// Eq. (correction:global) over the (at most 3 x 3) windows that hold the node,
// in a fixed order.  E: element-blocked m x m corrections.
template <typename T>
__device__ __forceinline__ T window_sum(const DirView<T>& dx, const DirView<T>& dy, const T* __restrict__ E, int gj,
                                        int gi) {
  const int p = dx.p, no = dx.n_o, m = dx.m, mm = m * m;
  const int ey_lo = floordiv(gj - no - 1, p), ey_hi = floordiv(gj + no, p);
  const int ex_lo = floordiv(gi - no - 1, p), ex_hi = floordiv(gi + no, p);
  T s = T(0);
  for (int eyu = ey_lo; eyu <= ey_hi; ++eyu) {
    int ey = eyu;
    if (dy.periodic) ey = ((ey % dy.n) + dy.n) % dy.n;
    else if (ey < 0 || ey >= dy.n) continue;
    const int a = gj - eyu * p + no;
    for (int exu = ex_lo; exu <= ex_hi; ++exu) {
      int ex = exu;
      if (dx.periodic) ex = ((ex % dx.n) + dx.n) % dx.n;
      else if (ex < 0 || ex >= dx.n) continue;
      const int b = gi - exu * p + no;
      s += E[(long)(ey * dx.n + ex) * mm + a * m + b];
    }
  }
  return s;
}

// window_sum for a compile-time order P: node g = e P + j (0 <= j < P) lies in
// the windows of elements e - 1 (when j <= n_o), e and e + 1 (when
// j >= P - n_o), at window index (e - e') P + j + n_o; the same windows in
// the same (ascending y, then x) order as window_sum, so the same sum.
template <int P, typename T>
__device__ __forceinline__ T window_sum_p(const DirView<T>& dx, const DirView<T>& dy, const T* __restrict__ E, int gj,
                                          int gi) {
  const int no = dx.n_o, m = P + 1 + 2 * no, mm = m * m;
  int ex[3], bx[3], nxc = 0, ey[3], by[3], nyc = 0;
  {
    const int e = gi / P, j = gi - e * P;
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      if ((d < 0 && j > no) || (d > 0 && j < P - no)) continue;
      int ee = e + d;
      if (dx.periodic) ee = ee < 0 ? ee + dx.n : (ee >= dx.n ? ee - dx.n : ee);
      else if (ee < 0 || ee >= dx.n) continue;
      ex[nxc] = ee;
      bx[nxc] = j - d * P + no;
      ++nxc;
    }
  }
  {
    const int e = gj / P, j = gj - e * P;
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      if ((d < 0 && j > no) || (d > 0 && j < P - no)) continue;
      int ee = e + d;
      if (dy.periodic) ee = ee < 0 ? ee + dy.n : (ee >= dy.n ? ee - dy.n : ee);
      else if (ee < 0 || ee >= dy.n) continue;
      ey[nyc] = ee;
      by[nyc] = j - d * P + no;
      ++nyc;
    }
  }
  T s = T(0);
  for (int iy = 0; iy < nyc; ++iy) {
    const T* Er = E + (long)ey[iy] * dx.n * mm + by[iy] * m;
    for (int ix = 0; ix < nxc; ++ix) s += Er[(long)ex[ix] * mm + bx[ix]];
  }
  return s;
}

}  // namespace sem

namespace sem {

// Programmatic dependent launch (sm_90+).  Every kernel of the solver opens
// with pdl_enter(): wait until the kernel before it in the stream has completed
// and its writes are visible (returns at once when the launch carried no
// programmatic dependency).  launch_pdl() enqueues with the programmatic-
// serialization attribute, so the launch of the next kernel is prepared while
// this one finishes; no kernel reads anything before its predecessor has
// completed.  No kernel triggers its dependents early: measured on the 64 x 64,
// p = 16 solve, an early trigger let waiting CTAs of the next kernel hold SM
// resources (2.71 ms per solve against 2.56 ms without it, 2.58 ms with the
// attribute off).
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace sem

namespace sem {

// value of type TF as type T (the hardware conversion: measured faster on the
// mixed-precision V-cycle than a conversion by integer operations on the bits)
template <typename T, typename TF>
__device__ __forceinline__ T convert_to(TF v) {
  return static_cast<T>(v);
}

}  // namespace sem
