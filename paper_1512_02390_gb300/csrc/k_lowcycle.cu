// The lower part of the V-cycle (Alg. 3) in ONE persistent cooperative kernel:
// for every level l = top .. 1 (p_l <= 8) one Schwarz step from u_l = 0
// (Alg. 2: the mma.sync sweep writes the corrections E_l; the residual kernel
// body assembles u_l from them and forms r_l = f_l - A_l u_l), the
// restriction f_{l-1} = I_l^T r_l, the exact coarse solve u_0 = A_0^+ f_0
// (global fast diagonalisation, Sec. 3.2), then the prolongations
// u_l += I_l u_{l-1} back up to level top.  The phases are the same tile and
// subdomain bodies the one-kernel-per-step path launches (level_ops.cuh),
// separated by grid barriers instead of kernel boundaries: the low levels are
// small and their launches cost more than their work.
//
// The grid barrier is bounded: a CTA that waits longer than about one second
// sets *err and goes on (the host reports SEM_TIMEOUT); every CTA of the grid is
// resident (cooperative launch).
#include "kernels.h"
#include "level_ops.cuh"

namespace sem {

namespace {

constexpr int kLowThreads = 256;
constexpr int kLowWarps = kLowThreads / 32;
constexpr long long kBarrierCycles = 1LL << 31;

// bar[0]: arrivals, bar[1]: generation
__device__ __forceinline__ void grid_barrier(unsigned* bar, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > kBarrierCycles) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// one Schwarz step from zero, the residual and the restriction on level
// l = log2(P)
template <int MODE, int P>
__device__ __forceinline__ void level_down(const LowCycle& c, unsigned char* smem) {
  constexpr int l = ilog2_c(P);
  const LowLevel& L = c.lev[l];
  const int nsub = L.x.n * L.y.n;
  const int warp = threadIdx.x >> 5;
  sweep_mma_warp<float, MODE, 16>(L.x, L.y, L.f, L.E, nullptr, nsub, blockIdx.x * kLowWarps + warp,
                                  gridDim.x * kLowWarps,
                                  reinterpret_cast<float*>(smem) + warp * MmaSmem<16>::PER_WARP);
  grid_barrier(c.bar, c.err);
  // u_l = sum_s R_s^T E_s and r_l = f_l - A_l u_l, tile by tile
  constexpr int TE = Tile<P>::TE;
  const int ntx = (L.x.n + TE - 1) / TE, nty = (L.y.n + TE - 1) / TE;
  for (int t = blockIdx.x; t < ntx * nty; t += gridDim.x) {
    const int by = t / ntx, bx = t - by * ntx;
    apply_tile<float, float, P>(L.x, L.y, nullptr, L.f, L.r, 0, nullptr, L.E, L.u, PcgFuse(), bx, by, ntx, nty, smem);
    __syncthreads();
  }
  grid_barrier(c.bar, c.err);
  // f_{l-1} = I_l^T r_l
  const LowLevel& C = c.lev[l - 1];
  constexpr int TT_E = TT<P>::TE;
  const int ctx = (C.x.n + TT_E - 1) / TT_E, cty = (C.y.n + TT_E - 1) / TT_E;
  for (int t = blockIdx.x; t < ctx * cty; t += gridDim.x) {
    const int by = t / ctx, bx = t - by * ctx;
    restrict_tile<float, P>(L.x, L.y, C.x, C.y, L.J, L.r, C.f, bx, by, smem);
    __syncthreads();
  }
  grid_barrier(c.bar, c.err);
}

// u_l += I_l u_{l-1} on level l = log2(P)
template <int P>
__device__ __forceinline__ void level_up(const LowCycle& c, unsigned char* smem) {
  constexpr int l = ilog2_c(P);
  const LowLevel& L = c.lev[l];
  const LowLevel& C = c.lev[l - 1];
  constexpr int TE = TT<P>::TE;
  const int ntx = (L.x.n + TE - 1) / TE, nty = (L.y.n + TE - 1) / TE;
  for (int t = blockIdx.x; t < ntx * nty; t += gridDim.x) {
    const int by = t / ntx, bx = t - by * ntx;
    prolong_tile<float, float, P>(L.x, L.y, C.x, C.y, L.J, C.u, L.u, L.u, bx, by, smem);
    __syncthreads();
  }
  grid_barrier(c.bar, c.err);
}

// The coarse solve U = S_y [(S_y^T F S_x) ./ (lambda_y + lambda_x^T)] S_x^T in
// FP32 (at most 64 x 64 unknowns per problem), row by row: phase 1 writes the
// scaled spectral coefficients W of problem k, row a, to the scratch; phase 2
// forms solution row j from all of W.  Right side and solution are projected to
// zero mean when the coarse operator is singular (periodic).
__device__ __forceinline__ void coarse_solve(const LowCycle& c, unsigned char* smem) {
  const CoarseView& cv = c.coarse;
  const LowLevel& Z = c.lev[0];
  const int nux = cv.nux, nuy = cv.nuy, t = threadIdx.x;
  float* wa = reinterpret_cast<float*>(smem);  // 64
  float* wb = wa + 64;                          // 64
  double* sred = reinterpret_cast<double*>(wb + 64);
  const int nb = cv.batch > 0 ? cv.batch : 1;
  for (int row = blockIdx.x; row < nb * nuy; row += gridDim.x) {
    const int k = row / nuy, a = row - k * nuy;
    const float* F = Z.f + (long)(cv.firsty + k * cv.block_rows) * cv.Nx + cv.firstx;
    float shift = 0.f;
    if (cv.periodic) {
      double acc = 0.0;
      for (int idx = t; idx < nux * nuy; idx += blockDim.x) acc += F[(long)(idx / nux) * cv.Nx + idx % nux];
      shift = (float)(block_sum(acc, sred) / ((double)nux * nuy));
    }
    if (t < nux) {  // wa[i] = sum_j S_y[j][a] (F[j][i] - shift)
      float s = 0.f;
      for (int j = 0; j < nuy; ++j) s = fmaf(cv.Sy32[j * nuy + a], F[(long)j * cv.Nx + t] - shift, s);
      wa[t] = s;
    }
    __syncthreads();
    if (t < nux) {  // W[a][b] = sum_i wa[i] S_x[i][b] / (lambda_y[a] + lambda_x[b])
      float s = 0.f;
      for (int i = 0; i < nux; ++i) s = fmaf(wa[i], cv.Sx32[i * nux + t], s);
      c.cw[((long)k * 64 + a) * 64 + t] = (cv.periodic && a == 0 && t == 0) ? 0.f : s / (cv.ly32[a] + cv.lx32[t]);
    }
    __syncthreads();
  }
  grid_barrier(c.bar, c.err);
  for (int row = blockIdx.x; row < nb * nuy; row += gridDim.x) {
    const int k = row / nuy, j = row - k * nuy;
    const float* W = c.cw + (long)k * 64 * 64;
    float mean_u = 0.f;
    if (cv.periodic) {  // mean(U) = c_y^T W c_x / N
      double acc = 0.0;
      for (int idx = t; idx < nux * nuy; idx += blockDim.x) {
        const int a = idx / nux, b = idx - a * nux;
        acc += (double)cv.cy32[a] * W[a * 64 + b] * cv.cx32[b];
      }
      mean_u = (float)(block_sum(acc, sred) / ((double)nux * nuy));
    }
    if (t < nux) {  // wb[b] = sum_a S_y[j][a] W[a][b]
      float s = 0.f;
      for (int a = 0; a < nuy; ++a) s = fmaf(cv.Sy32[j * nuy + a], W[a * 64 + t], s);
      wb[t] = s;
    }
    __syncthreads();
    if (t < nux) {  // U[j][i] = sum_b wb[b] S_x[i][b]
      float s = 0.f;
      for (int b = 0; b < nux; ++b) s = fmaf(wb[b], cv.Sx32[t * nux + b], s);
      Z.u[(long)(cv.firsty + k * cv.block_rows + j) * cv.Nx + cv.firstx + t] = s - mean_u;
    }
    __syncthreads();
  }
  grid_barrier(c.bar, c.err);
}

template <int MODE, int P>
__device__ __forceinline__ void down_from(const LowCycle& c, unsigned char* smem) {
  level_down<MODE, P>(c, smem);
  if constexpr (P > 2) down_from<MODE, P / 2>(c, smem);
}

template <int P>
__device__ __forceinline__ void up_to(const LowCycle& c, unsigned char* smem) {
  if constexpr (P > 2) up_to<P / 2>(c, smem);
  level_up<P>(c, smem);
}

// PT: order of the highest level handled (level c.top)
template <int MODE, int PT>
__global__ void __launch_bounds__(kLowThreads) k_low_cycle(LowCycle c) {
  extern __shared__ __align__(16) unsigned char smem_low[];
  down_from<MODE, PT>(c, smem_low);
  coarse_solve(c, smem_low);
  up_to<PT>(c, smem_low);
}

template <int MODE, int PT>
constexpr size_t low_smem() {
  size_t s = sizeof(float) * MmaSmem<16>::PER_WARP * kLowWarps;
  s = s > apply_smem<float, PT>() ? s : apply_smem<float, PT>();
  s = s > restrict_smem<float, PT>() ? s : restrict_smem<float, PT>();
  s = s > prolong_smem<float, PT>() ? s : prolong_smem<float, PT>();
  return s;
}

template <int MODE, int PT>
cudaError_t low_launch(const LowCycle& c, int* grid_out, cudaStream_t s) {
  const size_t sm = low_smem<MODE, PT>();
  cudaError_t e = allow_smem(k_low_cycle<MODE, PT>, sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_low_cycle<MODE, PT>, kLowThreads, sm)) !=
      cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = sms * std::min(per_sm, 2);
  if (grid_out) *grid_out = grid;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kLowThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_low_cycle<MODE, PT>, c);
}

}  // namespace

cudaError_t launch_low_cycle(const LowCycle& c, int mode, int top_p, int* grid, cudaStream_t s) {
  if (c.top < 1 || c.top > 3 || (1 << c.top) != top_p || c.coarse.nux > 64 || c.coarse.nuy > 64)
    return cudaErrorInvalidValue;
  if (mode == 1) {
    switch (top_p) {
      case 2: return low_launch<1, 2>(c, grid, s);
      case 4: return low_launch<1, 4>(c, grid, s);
      case 8: return low_launch<1, 8>(c, grid, s);
    }
  } else if (mode == 2) {
    switch (top_p) {
      case 2: return low_launch<2, 2>(c, grid, s);
      case 4: return low_launch<2, 4>(c, grid, s);
      case 8: return low_launch<2, 8>(c, grid, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace sem
