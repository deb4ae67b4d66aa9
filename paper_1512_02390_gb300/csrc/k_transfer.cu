// Grid transfer between multigrid levels p_l = 2^l (Sec. 3.2, Alg. 3) and
// the coarse solution u_0 = A_0^+ f_0.
//
// I_l = P_y (x) P_x with the global 1D embedded interpolation P:
//   P[i, I] = J[i - e p_f, I - e p_c] for the fine node i of element e (the
// interface node counted once, as local node 0 of the element to its right),
// J[i', k] = phi_k^{(p_c)}(xi_i'^{(p_f)}).  Prolongation evaluates
// u_f = P_y U_c P_x^T; restriction is its exact transpose F_c = P_y^T R_f P_x.
// Both are separable and done as two 1D contractions through shared memory,
// one CTA per tile of elements, every output node written once.
//
// Coarse solve: A_0 = M_y (x) L_x + L_y (x) M_x at p = 1 is inverted by global
// fast diagonalisation over the unknowns, U = S_y [(S_y^T F S_x) ./ (lam_y +
// lam_x^T)] S_x^T, FP64.  For a periodic (singular) A_0 the right side is
// projected to zero mean, the (0, 0) eigen-pair is dropped and the result is
// made orthogonal to the constants: the Moore-Penrose solution A_0^+ f_0.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "kernels.h"
#include "level_ops.cuh"

namespace sem {

namespace {

// The finest level's transfer launches have one CTA per 2 x 2 elements (1024
// at 64 x 64, p = 16): at 32 registers 8 CTAs fit an SM and they run in one
// wave instead of two.  FP64 and p = 32 restrictions would spill at 32.
template <typename T, int PF>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && PF <= 16) ? 8 : 1) k_restrict(DirView<T> fx, DirView<T> fy, DirView<T> cx, DirView<T> cy,
                                                  const T* __restrict__ J, const T* __restrict__ rf,
                                                  T* __restrict__ fc) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  restrict_tile<T, PF>(fx, fy, cx, cy, J, rf, fc, blockIdx.x, blockIdx.y, smem_raw);
}

template <typename T, typename TOut, int PF>
__global__ void __launch_bounds__(256, 8) k_prolong(DirView<T> fx, DirView<T> fy, DirView<T> cx, DirView<T> cy,
                                                 const T* __restrict__ J, const T* __restrict__ uc,
                                                 const T* in, TOut* out) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  prolong_tile<T, TOut, PF>(fx, fy, cx, cy, J, uc, in, out, blockIdx.x, blockIdx.y, smem_raw);
}

// the finest prolongation of the V-cycle writing z, with z.q, z.r and beta
template <typename T, int PF>
__global__ void __launch_bounds__(256, 8) k_prolong_dot(DirView<T> fx, DirView<T> fy, DirView<T> cx, DirView<T> cy,
                                                     const T* __restrict__ J, const T* __restrict__ uc,
                                                     const T* in, double* out, PcgDot dot) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  prolong_tile<T, double, PF, true>(fx, fy, cx, cy, J, uc, in, out, blockIdx.x, blockIdx.y, smem_raw, &dot);
}

// the up-leg of the V-cycle in one launch (prolong_chain_tile)
template <typename T, int PF, bool DOT>
__global__ void __launch_bounds__(kChainThreads, 8) k_prolong_chain(ProlongChain<T> c, DirView<T> fx, DirView<T> fy,
                                                                 const T* __restrict__ J, const T* in, double* out,
                                                                 PcgDot dot) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  prolong_chain_tile<T, double, PF, DOT>(c.x, c.y, c.u, c.J, fx, fy, J, in, out, blockIdx.x, blockIdx.y, smem_raw,
                                         &dot);
}

// Coarse solve as four small FP64 products over the unknowns (F: nuy x nux):
//   T1 = S_y^T (F - mu),  T2 = (T1 S_x) ./ (lam_y + lam_x^T),  T3 = S_y T2,
//   U  = T3 S_x^T - mean(U)
// (mu, the mean and the dropped (0,0) pair only for the periodic, singular
// A_0).  One generic kernel: a CTA computes an 8 x 8 output tile with the
// reduction dimension split over 4 thread groups (256 threads), so ~64 CTAs
// share the FP64 work of a 63^3 product instead of one CTA per row.
enum CoarseStep { kStep1 = 0, kStep2 = 1, kStep3 = 2, kStep4 = 3 };

template <typename T>
__global__ void __launch_bounds__(256) k_coarse_gemm(CoarseView c, int step, const T* __restrict__ f0,
                                                     T* __restrict__ u0) {
  pdl_enter();
  constexpr int TM = 8, TK = 4;
  __shared__ double sred[kRedThreads];
  __shared__ double part[TK][TM][TM + 1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nux = c.nux, nuy = c.nuy;
  // stacked problems: block z has its own right side rows and scratch
  const int fy0 = c.firsty + blockIdx.z * c.block_rows;
  c.T1 += (long)blockIdx.z * nux * nuy;
  c.T2 += (long)blockIdx.z * nux * nuy;
  // steps 1 and 3 contract over y (nuy), steps 2 and 4 over x (nux)
  const int K = (step == kStep1 || step == kStep3) ? nuy : nux;
  double* sA = reinterpret_cast<double*>(smem_raw);  // TM x K
  double* sB = sA + TM * K;                           // K x TM
  const int rows = nuy, cols = nux;
  const int r0 = blockIdx.y * TM, c0 = blockIdx.x * TM;
  const int t = threadIdx.x, kg = t / (TM * TM), rr = (t / TM) % TM, cc = t % TM;
  double shift = 0.0;
  if (c.periodic && (step == kStep1 || step == kStep4)) {
    double acc = 0.0;
    if (step == kStep1) {
      for (int idx = t; idx < nux * nuy; idx += blockDim.x) {
        const int j = idx / nux, i = idx - j * nux;
        acc += (double)f0[(long)(fy0 + j) * c.Nx + c.firstx + i];
      }
    } else {  // mean(U) = c_y^T T2 c_x / N (T2 is intact: step 3 wrote T1)
      for (int idx = t; idx < nux * nuy; idx += blockDim.x) {
        const int a = idx / nux, b = idx - a * nux;
        acc += c.cy[a] * c.T2[idx] * c.cx[b];
      }
    }
    shift = block_sum(acc, sred) / ((double)nux * nuy);
  }
  // stage the operand panels (coalesced along the contiguous index)
  for (int idx = t; idx < TM * K; idx += blockDim.x) {
    int r, k;
    double a = 0.0;
    if (step == kStep1) {  // a(row, k) = S_y[k][row]: contiguous in row
      k = idx / TM;
      r = idx - k * TM;
      if (r0 + r < rows) a = c.Sy[k * nuy + r0 + r];
    } else {                 // rows of T1 / S_y: contiguous in k
      r = idx / K;
      k = idx - r * K;
      if (r0 + r < rows) a = (step == kStep3) ? c.Sy[(r0 + r) * nuy + k] : c.T1[(long)(r0 + r) * nux + k];
    }
    sA[r * K + k] = a;
  }
  for (int idx = t; idx < TM * K; idx += blockDim.x) {
    int k, q;
    double b = 0.0;
    if (step == kStep4) {  // b(k, col) = S_x[col][k]: contiguous in k
      q = idx / K;
      k = idx - q * K;
      if (c0 + q < cols) b = c.Sx[(c0 + q) * nux + k];
    } else {                 // rows of F / S_x / T2: contiguous in col
      k = idx / TM;
      q = idx - k * TM;
      if (c0 + q < cols) {
        if (step == kStep1) b = (double)f0[(long)(fy0 + k) * c.Nx + c.firstx + c0 + q] - shift;
        else if (step == kStep2) b = c.Sx[k * nux + c0 + q];
        else b = c.T2[(long)k * nux + c0 + q];
      }
    }
    sB[k * TM + q] = b;
  }
  __syncthreads();
  double s = 0.0;
  for (int k = kg; k < K; k += TK) s += sA[rr * K + k] * sB[k * TM + cc];
  part[kg][rr][cc] = s;
  __syncthreads();
  const int row = r0 + rr, col = c0 + cc;
  if (kg == 0 && row < rows && col < cols) {
    double v = part[0][rr][cc] + part[1][rr][cc] + part[2][rr][cc] + part[3][rr][cc];
    const long o = (long)row * nux + col;
    switch (step) {
      case kStep1: c.T1[o] = v; break;
      case kStep2: c.T2[o] = (c.periodic && row == 0 && col == 0) ? 0.0 : v / (c.ly[row] + c.lx[col]); break;
      case kStep3: c.T1[o] = v; break;  // S_y T2 reuses the T1 buffer
      default: u0[(long)(fy0 + row) * c.Nx + c.firstx + col] = T(v - shift);
    }
  }
}

// u0 = Binv f0: one warp per unknown row, FP64 accumulation, coalesced reads
// of the dense inverse (variable diffusivity, Dirichlet walls)
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_dense(CoarseView c, const double* __restrict__ Binv,
                                                      const T* __restrict__ f0, T* __restrict__ u0) {
  pdl_enter();
  const int n = c.nux * c.nuy;
  const int fy0 = c.firsty + blockIdx.y * c.block_rows;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = Binv + (long)warp * n;
  double s = 0.0;
  for (int k = lane; k < n; k += 32) {
    const int j = k / c.nux, i = k - j * c.nux;
    s += row[k] * (double)f0[(long)(fy0 + j) * c.Nx + c.firstx + i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const int j = warp / c.nux, i = warp - j * c.nux;
    u0[(long)(fy0 + j) * c.Nx + c.firstx + i] = T(s);
  }
}

template <typename T, int PF>
cudaError_t restrict_p(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx, const DirView<T>& cy,
                       const T* J, const T* rf, T* fc, cudaStream_t s) {
  using Q = TT<PF>;
  const size_t sm = restrict_smem<T, PF>();
  cudaError_t e = allow_smem(k_restrict<T, PF>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((cx.n + Q::TE - 1) / Q::TE, (cy.n + Q::TE - 1) / Q::TE);
  {
    const cudaError_t e_ = launch_pdl(k_restrict<T, PF>, dim3(grid), dim3(256), sm, s, fx, fy, cx, cy, J, rf, fc);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

template <typename T, typename TOut, int PF>
cudaError_t prolong_p(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx, const DirView<T>& cy,
                      const T* J, const T* uc, const T* in, TOut* out, cudaStream_t s) {
  using Q = TT<PF>;
  const size_t sm = prolong_smem<T, PF>();
  cudaError_t e = allow_smem(k_prolong<T, TOut, PF>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((fx.n + Q::TE - 1) / Q::TE, (fy.n + Q::TE - 1) / Q::TE);
  {
    const cudaError_t e_ = launch_pdl(k_prolong<T, TOut, PF>, dim3(grid), dim3(256), sm, s, fx, fy, cx, cy, J, uc, in, out);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

template <typename T, int PF>
cudaError_t prolong_dot_p(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx, const DirView<T>& cy,
                          const T* J, const T* uc, const T* in, double* out, const PcgDot& dot, cudaStream_t s) {
  using Q = TT<PF>;
  const size_t sm = prolong_smem<T, PF>();
  cudaError_t e = allow_smem(k_prolong_dot<T, PF>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((fx.n + Q::TE - 1) / Q::TE, (fy.n + Q::TE - 1) / Q::TE);
  if (2L * grid.x * grid.y > kMaxPartials) return cudaErrorInvalidConfiguration;
  {
    const cudaError_t e_ = launch_pdl(k_prolong_dot<T, PF>, dim3(grid), dim3(256), sm, s, fx, fy, cx, cy, J, uc, in, out, dot);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

template <typename T, int PF, bool DOT>
cudaError_t prolong_chain_p(const ProlongChain<T>& c, const DirView<T>& fx, const DirView<T>& fy, const T* J,
                            const T* in, double* out, const PcgDot& dot, cudaStream_t s) {
  using G = ChainGeo<PF>;
  const size_t sm = prolong_chain_smem<T, PF>();
  cudaError_t e = allow_smem(k_prolong_chain<T, PF, DOT>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((fx.n + G::TE - 1) / G::TE, (fy.n + G::TE - 1) / G::TE);
  if (DOT && 2L * grid.x * grid.y > kMaxPartials) return cudaErrorInvalidConfiguration;
  e = launch_pdl(k_prolong_chain<T, PF, DOT>, grid, dim3(kChainThreads), sm, s, c, fx, fy, J, in, out, dot);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename T, int PF>
cudaError_t prolong_chain_d(const ProlongChain<T>& c, const DirView<T>& fx, const DirView<T>& fy, const T* J,
                            const T* in, double* out, const PcgDot* dot, cudaStream_t s) {
  if (dot) return prolong_chain_p<T, PF, true>(c, fx, fy, J, in, out, *dot, s);
  return prolong_chain_p<T, PF, false>(c, fx, fy, J, in, out, PcgDot{}, s);
}

template <int PF>
long prolong_ctas_p(int nx, int ny) {
  constexpr int TE = TT<PF>::TE;
  return (long)((nx + TE - 1) / TE) * ((ny + TE - 1) / TE);
}

}  // namespace

long prolong_ctas(int p, int nx, int ny) {
  switch (p) {
    case 2: return prolong_ctas_p<2>(nx, ny);
    case 4: return prolong_ctas_p<4>(nx, ny);
    case 8: return prolong_ctas_p<8>(nx, ny);
    case 16: return prolong_ctas_p<16>(nx, ny);
    case 32: return prolong_ctas_p<32>(nx, ny);
    default: return -1;
  }
}

template <typename T>
cudaError_t launch_prolong_dot(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx,
                               const DirView<T>& cy, const T* J, const T* uc, const T* in, double* out,
                               const PcgDot& dot, cudaStream_t s) {
  switch (fx.p) {
    case 2: return prolong_dot_p<T, 2>(fx, fy, cx, cy, J, uc, in, out, dot, s);
    case 4: return prolong_dot_p<T, 4>(fx, fy, cx, cy, J, uc, in, out, dot, s);
    case 8: return prolong_dot_p<T, 8>(fx, fy, cx, cy, J, uc, in, out, dot, s);
    case 16: return prolong_dot_p<T, 16>(fx, fy, cx, cy, J, uc, in, out, dot, s);
    case 32: return prolong_dot_p<T, 32>(fx, fy, cx, cy, J, uc, in, out, dot, s);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_prolong_dot<float>(const DirView<float>&, const DirView<float>&, const DirView<float>&,
                                               const DirView<float>&, const float*, const float*, const float*,
                                               double*, const PcgDot&, cudaStream_t);
template cudaError_t launch_prolong_dot<double>(const DirView<double>&, const DirView<double>&,
                                                const DirView<double>&, const DirView<double>&, const double*,
                                                const double*, const double*, double*, const PcgDot&, cudaStream_t);

template <typename T>
cudaError_t launch_prolong_chain(const ProlongChain<T>& c, const DirView<T>& fx, const DirView<T>& fy, const T* J,
                                 const T* in, double* out, const PcgDot* dot, cudaStream_t s) {
  switch (fx.p) {
    case 4: return prolong_chain_d<T, 4>(c, fx, fy, J, in, out, dot, s);
    case 8: return prolong_chain_d<T, 8>(c, fx, fy, J, in, out, dot, s);
    case 16: return prolong_chain_d<T, 16>(c, fx, fy, J, in, out, dot, s);
    case 32: return prolong_chain_d<T, 32>(c, fx, fy, J, in, out, dot, s);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_prolong_chain<float>(const ProlongChain<float>&, const DirView<float>&,
                                                 const DirView<float>&, const float*, const float*, double*,
                                                 const PcgDot*, cudaStream_t);
template cudaError_t launch_prolong_chain<double>(const ProlongChain<double>&, const DirView<double>&,
                                                  const DirView<double>&, const double*, const double*, double*,
                                                  const PcgDot*, cudaStream_t);

template <typename T>
cudaError_t launch_restrict(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx, const DirView<T>& cy,
                            const T* J, const T* rf, T* fc, cudaStream_t s) {
  switch (fx.p) {
    case 2: return restrict_p<T, 2>(fx, fy, cx, cy, J, rf, fc, s);
    case 4: return restrict_p<T, 4>(fx, fy, cx, cy, J, rf, fc, s);
    case 8: return restrict_p<T, 8>(fx, fy, cx, cy, J, rf, fc, s);
    case 16: return restrict_p<T, 16>(fx, fy, cx, cy, J, rf, fc, s);
    case 32: return restrict_p<T, 32>(fx, fy, cx, cy, J, rf, fc, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, typename TOut>
cudaError_t launch_prolong(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx, const DirView<T>& cy,
                           const T* J, const T* uc, const T* in, TOut* out, cudaStream_t s) {
  switch (fx.p) {
    case 2: return prolong_p<T, TOut, 2>(fx, fy, cx, cy, J, uc, in, out, s);
    case 4: return prolong_p<T, TOut, 4>(fx, fy, cx, cy, J, uc, in, out, s);
    case 8: return prolong_p<T, TOut, 8>(fx, fy, cx, cy, J, uc, in, out, s);
    case 16: return prolong_p<T, TOut, 16>(fx, fy, cx, cy, J, uc, in, out, s);
    case 32: return prolong_p<T, TOut, 32>(fx, fy, cx, cy, J, uc, in, out, s);
    default: return cudaErrorInvalidValue;
  }
}

// The same exact coarse solve, u_0 = A_0^+ f_0 by the global fast
// diagonalisation U = S_y [(S_y^T F S_x) ./ (lambda_y + lambda_x^T)] S_x^T,
// in FP32 for coarse grids of at most 64 x 64 unknowns (the mixed-precision
// V-cycle) by ONE thread-block cluster of 8 CTAs per problem: CTA c owns rows
// 8c .. 8c+7 of every product.  The first two products and the scaling need
// only the CTA's own rows; the third contracts over all rows, which each CTA
// reads from its peers' shared memory (distributed shared memory) after a
// cluster barrier.
constexpr int kC32 = 64, kC32P = 65, kCl = 8, kClRows = kC32 / kCl;  // tile, pitch, cluster, rows per CTA
constexpr int kClThreads = kClRows * 32;  // threads per CTA: one warp per owned row
// Tile passes per thread.  The tile loads (global, and peer shared memory in
// the gather) are all issued before the first store, one round trip each.
constexpr int kClPass = kC32 * kC32 / kClThreads;

__global__ void __launch_bounds__(kClThreads) k_coarse_fdm32(CoarseView c, const float* __restrict__ f0,
                                                     float* __restrict__ u0) {
  pdl_enter();
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) unsigned char smem_c32[];
  float* Sx = reinterpret_cast<float*>(smem_c32);  // 64 x 65
  float* Sy = Sx + kC32 * kC32P;                    // 64 x 65
  float* F = Sy + kC32 * kC32P;                     // 64 x 65: the right side, then the gathered W1
  float* Wa = F + kC32 * kC32P;                     // 8 x 65: own rows of S_y^T F, then of S_y W1
  float* Wb = Wa + kClRows * kC32P;                 // 8 x 65: own rows of the scaled W1 (read by peers)
  __shared__ float lx[kC32], ly[kC32], cx[kC32], cy[kC32];
  __shared__ double sred[kRedThreads];
  const int nux = c.nux, nuy = c.nuy, t = threadIdx.x;
  const int r0 = rank * kClRows;
  const int fy0 = c.firsty + (blockIdx.x / kCl) * c.block_rows;
  {
    float vx[kClPass], vy[kClPass], vf[kClPass];
#pragma unroll
    for (int j = 0; j < kClPass; ++j) {
      const int idx = t + j * kClThreads, a = idx / kC32, b = idx - a * kC32;
      vx[j] = (a < nux && b < nux) ? c.Sx32[a * nux + b] : 0.f;
      vy[j] = (a < nuy && b < nuy) ? c.Sy32[a * nuy + b] : 0.f;
      vf[j] = (a < nuy && b < nux) ? f0[(long)(fy0 + a) * c.Nx + c.firstx + b] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < kClPass; ++j) {
      const int idx = t + j * kClThreads, a = idx / kC32, b = idx - a * kC32;
      Sx[a * kC32P + b] = vx[j];
      Sy[a * kC32P + b] = vy[j];
      F[a * kC32P + b] = vf[j];
    }
  }
  for (int i = t; i < kC32; i += blockDim.x) {
    lx[i] = i < nux ? c.lx32[i] : 1.f;
    ly[i] = i < nuy ? c.ly32[i] : 1.f;
    cx[i] = (c.periodic && i < nux) ? c.cx32[i] : 0.f;
    cy[i] = (c.periodic && i < nuy) ? c.cy32[i] : 0.f;
  }
  __syncthreads();
  float shift = 0.f;
  if (c.periodic) {  // right side projected to zero mean (every CTA computes it)
    double acc = 0.0;
    for (int idx = t; idx < nux * nuy; idx += blockDim.x) acc += F[(idx / nux) * kC32P + idx % nux];
    shift = (float)(block_sum(acc, sred) / ((double)nux * nuy));
  }
  // thread t: own row rr = t / 32, columns q = t % 32 and t % 32 + 32
  const int rr = t >> 5, q0 = t & 31, row = r0 + rr;
  {  // Wa = rows of S_y^T (F - shift)
    float a0 = 0.f, a1 = 0.f;
    for (int j = 0; j < nuy; ++j) {
      const float s = Sy[j * kC32P + row];
      a0 = fmaf(s, F[j * kC32P + q0] - shift, a0);
      a1 = fmaf(s, F[j * kC32P + q0 + 32] - shift, a1);
    }
    Wa[rr * kC32P + q0] = a0;
    Wa[rr * kC32P + q0 + 32] = a1;
  }
  __syncthreads();
  {  // Wb = rows of (Wa S_x) ./ (lambda_y + lambda_x^T); the null pair dropped when periodic
    float a0 = 0.f, a1 = 0.f;
    for (int i = 0; i < nux; ++i) {
      const float w = Wa[rr * kC32P + i];
      a0 = fmaf(w, Sx[i * kC32P + q0], a0);
      a1 = fmaf(w, Sx[i * kC32P + q0 + 32], a1);
    }
    Wb[rr * kC32P + q0] = (c.periodic && row == 0 && q0 == 0) ? 0.f : a0 / (ly[row] + lx[q0]);
    Wb[rr * kC32P + q0 + 32] = a1 / (ly[row] + lx[q0 + 32]);
  }
  cluster.sync();
  // gather every CTA's rows of W1 (over the right side, no longer needed)
  {
    float vw[kClPass];
#pragma unroll
    for (int j = 0; j < kClPass; ++j) {
      const int idx = t + j * kClThreads, a = idx / kC32, b = idx - a * kC32;
      vw[j] = cluster.map_shared_rank(Wb, a / kClRows)[(a % kClRows) * kC32P + b];
    }
#pragma unroll
    for (int j = 0; j < kClPass; ++j) {
      const int idx = t + j * kClThreads, a = idx / kC32, b = idx - a * kC32;
      F[a * kC32P + b] = vw[j];
    }
  }
  cluster.sync();  // peers are done reading this CTA's rows
  float mean_u = 0.f;
  if (c.periodic) {  // mean(U) = c_y^T W1 c_x / N: the solution is returned with zero mean
    double acc = 0.0;
    for (int idx = t; idx < nux * nuy; idx += blockDim.x) {
      const int a = idx / nux, b = idx - a * nux;
      acc += (double)cy[a] * F[a * kC32P + b] * cx[b];
    }
    mean_u = (float)(block_sum(acc, sred) / ((double)nux * nuy));
  }
  {  // Wa = rows of S_y W1
    float a0 = 0.f, a1 = 0.f;
    for (int a = 0; a < nuy; ++a) {
      const float s = Sy[row * kC32P + a];
      a0 = fmaf(s, F[a * kC32P + q0], a0);
      a1 = fmaf(s, F[a * kC32P + q0 + 32], a1);
    }
    Wa[rr * kC32P + q0] = a0;
    Wa[rr * kC32P + q0 + 32] = a1;
  }
  __syncthreads();
  {  // U = rows of Wa S_x^T
    float a0 = 0.f, a1 = 0.f;
    for (int b = 0; b < nux; ++b) {
      const float w = Wa[rr * kC32P + b];
      a0 = fmaf(w, Sx[q0 * kC32P + b], a0);
      a1 = fmaf(w, Sx[(q0 + 32) * kC32P + b], a1);
    }
    if (row < nuy) {
      float* out = u0 + (long)(fy0 + row) * c.Nx + c.firstx;
      if (q0 < nux) out[q0] = a0 - mean_u;
      if (q0 + 32 < nux) out[q0 + 32] = a1 - mean_u;
    }
  }
}

template <typename T>
cudaError_t launch_coarse(const CoarseView& c, const T* f0, T* u0, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (c.nux <= kC32 && c.nuy <= kC32) {
      const size_t sm = sizeof(float) * (3 * kC32 + 2 * kClRows) * kC32P;
      cudaError_t e = allow_smem(k_coarse_fdm32, sm);
      if (e != cudaSuccess) return e;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(kCl * std::max(1, c.batch));
      cfg.blockDim = dim3(kClThreads);
      cfg.dynamicSmemBytes = sm;
      cfg.stream = s;
      cudaLaunchAttribute attr[2];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = kCl;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[1].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 2;
      return cudaLaunchKernelEx(&cfg, k_coarse_fdm32, c, f0, u0);
    }
  }
  dim3 grid((c.nux + 7) / 8, (c.nuy + 7) / 8, std::max(1, c.batch));
  const size_t sm = 2 * 8 * sizeof(double) * (size_t)std::max(c.nux, c.nuy);
  cudaError_t e0 = allow_smem(k_coarse_gemm<T>, sm);
  if (e0 != cudaSuccess) return e0;
  for (int step = kStep1; step <= kStep4; ++step) {
    {
      const cudaError_t e_ = launch_pdl(k_coarse_gemm<T>, dim3(grid), dim3(256), sm, s, c, step, f0, u0);
      if (e_ != cudaSuccess) return e_;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_coarse_dense(const CoarseView& c, const double* Binv, const T* f0, T* u0, cudaStream_t s) {
  const int n = c.nux * c.nuy;
  const dim3 grid((n + 7) / 8, std::max(1, c.batch));
  {
    const cudaError_t e_ = launch_pdl(k_coarse_dense<T>, dim3(grid), dim3(256), 0, s, c, Binv, f0, u0);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}
template cudaError_t launch_coarse_dense<double>(const CoarseView&, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_coarse_dense<float>(const CoarseView&, const double*, const float*, float*, cudaStream_t);

template cudaError_t launch_restrict<double>(const DirView<double>&, const DirView<double>&, const DirView<double>&,
                                             const DirView<double>&, const double*, const double*, double*,
                                             cudaStream_t);
template cudaError_t launch_restrict<float>(const DirView<float>&, const DirView<float>&, const DirView<float>&,
                                            const DirView<float>&, const float*, const float*, float*, cudaStream_t);
template cudaError_t launch_prolong<double, double>(const DirView<double>&, const DirView<double>&,
                                                    const DirView<double>&, const DirView<double>&, const double*,
                                                    const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_prolong<float, float>(const DirView<float>&, const DirView<float>&, const DirView<float>&,
                                                  const DirView<float>&, const float*, const float*, const float*,
                                                  float*, cudaStream_t);
template cudaError_t launch_prolong<float, double>(const DirView<float>&, const DirView<float>&, const DirView<float>&,
                                                   const DirView<float>&, const float*, const float*, const float*,
                                                   double*, cudaStream_t);
template cudaError_t launch_coarse<double>(const CoarseView&, const double*, double*, cudaStream_t);
template cudaError_t launch_coarse<float>(const CoarseView&, const float*, float*, cudaStream_t);

}  // namespace sem
