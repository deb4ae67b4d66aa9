// Weighted additive Schwarz sweep (Alg. 2, Eq. (correction:global)).
//
// k_sweep_simt: one CTA per subdomain s (extended element).  It gathers the
// m x m window R_s r (m = p + 1 + 2 n_o; slots outside a Dirichlet mesh read
// 0), applies the fast-diagonalisation inverse of Eq. (FDM)
//     X1 = S_y^T X,  X2 = X1 S_x ./ (lam_y + lam_x^T),  X4 = S_y X2,  X5 = X4 S_x^T,
// scales by the tensor-product weight w_y w_x^T (Eq. (weight function)) and
// writes W_s A_ss^{-1} R_s r into an element-blocked buffer E.  With a
// variable diffusivity the local solve is divided by nu_bar_s
// (Eq. (subproblem:solution)).
//
// k_scatter: node-centric, deterministic R_s^T sum: every node adds the
// E-entries of the (at most 3 x 3) windows that contain it, in a fixed order.
#include <algorithm>
#include <type_traits>

#include "kernels.h"
#include "level_ops.cuh"

namespace sem {

namespace {

template <typename T, typename TIn>
__global__ void __launch_bounds__(256) k_sweep_simt(DirView<T> dx, DirView<T> dy, const TIn* __restrict__ r,
                                                    T* __restrict__ E, const T* __restrict__ nu_inv) {
  pdl_enter();
  const int ex = blockIdx.x, ey = blockIdx.y;
  const int m = dx.m, mm = m * m, p = dx.p, no = dx.n_o;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);
  T* Y = X + mm;
  T* Sx = Y + mm;
  T* Sy = Sx + mm;
  T* lx = Sy + mm;
  T* ly = lx + m;
  T* wx = ly + m;
  T* wy = wx + m;
  const int tx = dx.tab[ex], ty = dy.tab[ey];
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    Sx[idx] = dx.S[(long)tx * mm + idx];
    Sy[idx] = dy.S[(long)ty * mm + idx];
    const int a = idx / m, b = idx - a * m;  // a: y slot, b: x slot
    const int gy = node_or_wall(ey * p + a - no, dy.N, dy.periodic, dy.segN);
    const int gx = node_or_wall(ex * p + b - no, dx.N, dx.periodic, dx.segN);
    X[idx] = (gx >= 0 && gy >= 0) ? T(r[(long)gy * dx.N + gx]) : T(0);
  }
  for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
    lx[idx] = dx.lam[tx * m + idx];
    ly[idx] = dy.lam[ty * m + idx];
    wx[idx] = dx.w[tx * m + idx];
    wy[idx] = dy.w[ty * m + idx];
  }
  __syncthreads();
  // X1 = S_y^T X : Y[a][i] = sum_j S_y[j][a] X[j][i]
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    const int a = idx / m, i = idx - a * m;
    T s = T(0);
    for (int j = 0; j < m; ++j) s += Sy[j * m + a] * X[j * m + i];
    Y[idx] = s;
  }
  __syncthreads();
  // X2 = X1 S_x ./ (lam_y + lam_x) : X[a][b]
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    const int a = idx / m, b = idx - a * m;
    T s = T(0);
    for (int i = 0; i < m; ++i) s += Y[a * m + i] * Sx[i * m + b];
    X[idx] = s / (ly[a] + lx[b]);
  }
  __syncthreads();
  // X4 = S_y X2 : Y[j][b] = sum_a S_y[j][a] X[a][b]
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    const int j = idx / m, b = idx - j * m;
    T s = T(0);
    for (int a = 0; a < m; ++a) s += Sy[j * m + a] * X[a * m + b];
    Y[idx] = s;
  }
  __syncthreads();
  // X5 = X4 S_x^T, weighted: E[j][i] = w_y[j] w_x[i] sum_b Y[j][b] S_x[i][b]
  const T scale = nu_inv ? nu_inv[ey * dx.n + ex] : T(1);
  T* Es = E + (long)(ey * dx.n + ex) * mm;
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    const int j = idx / m, i = idx - j * m;
    T s = T(0);
    for (int b = 0; b < m; ++b) s += Y[j * m + b] * Sx[i * m + b];
    Es[idx] = wy[j] * wx[i] * s * scale;
  }
}

// ---- tensor-core FDM ---------------------------------------------------------
template <typename TIn, int MODE, int MP>
__global__ void __launch_bounds__(32 * kMmaWarps) k_sweep_mma(DirView<float> dx, DirView<float> dy,
                                                              const TIn* __restrict__ r, float* __restrict__ E,
                                                              const float* __restrict__ nu_inv, int nsub) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  sweep_mma_warp<TIn, MODE, MP>(dx, dy, r, E, nu_inv, nsub, blockIdx.x * kMmaWarps + warp, gridDim.x * kMmaWarps,
                                reinterpret_cast<float*>(smem_raw) + warp * MmaSmem<MP>::PER_WARP);
}

template <typename TIn, int MODE, int MP>
cudaError_t sweep_mma_launch(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E,
                             const float* nu_inv, cudaStream_t s, int spw) {
  const size_t sm = sizeof(float) * MmaSmem<MP>::PER_WARP * kMmaWarps;
  cudaError_t e = allow_smem(k_sweep_mma<TIn, MODE, MP>, sm);
  if (e != cudaSuccess) return e;
  const int nsub = dx.n * dy.n;
  // about spw subdomains per warp; a warp that loops reuses its tables when
  // the next subdomain has the same type
  const int per = kMmaWarps * std::max(1, spw);
  const int grid = std::max(1, std::min((nsub + per - 1) / per, 152 * 16));
  {
    const cudaError_t e_ = launch_pdl(k_sweep_mma<TIn, MODE, MP>, dim3(grid), dim3(32 * kMmaWarps), sm, s, dx, dy, r, E, nu_inv, nsub);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

template <typename TIn, int MODE>
cudaError_t sweep_mma(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E,
                      const float* nu_inv, cudaStream_t s, int spw) {
  if (dx.m <= 16) return sweep_mma_launch<TIn, MODE, 16>(dx, dy, r, E, nu_inv, s, spw);
  if (dx.m <= 32) return sweep_mma_launch<TIn, MODE, 32>(dx, dy, r, E, nu_inv, s, spw);
  if (dx.m <= 48) return sweep_mma_launch<TIn, MODE, 48>(dx, dy, r, E, nu_inv, s, spw);
  return cudaErrorInvalidValue;
}

template <typename T, typename TOut>
__global__ void __launch_bounds__(256) k_scatter(DirView<T> dx, DirView<T> dy, const T* __restrict__ E,
                                                 TOut* __restrict__ u, int accum) {
  pdl_enter();
  const int p = dx.p, no = dx.n_o, m = dx.m, mm = m * m;
  const long n = (long)dx.N * dy.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int gj = (int)(idx / dx.N), gi = (int)(idx - (long)gj * dx.N);
    const bool wall = wall_node(gi, dx.N, dx.periodic, dx.segN) || wall_node(gj, dy.N, dy.periodic, dy.segN);
    if (wall) {
      if (!accum) u[idx] = TOut(0);
      continue;
    }
    // windows of element e cover global nodes e p - n_o .. e p + p + n_o
    const int ey_lo = floordiv(gj - p - no + p - 1, p), ey_hi = floordiv(gj + no, p);
    const int ex_lo = floordiv(gi - p - no + p - 1, p), ex_hi = floordiv(gi + no, p);
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
    u[idx] = accum ? TOut(u[idx] + convert_to<TOut>(s)) : convert_to<TOut>(s);
  }
}

}  // namespace

template <typename T, typename TIn>
cudaError_t launch_sweep(const DirView<T>& dx, const DirView<T>& dy, const TIn* r, T* E, int mode,
                         const T* nu_inv, cudaStream_t s, int spw) {
  if constexpr (std::is_same<T, float>::value) {
    if (mode == 1) return sweep_mma<TIn, 1>(dx, dy, r, E, nu_inv, s, spw);
    if (mode == 2) return sweep_mma<TIn, 2>(dx, dy, r, E, nu_inv, s, spw);
  }
  const int m = dx.m;
  const size_t sm = sizeof(T) * (4 * m * m + 4 * m);
  cudaError_t e = allow_smem(k_sweep_simt<T, TIn>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid(dx.n, dy.n);
  {
    const cudaError_t e_ = launch_pdl(k_sweep_simt<T, TIn>, dim3(grid), dim3(256), sm, s, dx, dy, r, E, nu_inv);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

template <typename T, typename TOut>
cudaError_t launch_scatter(const DirView<T>& dx, const DirView<T>& dy, const T* E, TOut* u, bool accum,
                           cudaStream_t s) {
  const long n = (long)dx.N * dy.N;
  const int grid = (int)std::min<long>((n + 255) / 256, 4 * 152 * 8);
  {
    const cudaError_t e_ = launch_pdl(k_scatter<T, TOut>, dim3(grid), dim3(256), 0, s, dx, dy, E, u, accum ? 1 : 0);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

template cudaError_t launch_sweep<double, double>(const DirView<double>&, const DirView<double>&, const double*,
                                                  double*, int, const double*, cudaStream_t, int);
template cudaError_t launch_sweep<float, float>(const DirView<float>&, const DirView<float>&, const float*, float*,
                                                int, const float*, cudaStream_t, int);
template cudaError_t launch_sweep<float, double>(const DirView<float>&, const DirView<float>&, const double*,
                                                 float*, int, const float*, cudaStream_t, int);
template cudaError_t launch_scatter<double, double>(const DirView<double>&, const DirView<double>&, const double*,
                                                    double*, bool, cudaStream_t);
template cudaError_t launch_scatter<float, float>(const DirView<float>&, const DirView<float>&, const float*,
                                                  float*, bool, cudaStream_t);
template cudaError_t launch_scatter<float, double>(const DirView<float>&, const DirView<float>&, const float*,
                                                   double*, bool, cudaStream_t);

}  // namespace sem
