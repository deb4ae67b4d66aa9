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
#include "kernels.h"

namespace sem {

namespace {

template <typename T, typename TIn>
__global__ void __launch_bounds__(256) k_sweep_simt(DirView<T> dx, DirView<T> dy, const TIn* __restrict__ r,
                                                    T* __restrict__ E, const float* __restrict__ nu_inv) {
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
    const int gy = node_or_wall(ey * p + a - no, dy.N, dy.periodic);
    const int gx = node_or_wall(ex * p + b - no, dx.N, dx.periodic);
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
  const T scale = nu_inv ? T(nu_inv[ey * dx.n + ex]) : T(1);
  T* Es = E + (long)(ey * dx.n + ex) * mm;
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    const int j = idx / m, i = idx - j * m;
    T s = T(0);
    for (int b = 0; b < m; ++b) s += Y[j * m + b] * Sx[i * m + b];
    Es[idx] = wy[j] * wx[i] * s * scale;
  }
}

template <typename T, typename TOut>
__global__ void __launch_bounds__(256) k_scatter(DirView<T> dx, DirView<T> dy, const T* __restrict__ E,
                                                 TOut* __restrict__ u, int accum) {
  const int p = dx.p, no = dx.n_o, m = dx.m, mm = m * m;
  const long n = (long)dx.N * dy.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int gj = (int)(idx / dx.N), gi = (int)(idx - (long)gj * dx.N);
    const bool wall = (!dx.periodic && (gi == 0 || gi == dx.N - 1)) || (!dy.periodic && (gj == 0 || gj == dy.N - 1));
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
    u[idx] = accum ? TOut(u[idx] + s) : TOut(s);
  }
}

}  // namespace

template <typename T, typename TIn>
cudaError_t launch_sweep(const DirView<T>& dx, const DirView<T>& dy, const TIn* r, T* E, int mode,
                         const float* nu_inv, cudaStream_t s) {
  (void)mode;
  const int m = dx.m;
  const size_t sm = sizeof(T) * (4 * m * m + 4 * m);
  cudaError_t e = allow_smem(k_sweep_simt<T, TIn>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid(dx.n, dy.n);
  k_sweep_simt<T, TIn><<<grid, 256, sm, s>>>(dx, dy, r, E, nu_inv);
  return cudaGetLastError();
}

template <typename T, typename TOut>
cudaError_t launch_scatter(const DirView<T>& dx, const DirView<T>& dy, const T* E, TOut* u, bool accum,
                           cudaStream_t s) {
  const long n = (long)dx.N * dy.N;
  const int grid = (int)std::min<long>((n + 255) / 256, 4 * 152 * 8);
  k_scatter<T, TOut><<<grid, 256, 0, s>>>(dx, dy, E, u, accum ? 1 : 0);
  return cudaGetLastError();
}

template cudaError_t launch_sweep<double, double>(const DirView<double>&, const DirView<double>&, const double*,
                                                  double*, int, const float*, cudaStream_t);
template cudaError_t launch_sweep<float, float>(const DirView<float>&, const DirView<float>&, const float*, float*,
                                                int, const float*, cudaStream_t);
template cudaError_t launch_sweep<float, double>(const DirView<float>&, const DirView<float>&, const double*,
                                                 float*, int, const float*, cudaStream_t);
template cudaError_t launch_scatter<double, double>(const DirView<double>&, const DirView<double>&, const double*,
                                                    double*, bool, cudaStream_t);
template cudaError_t launch_scatter<float, float>(const DirView<float>&, const DirView<float>&, const float*,
                                                  float*, bool, cudaStream_t);
template cudaError_t launch_scatter<float, double>(const DirView<float>&, const DirView<float>&, const float*,
                                                   double*, bool, cudaStream_t);

}  // namespace sem
