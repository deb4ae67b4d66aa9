// Multiplicative Schwarz sweep (Alg. 1) with a coloured subdomain order.
//
// Alg. 1 visits the subdomains one after another; before each local solve the
// residual r = f - A u is recomputed, and the local solution A_ss^{-1} R_s r
// is added on the element's own closed node set (element-local indices
// 0..p in both directions, interface nodes included, no weights), while the
// local problem itself is posed on the whole extended subdomain of Sec. 3.1.
//
// Order.  The subdomains are grouped into colour classes
// c = (e_y mod q_y) q_x + (e_x mod q_x), q = 3 on a Dirichlet mesh and the
// smallest divisor q >= 3 of n on a periodic one.  Two subdomains of a class
// are at least q >= 3 elements apart in x or in y (also across a periodic
// wrap), so the update of one (its element's closed nodes) changes the
// residual only on the element and its neighbours, which never reaches the
// other's window (n_o <= p - 1).  The subdomains of a class can therefore be
// solved at the same time with the same result as one after another; the
// classes run in increasing c, in decreasing c on every second sweep (the
// reversal of Alg. 1).  This class order replaces the paper's lexicographic
// order.
//
// k_mult: one CTA per subdomain of one class.  The CTA stages u on the
// (3p+1)^2 nodes of the element and its eight neighbours, the stiffness of the
// three element columns and rows involved and the assembled mass there, forms
// r on the window with the assembled tensor form
//     (A u)(j, i) = M_y(j) (L_x u_j)(i) + M_x(i) (L_y u^i)(j)
// (Eq. (system matrix)), applies the fast-diagonalisation inverse of Eq. (FDM)
// and adds the result to u on the closed element.  Within a class no CTA reads
// a node another one writes (the staged blocks of two class members are
// disjoint from each other's closed elements).
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace sem {

namespace {

template <typename T, typename TU, typename TF>
__global__ void __launch_bounds__(256) k_mult(DirView<T> dx, DirView<T> dy, TU* __restrict__ u,
                                              const TF* __restrict__ f, int cx, int cy, int qx, int qy) {
  pdl_enter();
  const int ex = cx + qx * (int)blockIdx.x, ey = cy + qy * (int)blockIdx.y;
  const int p = dx.p, np1 = p + 1, no = dx.n_o, m = dx.m, mm = m * m;
  const int B = 3 * p + 1;  // staged block: nodes (e - 1) p .. (e + 2) p per direction
  const int Nx = dx.N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* U = reinterpret_cast<T*>(smem_raw);  // B x B, row = y
  T* X = U + B * B;
  T* Y = X + mm;
  T* Sx = Y + mm;
  T* Sy = Sx + mm;
  T* lx = Sy + mm;
  T* ly = lx + m;
  T* Lx = ly + m;           // 3 x np1 x np1: element columns ex - 1, ex, ex + 1
  T* Ly = Lx + 3 * np1 * np1;
  T* Mx = Ly + 3 * np1 * np1;  // B: assembled mass at the block's nodes
  T* My = Mx + B;
  const int x0 = (ex - 1) * p, y0 = (ey - 1) * p;
  for (int idx = threadIdx.x; idx < B * B; idx += blockDim.x) {
    const int by = idx / B, bx = idx - by * B;
    const int gy = node_or_wall(y0 + by, dy.N, dy.periodic);
    const int gx = node_or_wall(x0 + bx, dx.N, dx.periodic);
    U[idx] = (gx >= 0 && gy >= 0) ? T(u[(long)gy * Nx + gx]) : T(0);
  }
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int gx = node_or_wall(x0 + b, dx.N, dx.periodic);
    const int gy = node_or_wall(y0 + b, dy.N, dy.periodic);
    Mx[b] = gx >= 0 ? dx.Mg[gx] : T(0);
    My[b] = gy >= 0 ? dy.Mg[gy] : T(0);
  }
  for (int idx = threadIdx.x; idx < 3 * np1 * np1; idx += blockDim.x) {
    const int k = idx / (np1 * np1), ab = idx - k * np1 * np1;
    int exk = ex - 1 + k, eyk = ey - 1 + k;
    if (dx.periodic) exk = (exk + dx.n) % dx.n;
    if (dy.periodic) eyk = (eyk + dy.n) % dy.n;
    Lx[idx] = (exk >= 0 && exk < dx.n) ? dx.Le[(long)exk * np1 * np1 + ab] : T(0);
    Ly[idx] = (eyk >= 0 && eyk < dy.n) ? dy.Le[(long)eyk * np1 * np1 + ab] : T(0);
  }
  const int tx = dx.tab[ex], ty = dy.tab[ey];
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    Sx[idx] = dx.S[(long)tx * mm + idx];
    Sy[idx] = dy.S[(long)ty * mm + idx];
  }
  for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
    lx[idx] = dx.lam[tx * m + idx];
    ly[idx] = dy.lam[ty * m + idx];
  }
  __syncthreads();
  // R_s r on the window: slot (a, b) is block node (a - n_o + p, b - n_o + p)
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    const int a = idx / m, b = idx - a * m;
    const int gy = node_or_wall(ey * p + a - no, dy.N, dy.periodic);
    const int gx = node_or_wall(ex * p + b - no, dx.N, dx.periodic);
    if (gx < 0 || gy < 0) {
      X[idx] = T(0);
      continue;
    }
    const int by = a - no + p, bx = b - no + p;  // 1 .. 3p - 1
    // (L_x u_j)(i): the element column holding bx, and its left neighbour
    // when bx is an interface node
    const int kx = bx / p, ix = bx - kx * p;
    const T* urow = U + by * B;
    T sx = T(0);
    {
      const T* Lr = Lx + (kx * np1 + ix) * np1;
      const T* ur = urow + kx * p;
      for (int k = 0; k <= p; ++k) sx += Lr[k] * ur[k];
      if (ix == 0) {
        const T* Ll = Lx + ((kx - 1) * np1 + p) * np1;
        const T* ul = urow + (kx - 1) * p;
        for (int k = 0; k <= p; ++k) sx += Ll[k] * ul[k];
      }
    }
    const int ky = by / p, iy = by - ky * p;
    T sy = T(0);
    {
      const T* Lr = Ly + (ky * np1 + iy) * np1;
      const T* uc = U + (ky * p) * B + bx;
      for (int k = 0; k <= p; ++k) sy += Lr[k] * uc[k * B];
      if (iy == 0) {
        const T* Ll = Ly + ((ky - 1) * np1 + p) * np1;
        const T* ul = U + ((ky - 1) * p) * B + bx;
        for (int k = 0; k <= p; ++k) sy += Ll[k] * ul[k * B];
      }
    }
    X[idx] = convert_to<T>(f[(long)gy * Nx + gx]) - (My[by] * sx + Mx[bx] * sy);
  }
  __syncthreads();
  // Eq. (FDM): X1 = S_y^T X, X2 = X1 S_x ./ (lam_y + lam_x), X4 = S_y X2, X5 = X4 S_x^T
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    const int a = idx / m, i = idx - a * m;
    T s = T(0);
    for (int j = 0; j < m; ++j) s += Sy[j * m + a] * X[j * m + i];
    Y[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    const int a = idx / m, b = idx - a * m;
    T s = T(0);
    for (int i = 0; i < m; ++i) s += Y[a * m + i] * Sx[i * m + b];
    X[idx] = s / (ly[a] + lx[b]);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    const int j = idx / m, b = idx - j * m;
    T s = T(0);
    for (int a = 0; a < m; ++a) s += Sy[j * m + a] * X[a * m + b];
    Y[idx] = s;
  }
  __syncthreads();
  // X5 on the closed element only, added to u
  for (int idx = threadIdx.x; idx < np1 * np1; idx += blockDim.x) {
    const int jl = idx / np1, il = idx - jl * np1;
    const int gy = node_or_wall(ey * p + jl, dy.N, dy.periodic);
    const int gx = node_or_wall(ex * p + il, dx.N, dx.periodic);
    if (gx < 0 || gy < 0) continue;
    const int j = jl + no, i = il + no;
    T s = T(0);
    for (int b = 0; b < m; ++b) s += Y[j * m + b] * Sx[i * m + b];
    TU* up = u + (long)gy * Nx + gx;
    *up = TU(*up + convert_to<TU>(s));
  }
}

}  // namespace

int mult_colours(int n, bool periodic) {
  if (!periodic) return 3;
  for (int q = 3; q <= n; ++q)
    if (n % q == 0) return q;
  return 0;
}

size_t mult_smem_bytes(int p, int m, size_t tsize) {
  const size_t B = 3 * (size_t)p + 1, np1 = (size_t)p + 1;
  return tsize * (B * B + 4 * (size_t)m * m + 2 * (size_t)m + 6 * np1 * np1 + 2 * B);
}

template <typename T, typename TU, typename TF>
cudaError_t launch_mult_sweep(const DirView<T>& dx, const DirView<T>& dy, TU* u, const TF* f, bool reverse,
                              cudaStream_t s, int* launches) {
  const int qx = mult_colours(dx.n, dx.periodic != 0), qy = mult_colours(dy.n, dy.periodic != 0);
  if (qx < 3 || qy < 3 || dx.segN || dy.segN) return cudaErrorInvalidValue;
  const size_t sm = mult_smem_bytes(dx.p, dx.m, sizeof(T));
  cudaError_t e = allow_smem(k_mult<T, TU, TF>, sm);
  if (e != cudaSuccess) return e;
  const int nc = qx * qy;
  int nl = 0;
  for (int k = 0; k < nc; ++k) {
    const int c = reverse ? nc - 1 - k : k;
    const int cy = c / qx, cx = c - cy * qx;
    const int gx = (dx.n - cx + qx - 1) / qx, gy = (dy.n - cy + qy - 1) / qy;
    if (gx <= 0 || gy <= 0) continue;
    e = launch_pdl(k_mult<T, TU, TF>, dim3(gx, gy), dim3(256), sm, s, dx, dy, u, f, cx, cy, qx, qy);
    if (e != cudaSuccess) return e;
    ++nl;
  }
  if (launches) *launches = nl;
  return cudaGetLastError();
}

template cudaError_t launch_mult_sweep<double, double, double>(const DirView<double>&, const DirView<double>&,
                                                               double*, const double*, bool, cudaStream_t, int*);
template cudaError_t launch_mult_sweep<float, float, float>(const DirView<float>&, const DirView<float>&, float*,
                                                            const float*, bool, cudaStream_t, int*);
template cudaError_t launch_mult_sweep<float, float, double>(const DirView<float>&, const DirView<float>&, float*,
                                                             const double*, bool, cudaStream_t, int*);
template cudaError_t launch_mult_sweep<float, double, double>(const DirView<float>&, const DirView<float>&, double*,
                                                              const double*, bool, cudaStream_t, int*);

}  // namespace sem
