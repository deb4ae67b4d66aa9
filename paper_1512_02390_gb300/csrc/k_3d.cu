// Kernels of the three-dimensional extension (the paper's concluding section
// names the extension to three space dimensions as future work).
//
// A field is the node grid (Nz, Ny, Nx), x fastest.  Every kernel is
// deterministic: outputs are written once by their owner, sums run in a fixed
// order, no atomics on values.
//   k3_apply     node-centric A u of Eq. (system matrix) in 3D:
//                (A u)(k,j,i) = M_z M_y (L_x u)(i) + M_z M_x (L_y u)(j) + M_y M_x (L_z u)(k)
//                with the assembled 1D stiffness applied along each axis.
//   k3_sweep     one CTA per extended-element subdomain (Sec. 3.1): gather of
//                the m^3 window, the fast-diagonalisation inverse with three
//                contractions on each side (Eq. (FDM) one dimension up), the
//                weights W_z (x) W_y (x) W_x; writes the element-blocked E.
//   k3_scatter   node-centric R_s^T sum of Alg. 2 over the <= 27 windows.
//   k3_prolong   out = in + (J (x) J (x) J) uc element by element, sum-factorised;
//                each fine node written by the one element that owns it.
//   k3_restrict  (J (x) J (x) J)^T of every element's owned fine nodes into an
//                element-blocked buffer, then a node-centric coarse gather.
//   k3_axis      the dense contractions of the coarse fast diagonalisation.
#include <algorithm>

#include "kernels3d.h"

namespace sem {

namespace {

// (L u)(g) along one axis: u at axis node h is u[base + h * stride]; the
// assembled row of node g is the element row of each element holding g.
template <typename T>
__device__ __forceinline__ T axis_sum(const DirView<T>& d, int g, const T* __restrict__ u, long base, long stride) {
  const int p = d.p, np1 = p + 1;
  const int e = g / p, a = g - e * p;
  T s = T(0);
  {
    const T* L = d.Le + (long)e * np1 * np1 + a * np1;
    for (int k = 0; k <= p; ++k) {
      const int h = node_or_wall(e * p + k, d.N, d.periodic);
      if (h >= 0) s += L[k] * u[base + (long)h * stride];
    }
  }
  if (a == 0 && (e > 0 || d.periodic)) {
    const int el = e > 0 ? e - 1 : d.n - 1;
    const T* L = d.Le + (long)el * np1 * np1 + p * np1;
    for (int k = 0; k <= p; ++k) {
      const int h = node_or_wall(el * p + k, d.N, d.periodic);
      if (h >= 0) s += L[k] * u[base + (long)h * stride];
    }
  }
  return s;
}

template <typename T, typename TF>
__global__ void __launch_bounds__(256) k3_apply(DirView<T> dx, DirView<T> dy, DirView<T> dz, const T* __restrict__ u,
                                                const TF* __restrict__ f, T* __restrict__ out) {
  const long NX = dx.N, NY = dy.N, n = NX * NY * dz.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int gi = (int)(idx % NX);
    const int gj = (int)((idx / NX) % NY);
    const int gk = (int)(idx / (NX * NY));
    if (wall_node(gi, dx.N, dx.periodic) || wall_node(gj, dy.N, dy.periodic) || wall_node(gk, dz.N, dz.periodic)) {
      out[idx] = T(0);
      continue;
    }
    const T sx = axis_sum(dx, gi, u, idx - gi, 1);
    const T sy = axis_sum(dy, gj, u, idx - (long)gj * NX, NX);
    const T sz = axis_sum(dz, gk, u, idx - (long)gk * NX * NY, NX * NY);
    const T mx = dx.Mg[gi], my = dy.Mg[gj], mz = dz.Mg[gk];
    const T au = mz * my * sx + mz * mx * sy + my * mx * sz;
    out[idx] = f ? T(f[idx]) - au : au;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k3_mass(DirView<T> dx, DirView<T> dy, DirView<T> dz, const T* __restrict__ fn,
                                               T* __restrict__ b) {
  const long NX = dx.N, NY = dy.N, n = NX * NY * dz.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int gi = (int)(idx % NX), gj = (int)((idx / NX) % NY), gk = (int)(idx / (NX * NY));
    const bool wall =
        wall_node(gi, dx.N, dx.periodic) || wall_node(gj, dy.N, dy.periodic) || wall_node(gk, dz.N, dz.periodic);
    b[idx] = wall ? T(0) : dz.Mg[gk] * dy.Mg[gj] * dx.Mg[gi] * fn[idx];
  }
}

// Shared memory of k3_sweep: two m^3 buffers, three m x m tables, six m-vectors.
template <typename T>
size_t sweep3_smem(int m) {
  return sizeof(T) * (2 * (size_t)m * m * m + 3 * (size_t)m * m + 6 * (size_t)m);
}

template <typename T>
__global__ void __launch_bounds__(256) k3_sweep(DirView<T> dx, DirView<T> dy, DirView<T> dz, const T* __restrict__ r,
                                                T* __restrict__ E) {
  const int ex = blockIdx.x, ey = blockIdx.y, ez = blockIdx.z;
  const int m = dx.m, mm = m * m, mmm = mm * m, p = dx.p, no = dx.n_o;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);
  T* Y = X + mmm;
  T* Sx = Y + mmm;
  T* Sy = Sx + mm;
  T* Sz = Sy + mm;
  T* lx = Sz + mm;
  T* ly = lx + m;
  T* lz = ly + m;
  T* wx = lz + m;
  T* wy = wx + m;
  T* wz = wy + m;
  const int tx = dx.tab[ex], ty = dy.tab[ey], tz = dz.tab[ez];
  const long NX = dx.N, NY = dy.N;
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {
    const int c = idx / mm, b = (idx / m) % m, a = idx % m;  // z, y, x slots
    const int gz = node_or_wall(ez * p + c - no, dz.N, dz.periodic);
    const int gy = node_or_wall(ey * p + b - no, dy.N, dy.periodic);
    const int gx = node_or_wall(ex * p + a - no, dx.N, dx.periodic);
    X[idx] = (gx >= 0 && gy >= 0 && gz >= 0) ? r[((long)gz * NY + gy) * NX + gx] : T(0);
  }
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
    Sx[idx] = dx.S[(long)tx * mm + idx];
    Sy[idx] = dy.S[(long)ty * mm + idx];
    Sz[idx] = dz.S[(long)tz * mm + idx];
  }
  for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
    lx[idx] = dx.lam[tx * m + idx];
    ly[idx] = dy.lam[ty * m + idx];
    lz[idx] = dz.lam[tz * m + idx];
    wx[idx] = dx.w[tx * m + idx];
    wy[idx] = dy.w[ty * m + idx];
    wz[idx] = dz.w[tz * m + idx];
  }
  __syncthreads();
  // forward: contract the window slot of each axis with S (S^T applied)
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // z: Y[a'][j][i]
    const int c2 = idx / mm, rest = idx - c2 * mm;
    T s = T(0);
    for (int k = 0; k < m; ++k) s += Sz[k * m + c2] * X[k * mm + rest];
    Y[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // y: X[a'][b'][i]
    const int c2 = idx / mm, b2 = (idx / m) % m, i = idx % m;
    T s = T(0);
    for (int j = 0; j < m; ++j) s += Sy[j * m + b2] * Y[c2 * mm + j * m + i];
    X[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // x and the eigenvalue division
    const int c2 = idx / mm, b2 = (idx / m) % m, a2 = idx % m;
    T s = T(0);
    for (int i = 0; i < m; ++i) s += Sx[i * m + a2] * X[c2 * mm + b2 * m + i];
    Y[idx] = s / (lz[c2] + ly[b2] + lx[a2]);
  }
  __syncthreads();
  // backward: S applied along each axis
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // z: X[k][b'][a']
    const int k = idx / mm, rest = idx - k * mm;
    T s = T(0);
    for (int c2 = 0; c2 < m; ++c2) s += Sz[k * m + c2] * Y[c2 * mm + rest];
    X[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // y: Y[k][j][a']
    const int k = idx / mm, j = (idx / m) % m, a2 = idx % m;
    T s = T(0);
    for (int b2 = 0; b2 < m; ++b2) s += Sy[j * m + b2] * X[k * mm + b2 * m + a2];
    Y[idx] = s;
  }
  __syncthreads();
  T* Es = E + (((long)ez * dy.n + ey) * dx.n + ex) * mmm;
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // x, weights, out
    const int k = idx / mm, j = (idx / m) % m, i = idx % m;
    T s = T(0);
    for (int a2 = 0; a2 < m; ++a2) s += Sx[i * m + a2] * Y[k * mm + j * m + a2];
    Es[idx] = wz[k] * wy[j] * wx[i] * s;
  }
}

// element e' of the window holding node g along one axis, and the node's
// slot in it; returns the count (<= 3)
template <typename T>
__device__ __forceinline__ int windows_of(const DirView<T>& d, int g, int* el, int* slot) {
  const int p = d.p, no = d.n_o;
  const int lo = floordiv(g - no - 1, p), hi = floordiv(g + no, p);
  int c = 0;
  for (int eu = lo; eu <= hi; ++eu) {
    int e = eu;
    if (d.periodic) e = ((e % d.n) + d.n) % d.n;
    else if (e < 0 || e >= d.n) continue;
    el[c] = e;
    slot[c] = g - eu * p + no;
    ++c;
  }
  return c;
}

template <typename T, typename TOut>
__global__ void __launch_bounds__(256) k3_scatter(DirView<T> dx, DirView<T> dy, DirView<T> dz, const T* __restrict__ E,
                                                  TOut* __restrict__ u, int accum) {
  const int m = dx.m;
  const long mmm = (long)m * m * m;
  const long NX = dx.N, NY = dy.N, n = NX * NY * dz.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int gi = (int)(idx % NX), gj = (int)((idx / NX) % NY), gk = (int)(idx / (NX * NY));
    if (wall_node(gi, dx.N, dx.periodic) || wall_node(gj, dy.N, dy.periodic) || wall_node(gk, dz.N, dz.periodic)) {
      if (!accum) u[idx] = TOut(0);
      continue;
    }
    int ex[3], sx[3], ey[3], sy[3], ez[3], sz[3];
    const int nx = windows_of(dx, gi, ex, sx), ny = windows_of(dy, gj, ey, sy), nz = windows_of(dz, gk, ez, sz);
    T s = T(0);
    for (int a = 0; a < nz; ++a)
      for (int b = 0; b < ny; ++b)
        for (int c = 0; c < nx; ++c)
          s += E[(((long)ez[a] * dy.n + ey[b]) * dx.n + ex[c]) * mmm + ((long)sz[a] * m + sy[b]) * m + sx[c]];
    u[idx] = accum ? TOut(u[idx] + TOut(s)) : TOut(s);
  }
}

// fine node g of element e at local index l is owned by e when l < p, and the
// last local index belongs to the last element of a Dirichlet direction
template <typename T>
__device__ __forceinline__ bool owns(const DirView<T>& d, int e, int l) {
  return l < d.p || (!d.periodic && e == d.n - 1);
}

// global node of local index l of element e (wrapped when periodic)
template <typename T>
__device__ __forceinline__ int node_of(const DirView<T>& d, int e, int l) {
  const int g = e * d.p + l;
  return d.periodic ? g % d.N : g;
}

template <typename T, typename TOut>
__global__ void __launch_bounds__(256) k3_prolong(DirView<T> fx, DirView<T> fy, DirView<T> fz, DirView<T> cx,
                                                  DirView<T> cy, DirView<T> cz, const T* __restrict__ J,
                                                  const T* __restrict__ uc, const T* __restrict__ in,
                                                  TOut* __restrict__ out) {
  const int ex = blockIdx.x, ey = blockIdx.y, ez = blockIdx.z;
  const int pf = fx.p, pc = cx.p, nf = pf + 1, nc = pc + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* U0 = reinterpret_cast<T*>(smem_raw);  // nc^3
  T* T1 = U0 + nc * nc * nc;               // nc x nc x nf
  T* T2 = T1 + nc * nc * nf;               // nc x nf x nf
  T* sJ = T2 + nc * nf * nf;               // nf x nc
  const long CX = cx.N, CY = cy.N;
  for (int idx = threadIdx.x; idx < nc * nc * nc; idx += blockDim.x) {
    const int c = idx / (nc * nc), b = (idx / nc) % nc, a = idx % nc;
    const int gz = node_or_wall(ez * pc + c, cz.N, cz.periodic);
    const int gy = node_or_wall(ey * pc + b, cy.N, cy.periodic);
    const int gx = node_or_wall(ex * pc + a, cx.N, cx.periodic);
    U0[idx] = (gx >= 0 && gy >= 0 && gz >= 0) ? uc[((long)gz * CY + gy) * CX + gx] : T(0);
  }
  for (int idx = threadIdx.x; idx < nf * nc; idx += blockDim.x) sJ[idx] = J[idx];
  __syncthreads();
  for (int idx = threadIdx.x; idx < nc * nc * nf; idx += blockDim.x) {
    const int c = idx / (nc * nf), b = (idx / nf) % nc, i = idx % nf;
    T s = T(0);
    for (int a = 0; a < nc; ++a) s += sJ[i * nc + a] * U0[(c * nc + b) * nc + a];
    T1[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nc * nf * nf; idx += blockDim.x) {
    const int c = idx / (nf * nf), j = (idx / nf) % nf, i = idx % nf;
    T s = T(0);
    for (int b = 0; b < nc; ++b) s += sJ[j * nc + b] * T1[(c * nc + b) * nf + i];
    T2[idx] = s;
  }
  __syncthreads();
  const long FX = fx.N, FY = fy.N;
  for (int idx = threadIdx.x; idx < nf * nf * nf; idx += blockDim.x) {
    const int k = idx / (nf * nf), j = (idx / nf) % nf, i = idx % nf;
    if (!owns(fz, ez, k) || !owns(fy, ey, j) || !owns(fx, ex, i)) continue;
    const int gz = node_of(fz, ez, k), gy = node_of(fy, ey, j), gx = node_of(fx, ex, i);
    const long o = ((long)gz * FY + gy) * FX + gx;
    if (wall_node(gx, fx.N, fx.periodic) || wall_node(gy, fy.N, fy.periodic) || wall_node(gz, fz.N, fz.periodic)) {
      out[o] = TOut(0);
      continue;
    }
    T s = T(0);
    for (int c = 0; c < nc; ++c) s += sJ[k * nc + c] * T2[(c * nf + j) * nf + i];
    out[o] = in ? TOut(TOut(in[o]) + TOut(s)) : TOut(s);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k3_restrict_elem(DirView<T> fx, DirView<T> fy, DirView<T> fz, DirView<T> cx,
                                                        const T* __restrict__ J, const T* __restrict__ rf,
                                                        T* __restrict__ Ec) {
  const int ex = blockIdx.x, ey = blockIdx.y, ez = blockIdx.z;
  const int pf = fx.p, pc = cx.p, nf = pf + 1, nc = pc + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* R = reinterpret_cast<T*>(smem_raw);  // nf^3 owned fine values
  T* T1 = R + nf * nf * nf;               // nf x nf x nc
  T* T2 = T1 + nf * nf * nc;              // nf x nc x nc
  T* sJ = T2 + nf * nc * nc;              // nf x nc
  const long FX = fx.N, FY = fy.N;
  for (int idx = threadIdx.x; idx < nf * nf * nf; idx += blockDim.x) {
    const int k = idx / (nf * nf), j = (idx / nf) % nf, i = idx % nf;
    T v = T(0);
    if (owns(fz, ez, k) && owns(fy, ey, j) && owns(fx, ex, i)) {
      const int gz = node_or_wall(ez * pf + k, fz.N, fz.periodic);
      const int gy = node_or_wall(ey * pf + j, fy.N, fy.periodic);
      const int gx = node_or_wall(ex * pf + i, fx.N, fx.periodic);
      if (gx >= 0 && gy >= 0 && gz >= 0) v = rf[((long)gz * FY + gy) * FX + gx];
    }
    R[idx] = v;
  }
  for (int idx = threadIdx.x; idx < nf * nc; idx += blockDim.x) sJ[idx] = J[idx];
  __syncthreads();
  for (int idx = threadIdx.x; idx < nf * nf * nc; idx += blockDim.x) {  // x: T1[k][j][a]
    const int k = idx / (nf * nc), j = (idx / nc) % nf, a = idx % nc;
    T s = T(0);
    for (int i = 0; i < nf; ++i) s += sJ[i * nc + a] * R[(k * nf + j) * nf + i];
    T1[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nf * nc * nc; idx += blockDim.x) {  // y: T2[k][b][a]
    const int k = idx / (nc * nc), b = (idx / nc) % nc, a = idx % nc;
    T s = T(0);
    for (int j = 0; j < nf; ++j) s += sJ[j * nc + b] * T1[(k * nf + j) * nc + a];
    T2[idx] = s;
  }
  __syncthreads();
  T* Es = Ec + (((long)ez * fy.n + ey) * fx.n + ex) * nc * nc * nc;
  for (int idx = threadIdx.x; idx < nc * nc * nc; idx += blockDim.x) {  // z: Ec[c][b][a]
    const int c = idx / (nc * nc), rest = idx - c * nc * nc;
    T s = T(0);
    for (int k = 0; k < nf; ++k) s += sJ[k * nc + c] * T2[k * nc * nc + rest];
    Es[idx] = s;
  }
}

// elements holding coarse node g along one axis (local index pc or 0)
template <typename T>
__device__ __forceinline__ int elems_of(const DirView<T>& c, int g, int* el, int* loc) {
  const int p = c.p;
  const int e = g / p, a = g - e * p;
  int n = 0;
  if (a == 0 && (e > 0 || c.periodic)) {
    el[n] = e > 0 ? e - 1 : c.n - 1;
    loc[n] = p;
    ++n;
  }
  if (e < c.n) {
    el[n] = e;
    loc[n] = a;
    ++n;
  }
  return n;
}

template <typename T>
__global__ void __launch_bounds__(256) k3_restrict_gather(DirView<T> cx, DirView<T> cy, DirView<T> cz,
                                                          const T* __restrict__ Ec, T* __restrict__ fc) {
  const int nc = cx.p + 1;
  const long NX = cx.N, NY = cy.N, n = NX * NY * cz.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int gi = (int)(idx % NX), gj = (int)((idx / NX) % NY), gk = (int)(idx / (NX * NY));
    if (wall_node(gi, cx.N, cx.periodic) || wall_node(gj, cy.N, cy.periodic) || wall_node(gk, cz.N, cz.periodic)) {
      fc[idx] = T(0);
      continue;
    }
    int ex[2], ax[2], ey[2], ay[2], ez[2], az[2];
    const int nx = elems_of(cx, gi, ex, ax), ny = elems_of(cy, gj, ey, ay), nz = elems_of(cz, gk, ez, az);
    T s = T(0);
    for (int a = 0; a < nz; ++a)
      for (int b = 0; b < ny; ++b)
        for (int c = 0; c < nx; ++c)
          s += Ec[(((long)ez[a] * cy.n + ey[b]) * cx.n + ex[c]) * nc * nc * nc + (az[a] * nc + ay[b]) * nc + ax[c]];
    fc[idx] = s;
  }
}

// Coarse fast diagonalisation on the compact unknown grid (nuz, nuy, nux).
// compact <-> node grid: unpack = 0 copies the grid's unknowns into the
// compact array, 1 the compact array into the grid (its walls stay 0)
template <typename T>
__global__ void __launch_bounds__(256) k3_pack(T* __restrict__ g, T* __restrict__ c, Coarse3<T> cv, int unpack) {
  const long n = (long)cv.nu[0] * cv.nu[1] * cv.nu[2];
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int a = (int)(idx % cv.nu[0]), b = (int)((idx / cv.nu[0]) % cv.nu[1]);
    const int k = (int)(idx / ((long)cv.nu[0] * cv.nu[1]));
    const long o = ((long)(cv.first[2] + k) * cv.N[1] + cv.first[1] + b) * cv.N[0] + cv.first[0] + a;
    if (unpack) g[o] = c[idx];
    else c[idx] = g[o];
  }
}

// out = M in along `axis` (0 x, 1 y, 2 z) of the compact grid; M(i, a) is
// S[a * nu + i] when tr (S^T) and S[i * nu + a] otherwise.  With lam != null
// the result is divided by lam_z + lam_y + lam_x (mode (0,0,0) dropped when
// the problem is singular).
template <typename T>
__global__ void __launch_bounds__(256) k3_axis(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ S,
                                               Coarse3<T> cv, int axis, int tr, int divide) {
  const int nu0 = cv.nu[0], nu1 = cv.nu[1], nu2 = cv.nu[2];
  const long n = (long)nu0 * nu1 * nu2;
  const int nu = cv.nu[axis];
  const long stride = axis == 0 ? 1 : (axis == 1 ? nu0 : (long)nu0 * nu1);
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int c0 = (int)(idx % nu0), c1 = (int)((idx / nu0) % nu1), c2 = (int)(idx / ((long)nu0 * nu1));
    const int i = axis == 0 ? c0 : (axis == 1 ? c1 : c2);
    const long base = idx - (long)i * stride;
    T s = T(0);
    for (int a = 0; a < nu; ++a) s += (tr ? S[(long)a * nu + i] : S[(long)i * nu + a]) * in[base + a * stride];
    if (divide) {
      const T den = cv.lam[0][c0] + cv.lam[1][c1] + cv.lam[2][c2];
      s = (cv.singular && c0 == 0 && c1 == 0 && c2 == 0) ? T(0) : s / den;
    }
    out[idx] = s;
  }
}

// x -= mean(x) over the compact coarse grid, one CTA (fixed-order sum)
template <typename T>
__global__ void __launch_bounds__(1024) k3_sub_mean(T* x, long n) {
  __shared__ double red[1024];
  double s = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) s += (double)x[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const T mean = T(red[0] / (double)n);
  for (long i = threadIdx.x; i < n; i += blockDim.x) x[i] -= mean;
}

__global__ void __launch_bounds__(256) k3_dot(const double* __restrict__ a, const double* __restrict__ b, long n,
                                              double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) s += a[i] * b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// y = a x + b y (x may be null: y = b y)
__global__ void __launch_bounds__(256) k3_axpby(long n, double a, const double* __restrict__ x, double b,
                                                double* __restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = (x ? a * x[i] : 0.0) + b * y[i];
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k3_convert(long n, const TA* __restrict__ a, TB* __restrict__ b) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) b[i] = TB(a[i]);
}

int grid_for(long n) { return (int)std::max<long>(1, std::min<long>((n + 255) / 256, 152 * 16)); }

}  // namespace

template <typename T, typename TF>
cudaError_t launch3_apply(const Dir3<T>& d, const T* u, const TF* f, T* out, cudaStream_t s) {
  const long n = (long)d.x.N * d.y.N * d.z.N;
  k3_apply<T, TF><<<grid_for(n), 256, 0, s>>>(d.x, d.y, d.z, u, f, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch3_mass(const Dir3<T>& d, const T* fn, T* b, cudaStream_t s) {
  const long n = (long)d.x.N * d.y.N * d.z.N;
  k3_mass<T><<<grid_for(n), 256, 0, s>>>(d.x, d.y, d.z, fn, b);
  return cudaGetLastError();
}

template <typename T>
size_t sweep3_smem_bytes(int m) {
  return sweep3_smem<T>(m);
}

template <typename T, typename TOut>
cudaError_t launch3_sweep(const Dir3<T>& d, const T* r, T* E, TOut* u, bool accum, cudaStream_t s) {
  const size_t sm = sweep3_smem<T>(d.x.m);
  cudaError_t e = allow_smem(k3_sweep<T>, sm);
  if (e != cudaSuccess) return e;
  k3_sweep<T><<<dim3(d.x.n, d.y.n, d.z.n), 256, sm, s>>>(d.x, d.y, d.z, r, E);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long n = (long)d.x.N * d.y.N * d.z.N;
  k3_scatter<T, TOut><<<grid_for(n), 256, 0, s>>>(d.x, d.y, d.z, E, u, accum ? 1 : 0);
  return cudaGetLastError();
}

template <typename T, typename TOut>
cudaError_t launch3_prolong(const Dir3<T>& f, const Dir3<T>& c, const T* J, const T* uc, const T* in, TOut* out,
                            cudaStream_t s) {
  const int nf = f.x.p + 1, nc = c.x.p + 1;
  const size_t sm = sizeof(T) * (nc * nc * nc + nc * nc * nf + nc * nf * nf + nf * nc);
  cudaError_t e = allow_smem(k3_prolong<T, TOut>, sm);
  if (e != cudaSuccess) return e;
  k3_prolong<T, TOut><<<dim3(f.x.n, f.y.n, f.z.n), 256, sm, s>>>(f.x, f.y, f.z, c.x, c.y, c.z, J, uc, in, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch3_restrict(const Dir3<T>& f, const Dir3<T>& c, const T* J, const T* rf, T* Ec, T* fc,
                             cudaStream_t s) {
  const int nf = f.x.p + 1, nc = c.x.p + 1;
  const size_t sm = sizeof(T) * (nf * nf * nf + nf * nf * nc + nf * nc * nc + nf * nc);
  cudaError_t e = allow_smem(k3_restrict_elem<T>, sm);
  if (e != cudaSuccess) return e;
  k3_restrict_elem<T><<<dim3(f.x.n, f.y.n, f.z.n), 256, sm, s>>>(f.x, f.y, f.z, c.x, J, rf, Ec);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long n = (long)c.x.N * c.y.N * c.z.N;
  k3_restrict_gather<T><<<grid_for(n), 256, 0, s>>>(c.x, c.y, c.z, Ec, fc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch3_coarse(const Coarse3<T>& cv, T* w1, T* w2, T* f0, T* u0, cudaStream_t s) {
  const long n = (long)cv.nu[0] * cv.nu[1] * cv.nu[2];
  const int g = grid_for(n);
  k3_pack<T><<<g, 256, 0, s>>>(f0, w1, cv, 0);
  // forward: S^T along x, y, z, the division by the eigenvalue sums fused into the last
  k3_axis<T><<<g, 256, 0, s>>>(w1, w2, cv.S[0], cv, 0, 1, 0);
  k3_axis<T><<<g, 256, 0, s>>>(w2, w1, cv.S[1], cv, 1, 1, 0);
  k3_axis<T><<<g, 256, 0, s>>>(w1, w2, cv.S[2], cv, 2, 1, 1);
  // backward: S along z, y, x
  k3_axis<T><<<g, 256, 0, s>>>(w2, w1, cv.S[2], cv, 2, 0, 0);
  k3_axis<T><<<g, 256, 0, s>>>(w1, w2, cv.S[1], cv, 1, 0, 0);
  k3_axis<T><<<g, 256, 0, s>>>(w2, w1, cv.S[0], cv, 0, 0, 0);
  if (cv.singular) k3_sub_mean<T><<<1, 1024, 0, s>>>(w1, n);
  k3_pack<T><<<g, 256, 0, s>>>(u0, w1, cv, 1);
  return cudaGetLastError();
}

cudaError_t launch3_dot(const double* a, const double* b, long n, double* part, int* nparts, cudaStream_t s) {
  const int g = std::min(grid_for(n), kDot3Parts);
  k3_dot<<<g, 256, 0, s>>>(a, b, n, part);
  *nparts = g;
  return cudaGetLastError();
}

cudaError_t launch3_axpby(long n, double a, const double* x, double b, double* y, cudaStream_t s) {
  k3_axpby<<<grid_for(n), 256, 0, s>>>(n, a, x, b, y);
  return cudaGetLastError();
}

template <typename TA, typename TB>
cudaError_t launch3_convert(long n, const TA* a, TB* b, cudaStream_t s) {
  k3_convert<TA, TB><<<grid_for(n), 256, 0, s>>>(n, a, b);
  return cudaGetLastError();
}

#define INST3(T)                                                                                                     \
  template cudaError_t launch3_mass<T>(const Dir3<T>&, const T*, T*, cudaStream_t);                                \
  template size_t sweep3_smem_bytes<T>(int);                                                                        \
  template cudaError_t launch3_restrict<T>(const Dir3<T>&, const Dir3<T>&, const T*, const T*, T*, T*,             \
                                           cudaStream_t);                                                           \
  template cudaError_t launch3_coarse<T>(const Coarse3<T>&, T*, T*, T*, T*, cudaStream_t);
INST3(double)
INST3(float)
template cudaError_t launch3_apply<double, double>(const Dir3<double>&, const double*, const double*, double*,
                                                   cudaStream_t);
template cudaError_t launch3_apply<float, float>(const Dir3<float>&, const float*, const float*, float*, cudaStream_t);
template cudaError_t launch3_sweep<double, double>(const Dir3<double>&, const double*, double*, double*, bool,
                                                   cudaStream_t);
template cudaError_t launch3_sweep<float, float>(const Dir3<float>&, const float*, float*, float*, bool, cudaStream_t);
template cudaError_t launch3_sweep<float, double>(const Dir3<float>&, const float*, float*, double*, bool,
                                                  cudaStream_t);
template cudaError_t launch3_prolong<double, double>(const Dir3<double>&, const Dir3<double>&, const double*,
                                                     const double*, const double*, double*, cudaStream_t);
template cudaError_t launch3_prolong<float, float>(const Dir3<float>&, const Dir3<float>&, const float*, const float*,
                                                   const float*, float*, cudaStream_t);
template cudaError_t launch3_convert<double, float>(long, const double*, float*, cudaStream_t);
template cudaError_t launch3_convert<float, double>(long, const float*, double*, cudaStream_t);

}  // namespace sem
