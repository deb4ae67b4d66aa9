// Sum-factorised SEM Laplacian, Eq. (system matrix): A = M_y (x) L_x + L_y (x) M_x.
//
// Node-centric form: for node (j, i) of the global grid
//   (A u)_{ji} = Mg_y[j] * sum_k Lg_x[i, k] u_{jk} + Mg_x[i] * sum_k Lg_y[j, k] u_{ki}
// where the assembled 1D stiffness row Lg[i, .] is the element row of the
// element holding i, plus the last row of the left neighbour when i sits on an
// element interface.  A CTA owns a tile of TE x TE elements (32 x 32 nodes,
// 16 x 16 at P <= 4), stages the tile plus one element of halo on the low side
// in shared memory, and writes every owned node exactly once: no atomics,
// deterministic.
#include <algorithm>
#include <type_traits>

#include "kernels.h"
#include "level_ops.cuh"

namespace sem {

namespace {

template <typename T, typename TF, int P>
__global__ void __launch_bounds__(256) k_apply(DirView<T> dx, DirView<T> dy, const T* __restrict__ u,
                                               const TF* __restrict__ f, T* __restrict__ out, int dot,
                                               double* __restrict__ part, const T* __restrict__ E,
                                               T* __restrict__ uout, PcgFuse pf) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  apply_tile<T, TF, P>(dx, dy, u, f, out, dot, part, E, uout, pf, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y,
                       smem_raw);
}

// Even-odd variant of the same operator.  The 1D element stiffness of GLL
// collocation is centro-symmetric, L[p-a][p-b] = L[a][b] (D[p-i][p-j] = -D[i][j]
// and w_{p-q} = w_q), so the element-row product y = L x splits into
//   e_k = x_k + x_{p-k},  o_k = x_k - x_{p-k}   (k < p/2),  e_{p/2} = x_{p/2}
//   ye_a = sum_{k<=p/2} E[a][k] e_k,  yo_a = sum_{k<p/2} O[a][k] o_k
//   y_a = ye_a + yo_a,  y_{p-a} = ye_a - yo_a
// with E[a][k] = (L[a][k] + L[a][p-k]) / 2 (E[a][p/2] = L[a][p/2]) and
// O[a][k] = (L[a][k] - L[a][p-k]) / 2: (p/2+1)^2 + (p/2)^2 FMAs per element
// row instead of (p+1)^2.  This halves the work of the FP64 operator, which is
// bound by the FP64 pipe on GB300.  Phases per CTA: build E/O of the tile's
// elements; x-products of every owned row (one thread per (a, row), rows
// across the warp so E/O are broadcast); y-products of every owned column;
// combine with the mass diagonals.
template <int P>
struct EOTile {
  static constexpr int H = P / 2;
  static constexpr int TE = Tile<P>::TE, TN = Tile<P>::TN, LN = Tile<P>::LN, NP = P + 1;
  static constexpr int LP = LN | 1;                         // odd pitch: conflict-free column reads
  static constexpr int NE = (H + 1) * (H + 1), NO = H * H;  // E and O table sizes
  static constexpr int EO = NE + NO;
  static constexpr int NV = 2 * H + 1;                      // e_0..e_H, o_0..o_{H-1} per element row
};

template <typename T, int P>
size_t apply_eo_smem() {
  using Q = EOTile<P>;
  const size_t t = (size_t)Q::LN * Q::LP                     // staged u
                   + 2 * (Q::TE + 1) * Q::EO                  // E/O per element, x and y
                   + (size_t)(Q::TE + 1) * Q::NV * Q::TN      // e/o vectors of one direction
                   + (size_t)Q::TN * (Q::TE + 1) * Q::NP      // x products (y products reuse the staged tile)
                   + 2 * (Q::TN + 1);                        // mass diagonals
  return sizeof(T) * t + sizeof(double) * kRedThreads;
}

// e/o vectors of one direction: ev[(slot * NV + k) * TN + lane-index], formed
// once per element row (x) or column (y) and shared by all its outputs
template <typename T, int P, bool XDIR>
__device__ __forceinline__ void form_eo(const T* su, T* ev) {
  using Q = EOTile<P>;
  constexpr int H = Q::H, TE = Q::TE, TN = Q::TN, LP = Q::LP, NV = Q::NV;
  for (int idx = threadIdx.x; idx < (TE + 1) * H * TN; idx += blockDim.x) {
    const int w = idx % TN;                 // owned row (x) or column (y)
    const int q = idx / TN;
    const int sl = q / H, k = q - sl * H;
    T xk, xm;
    if (XDIR) {
      const T* x = su + (w + P) * LP + sl * P;
      xk = x[k];
      xm = x[P - k];
    } else {
      const T* x = su + (sl * P) * LP + w + P;
      xk = x[k * LP];
      xm = x[(P - k) * LP];
    }
    ev[(sl * NV + k) * TN + w] = xk + xm;
    ev[(sl * NV + H + 1 + k) * TN + w] = xk - xm;
  }
  for (int idx = threadIdx.x; idx < (TE + 1) * TN; idx += blockDim.x) {
    const int w = idx % TN, sl = idx / TN;
    ev[(sl * NV + H) * TN + w] = XDIR ? su[(w + P) * LP + sl * P + H] : su[(sl * P + H) * LP + w + P];
  }
}

// element-local products of one direction from the e/o vectors; item (slot, a, w):
// slot 0 (low-side neighbour) needs only a = 0 (its y_P)
template <typename T, int P, bool XDIR>
__device__ __forceinline__ void eo_products(const T* eo, const T* ev, T* dst_base) {
  using Q = EOTile<P>;
  constexpr int H = Q::H, TE = Q::TE, TN = Q::TN, NP = Q::NP, EO = Q::EO, NE = Q::NE, NV = Q::NV;
  constexpr int XI = TN * (1 + TE * (H + 1));
  for (int idx = threadIdx.x; idx < XI; idx += blockDim.x) {
    const int w = idx % TN;
    const int q = idx / TN;
    const int sl = q == 0 ? 0 : 1 + (q - 1) / (H + 1);
    const int a = q == 0 ? 0 : (q - 1) % (H + 1);
    const T* E = eo + sl * EO + a * (H + 1);
    const T* O = eo + sl * EO + NE + min(a, H - 1) * H;  // row H of O is zero and not stored
    const T* e = ev + (sl * NV) * TN + w;
    const T* o = ev + (sl * NV + H + 1) * TN + w;
    T ye = T(0), yo = T(0);
#pragma unroll
    for (int k = 0; k <= H; ++k) ye += E[k] * e[k * TN];
    if (a < H) {  // the odd part of the middle row is zero (a is uniform across a warp: w = lane)
#pragma unroll
      for (int k = 0; k < H; ++k) yo += O[k] * o[k * TN];
    }
    if (XDIR) {
      T* dst = dst_base + (w * (TE + 1) + sl) * NP;  // [row][slot][a]
      if (a < H) dst[P - a] = ye - yo;
      dst[a] = ye + yo;
    } else {
      T* dst = dst_base + (sl * NP) * TN + w;         // [slot][b][col]
      if (a < H) dst[(P - a) * TN] = ye - yo;
      dst[a * TN] = ye + yo;
    }
  }
}

template <typename T, typename TF, int P>
__global__ void __launch_bounds__(256) k_apply_eo(DirView<T> dx, DirView<T> dy, const T* __restrict__ u,
                                                  const TF* __restrict__ f, T* __restrict__ out, int dot,
                                                  double* __restrict__ part, const T* __restrict__ E,
                                                  T* __restrict__ uout, PcgFuse pf) {
  pdl_enter();
  using Q = EOTile<P>;
  constexpr int H = Q::H, TE = Q::TE, TN = Q::TN, LN = Q::LN, LP = Q::LP, NP = Q::NP, EO = Q::EO, NE = Q::NE,
                NV = Q::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);   // LN x LP
  T* eox = su + LN * LP;                      // (TE+1) x EO
  T* eoy = eox + (TE + 1) * EO;
  T* ev = eoy + (TE + 1) * EO;                // (TE+1) x NV x TN, reused by x then y
  T* xb = ev + (TE + 1) * NV * TN;            // [row][slot][a]  x-products
  T* yb = su;                                 // [slot][b][col]  y-products, over the staged tile once
                                              // the y e/o vectors are formed
  static_assert(TN * (TE + 1) * NP <= LN * LP, "y products must fit in the staged tile");
  T* sMx = xb + TN * (TE + 1) * NP;
  T* sMy = sMx + (TN + 1);
  double* sred = reinterpret_cast<double*>(sMy + (TN + 1));

  const int ex0 = blockIdx.x * TE, ey0 = blockIdx.y * TE;
  const int Nx = dx.N, Ny = dy.N;
  const int gx0 = ex0 * P - P, gy0 = ey0 * P - P;
  const double beta = fused_beta(pf, blockIdx.y, gridDim.y);
  for (int idx = threadIdx.x; idx < LN * LN; idx += blockDim.x) {
    const int ly = idx / LN, lx = idx - ly * LN;
    const int gx = node_or_wall(gx0 + lx, Nx, dx.periodic, dx.segN);
    const int gy = node_or_wall(gy0 + ly, Ny, dy.periodic, dy.segN);
    su[ly * LP + lx] = stage_value<P>(u, E, dx, dy, pf, beta, gy, gx);
  }
  // E/O tables of slot s = element ex0 + s - 1 (slot 0: low-side neighbour)
  for (int idx = threadIdx.x; idx < 2 * (TE + 1) * EO; idx += blockDim.x) {
    const int dir = idx / ((TE + 1) * EO);
    const int rem = idx - dir * (TE + 1) * EO;
    const int sl = rem / EO, t = rem - sl * EO;
    const DirView<T>& d = dir ? dy : dx;
    int e = (dir ? ey0 : ex0) + sl - 1;
    if (d.periodic) e = (e + d.n) % d.n;
    T v = T(0);
    if (e >= 0 && e < d.n) {
      const T* L = d.Le + (long)e * NP * NP;
      if (t < NE) {
        const int a = t / (H + 1), k = t - a * (H + 1);
        v = (k == H) ? L[a * NP + H] : T(0.5) * (L[a * NP + k] + L[a * NP + P - k]);
      } else {
        const int a = (t - NE) / H, k = (t - NE) - a * H;
        v = T(0.5) * (L[a * NP + k] - L[a * NP + P - k]);
      }
    }
    (dir ? eoy : eox)[sl * EO + t] = v;
  }
  for (int idx = threadIdx.x; idx <= TN; idx += blockDim.x) {
    const int gx = ex0 * P + idx, gy = ey0 * P + idx;
    sMx[idx] = gx < Nx ? dx.Mg[gx] : T(0);
    sMy[idx] = gy < Ny ? dy.Mg[gy] : T(0);
  }
  __syncthreads();
  const bool lastx = ex0 + TE >= dx.n, lasty = ey0 + TE >= dy.n;
  const int ownx = min(TE, dx.n - ex0) * P + ((!dx.periodic && lastx) ? 1 : 0);
  const int owny = min(TE, dy.n - ey0) * P + ((!dy.periodic && lasty) ? 1 : 0);
  // staged values of this thread's owned nodes, kept for the dot product and
  // the assembled-correction output (the y products overwrite the tile)
  constexpr int KOWN = ((TN + 1) * (TN + 1) + 255) / 256;
  T own[KOWN];
#pragma unroll
  for (int q = 0; q < KOWN; ++q) {
    const int idx = threadIdx.x + 256 * q;
    own[q] = T(0);
    if (idx < ownx * owny) {
      const int jy = idx / ownx, ix = idx - jy * ownx;
      own[q] = su[(jy + P) * LP + ix + P];
    }
  }
  form_eo<T, P, true>(su, ev);
  __syncthreads();
  eo_products<T, P, true>(eox, ev, xb);
  __syncthreads();
  form_eo<T, P, false>(su, ev);
  __syncthreads();
  eo_products<T, P, false>(eoy, ev, yb);
  __syncthreads();

  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < KOWN; ++q) {
    const int idx = threadIdx.x + 256 * q;
    if (idx >= ownx * owny) break;
    const int jy = idx / ownx, ix = idx - jy * ownx;
    const int gi = ex0 * P + ix, gj = ey0 * P + jy;
    const long o = (long)gj * Nx + gi;
    const bool wall = wall_node(gi, Nx, dx.periodic, dx.segN) || wall_node(gj, Ny, dy.periodic, dy.segN);
    T val = T(0);
    if (!wall) {
      const int lex = ix / P, a = ix - lex * P;
      const int ley = jy / P, b = jy - ley * P;
      const T* xr = xb + (jy * (TE + 1) + lex + 1) * NP;
      T xs = xr[a];
      if (a == 0) xs += xr[P - NP];  // y_P of the left slot
      const T* yc = yb + ((ley + 1) * NP) * TN + ix;
      T ys = yc[b * TN];
      if (b == 0) ys += yc[(P - NP) * TN];
      val = sMy[jy] * xs + sMx[ix] * ys;
      if (f) val = convert_to<T>(f[o]) - val;
    }
    out[o] = val;
    if (uout) uout[o] = wall ? T(0) : own[q];
    if (dot == 1) acc += (double)own[q] * (double)val;
    else if (dot == 2) acc += (double)val * (double)val;
  }
  if (dot) {
    const double s = block_sum_w0(acc, sred);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// ---- variable diffusivity B(nu), Sec. 4.3, Eq. (diffusion) -------------------
// Element-local weak form with GLL quadrature (U: element coefficients, rows
// j = y, columns i = x, D the differentiation matrix):
//   ux = U D^T,  uy = D U,  V = (G_x .* ux) D + D^T (G_y .* uy)
// one CTA per element; V goes to the element-blocked scratch E, and a node
// gather then sums the (at most 2 x 2) element contributions of every node.
template <typename T, int P>
__global__ void __launch_bounds__(256) k_var_local(DirView<T> dx, DirView<T> dy, VarView<T> v,
                                                   const T* __restrict__ u) {
  pdl_enter();
  constexpr int NP = P + 1, NN = NP * NP;
  __shared__ T sU[NN], sD[NN], sA[NN], sB[NN];
  const int ex = blockIdx.x, ey = blockIdx.y;
  const long e = (long)ey * dx.n + ex;
  for (int idx = threadIdx.x; idx < NN; idx += blockDim.x) {
    const int j = idx / NP, i = idx - j * NP;
    const int gx = node_or_wall(ex * P + i, dx.N, dx.periodic, dx.segN);
    const int gy = node_or_wall(ey * P + j, dy.N, dy.periodic, dy.segN);
    sU[idx] = (gx >= 0 && gy >= 0) ? u[(long)gy * dx.N + gx] : T(0);
    sD[idx] = v.D[idx];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NN; idx += blockDim.x) {
    const int j = idx / NP, i = idx - j * NP;
    T ax = T(0), ay = T(0);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      ax += sD[i * NP + k] * sU[j * NP + k];
      ay += sD[j * NP + k] * sU[k * NP + i];
    }
    sA[idx] = v.Gx[e * NN + idx] * ax;
    sB[idx] = v.Gy[e * NN + idx] * ay;
  }
  __syncthreads();
  T* Es = v.E + e * NN;
  for (int idx = threadIdx.x; idx < NN; idx += blockDim.x) {
    const int j = idx / NP, a = idx - j * NP;
    T s = T(0);
#pragma unroll
    for (int q = 0; q < NP; ++q) s += sA[j * NP + q] * sD[q * NP + a] + sD[q * NP + j] * sB[q * NP + a];
    Es[idx] = s;
  }
}

// out = (f ? f - sum : sum) over the elements that hold each node
template <typename T>
__global__ void __launch_bounds__(256) k_var_gather(DirView<T> dx, DirView<T> dy, const T* __restrict__ E,
                                                    const T* __restrict__ u, const T* __restrict__ f,
                                                    T* __restrict__ out, int dot, double* __restrict__ part) {
  pdl_enter();
  __shared__ double sred[kRedThreads];
  const int p = dx.p, np1 = p + 1, nn = np1 * np1;
  const long n = (long)dx.N * dy.N;
  double acc = 0.0;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int gj = (int)(idx / dx.N), gi = (int)(idx - (long)gj * dx.N);
    const bool wall = wall_node(gi, dx.N, dx.periodic, dx.segN) || wall_node(gj, dy.N, dy.periodic, dy.segN);
    T val = T(0);
    if (!wall) {
      T s = T(0);
      const int ey_hi = gj / p, ex_hi = gi / p;
      for (int eyu = (gj % p == 0 ? ey_hi - 1 : ey_hi); eyu <= ey_hi; ++eyu) {
        int ey = eyu;
        if (dy.periodic) ey = ((ey % dy.n) + dy.n) % dy.n;
        else if (ey < 0 || ey >= dy.n) continue;
        const int b = gj - eyu * p;
        for (int exu = (gi % p == 0 ? ex_hi - 1 : ex_hi); exu <= ex_hi; ++exu) {
          int ex = exu;
          if (dx.periodic) ex = ((ex % dx.n) + dx.n) % dx.n;
          else if (ex < 0 || ex >= dx.n) continue;
          const int a = gi - exu * p;
          s += E[(long)(ey * dx.n + ex) * nn + b * np1 + a];
        }
      }
      val = f ? f[idx] - s : s;
    }
    out[idx] = val;
    if (dot == 1) acc += (double)u[idx] * (double)val;
    else if (dot == 2) acc += (double)val * (double)val;
  }
  if (dot) {
    const double sm = block_sum(acc, sred);
    if (threadIdx.x == 0) part[blockIdx.x] = sm;
  }
}

template <typename T, int P>
cudaError_t var_p(const DirView<T>& dx, const DirView<T>& dy, const VarView<T>& v, const T* u, cudaStream_t s) {
  dim3 grid(dx.n, dy.n);
  {
    const cudaError_t e_ = launch_pdl(k_var_local<T, P>, dim3(grid), dim3(256), 0, s, dx, dy, v, u);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_mass(DirView<double> dx, DirView<double> dy, const double* __restrict__ f,
                                               double* __restrict__ b, double* __restrict__ part) {
  pdl_enter();
  __shared__ double sred[kRedThreads];
  const long n = (long)dx.N * dy.N;
  double acc = 0.0;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int gj = (int)(idx / dx.N), gi = (int)(idx - (long)gj * dx.N);
    const bool wall = wall_node(gi, dx.N, dx.periodic, dx.segN) || wall_node(gj, dy.N, dy.periodic, dy.segN);
    const double v = wall ? 0.0 : dy.Mg[gj] * dx.Mg[gi] * f[idx];
    b[idx] = v;
    acc += v;
  }
  const double s = block_sum(acc, sred);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T, typename TF, int P>
cudaError_t apply_p(const DirView<T>& dx, const DirView<T>& dy, const T* u, const TF* f, T* out, int dot,
                    double* part, int* nparts, cudaStream_t s, const T* E, T* uout, const PcgFuse& pf, int eo) {
  using Tl = Tile<P>;
  dim3 grid((dx.n + Tl::TE - 1) / Tl::TE, (dy.n + Tl::TE - 1) / Tl::TE);
  if (dot && (int)(grid.x * grid.y) > kMaxPartials) return cudaErrorInvalidConfiguration;
  if (nparts) *nparts = grid.x * grid.y;
  // the even-odd form for P >= 4: always in FP64 (the FP64 pipe bounds it),
  // on request in FP32 (eo = 1; the autotuner decides)
  if constexpr (P >= 4) {  // below P = 4 the plain form only
    if (eo == 1 || (eo < 0 && std::is_same<T, double>::value)) {
      const size_t sm = apply_eo_smem<T, P>();
      cudaError_t e = allow_smem(k_apply_eo<T, TF, P>, sm);
      if (e != cudaSuccess) return e;
      return launch_pdl(k_apply_eo<T, TF, P>, dim3(grid), dim3(256), sm, s, dx, dy, u, f, out, dot, part, E, uout,
                        pf);
    }
  }
  const size_t sm = apply_smem<T, P>();
  cudaError_t e = allow_smem(k_apply<T, TF, P>, sm);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_apply<T, TF, P>, dim3(grid), dim3(256), sm, s, dx, dy, u, f, out, dot, part, E, uout, pf);
}

}  // namespace

template <typename T, typename TF>
cudaError_t launch_apply(const DirView<T>& dx, const DirView<T>& dy, const T* u, const TF* f, T* out, int dot,
                         double* part, int* nparts, cudaStream_t s, const T* E, T* uout, PcgFuse pf, int eo) {
  if (pf.z && !std::is_same<T, double>::value) return cudaErrorInvalidValue;
  switch (dx.p) {
    case 1: return apply_p<T, TF, 1>(dx, dy, u, f, out, dot, part, nparts, s, E, uout, pf, eo);
    case 2: return apply_p<T, TF, 2>(dx, dy, u, f, out, dot, part, nparts, s, E, uout, pf, eo);
    case 4: return apply_p<T, TF, 4>(dx, dy, u, f, out, dot, part, nparts, s, E, uout, pf, eo);
    case 8: return apply_p<T, TF, 8>(dx, dy, u, f, out, dot, part, nparts, s, E, uout, pf, eo);
    case 16: return apply_p<T, TF, 16>(dx, dy, u, f, out, dot, part, nparts, s, E, uout, pf, eo);
    case 32: return apply_p<T, TF, 32>(dx, dy, u, f, out, dot, part, nparts, s, E, uout, pf, eo);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_apply_var(const DirView<T>& dx, const DirView<T>& dy, const VarView<T>& v, const T* u, const T* f,
                             T* out, int dot, double* part, int* nparts, cudaStream_t s) {
  cudaError_t e;
  switch (dx.p) {
    case 2: e = var_p<T, 2>(dx, dy, v, u, s); break;
    case 4: e = var_p<T, 4>(dx, dy, v, u, s); break;
    case 8: e = var_p<T, 8>(dx, dy, v, u, s); break;
    case 16: e = var_p<T, 16>(dx, dy, v, u, s); break;
    case 32: e = var_p<T, 32>(dx, dy, v, u, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  const long n = (long)dx.N * dy.N;
  const int grid = (int)std::max<long>(1, std::min<long>((n + 255) / 256, 4 * 152));
  if (nparts) *nparts = grid;
  {
    const cudaError_t e_ = launch_pdl(k_var_gather<T>, dim3(grid), dim3(256), 0, s, dx, dy, v.E, u, f, out, dot, part);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

template cudaError_t launch_apply_var<double>(const DirView<double>&, const DirView<double>&, const VarView<double>&,
                                              const double*, const double*, double*, int, double*, int*,
                                              cudaStream_t);
template cudaError_t launch_apply_var<float>(const DirView<float>&, const DirView<float>&, const VarView<float>&,
                                             const float*, const float*, float*, int, double*, int*, cudaStream_t);

template cudaError_t launch_apply<double, double>(const DirView<double>&, const DirView<double>&, const double*,
                                                  const double*, double*, int, double*, int*, cudaStream_t,
                                                  const double*, double*, PcgFuse, int);
template cudaError_t launch_apply<float, float>(const DirView<float>&, const DirView<float>&, const float*,
                                                const float*, float*, int, double*, int*, cudaStream_t, const float*,
                                                float*, PcgFuse, int);
template cudaError_t launch_apply<float, double>(const DirView<float>&, const DirView<float>&, const float*,
                                                 const double*, float*, int, double*, int*, cudaStream_t,
                                                 const float*, float*, PcgFuse, int);

cudaError_t launch_mass(const DirView<double>& dx, const DirView<double>& dy, const double* f, double* b,
                        double* part, int* nparts, cudaStream_t s) {
  const int grid = 256;
  if (nparts) *nparts = grid;
  {
    const cudaError_t e_ = launch_pdl(k_mass, dim3(grid), dim3(kRedThreads), 0, s, dx, dy, f, b, part);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

}  // namespace sem
