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
#include "kernels.h"

namespace sem {

namespace {

template <int PF>
struct TT {
  static constexpr int PC = PF / 2;
  static constexpr int TE = (PF >= 32) ? 1 : 32 / PF;  // elements per tile per direction
  static constexpr int TNF = TE * PF;
  static constexpr int TNC = TE * PC;
  static constexpr int NPF = PF + 1, NPC = PC + 1;
};

// fc = I^T rf.  Fine nodes staged: [E0 pf - pf, E0 pf + TNF] per direction.
template <typename T, int PF>
__global__ void __launch_bounds__(256) k_restrict(DirView<T> fx, DirView<T> fy, DirView<T> cx, DirView<T> cy,
                                                  const T* __restrict__ J, const T* __restrict__ rf,
                                                  T* __restrict__ fc) {
  using Q = TT<PF>;
  constexpr int PC = Q::PC, TE = Q::TE, TNF = Q::TNF, TNC = Q::TNC, NPC = Q::NPC;
  constexpr int LN = TNF + PF + 1, LP = LN + 1, TP = TNC + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sr = reinterpret_cast<T*>(smem_raw);  // LN x LP fine residual
  T* st = sr + LN * LP;                     // LN x TP  x-contracted
  T* sJ = st + LN * TP;                     // NPF x NPC
  const int E0x = blockIdx.x * TE, E0y = blockIdx.y * TE;
  const int gx0 = E0x * PF - PF, gy0 = E0y * PF - PF;
  for (int idx = threadIdx.x; idx < LN * LN; idx += blockDim.x) {
    const int ly = idx / LN, lx = idx - ly * LN;
    const int gx = node_or_wall(gx0 + lx, fx.N, fx.periodic);
    const int gy = node_or_wall(gy0 + ly, fy.N, fy.periodic);
    sr[ly * LP + lx] = (gx >= 0 && gy >= 0) ? rf[(long)gy * fx.N + gx] : T(0);
  }
  for (int idx = threadIdx.x; idx < (PF + 1) * NPC; idx += blockDim.x) sJ[idx] = J[idx];
  __syncthreads();
  const bool lastx = E0x + TE >= cx.n, lasty = E0y + TE >= cy.n;
  const int ownx = min(TE, cx.n - E0x) * PC + ((!cx.periodic && lastx) ? 1 : 0);
  const int owny = min(TE, cy.n - E0y) * PC + ((!cy.periodic && lasty) ? 1 : 0);
  // x contraction for every staged fine row
  for (int idx = threadIdx.x; idx < LN * ownx; idx += blockDim.x) {
    const int ly = idx / ownx, ic = idx - ly * ownx;
    const int le = ic / PC, K = ic - le * PC;
    const T* row = sr + ly * LP + le * PF + PF;  // fine local node 0 of element E0x + le
    T t = T(0);
    if (le < TE) {
      if (K != 0) {
#pragma unroll
        for (int i = 1; i < PF; ++i) t += sJ[i * NPC + K] * row[i];
      } else {
#pragma unroll
        for (int i = 0; i < PF; ++i) t += sJ[i * NPC] * row[i];
#pragma unroll
        for (int i = 1; i < PF; ++i) t += sJ[i * NPC + PC] * row[i - PF];
      }
    }
    st[ly * TP + ic] = t;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < owny * ownx; idx += blockDim.x) {
    const int jc = idx / ownx, ic = idx - jc * ownx;
    const int gI = E0x * PC + ic, gJ = E0y * PC + jc;
    const bool wall = (!cx.periodic && (gI == 0 || gI == cx.N - 1)) || (!cy.periodic && (gJ == 0 || gJ == cy.N - 1));
    T v = T(0);
    if (!wall) {
      const int le = jc / PC, K = jc - le * PC;
      const T* col = st + (le * PF + PF) * TP + ic;
      if (K != 0) {
#pragma unroll
        for (int j = 1; j < PF; ++j) v += sJ[j * NPC + K] * col[j * TP];
      } else {
#pragma unroll
        for (int j = 0; j < PF; ++j) v += sJ[j * NPC] * col[j * TP];
#pragma unroll
        for (int j = 1; j < PF; ++j) v += sJ[j * NPC + PC] * col[(j - PF) * TP];
      }
    }
    fc[(long)gJ * cx.N + gI] = v;
  }
}

// out = in + I uc.  Coarse nodes staged: [E0 pc, E0 pc + TNC] per direction.
template <typename T, typename TOut, int PF>
__global__ void __launch_bounds__(256) k_prolong(DirView<T> fx, DirView<T> fy, DirView<T> cx, DirView<T> cy,
                                                 const T* __restrict__ J, const T* __restrict__ uc,
                                                 const T* in, TOut* out) {
  using Q = TT<PF>;
  constexpr int PC = Q::PC, TE = Q::TE, TNF = Q::TNF, TNC = Q::TNC, NPC = Q::NPC;
  constexpr int LC = TNC + 1, LCP = LC + 1, TP = TNF + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sc = reinterpret_cast<T*>(smem_raw);  // LC x LCP coarse values
  T* st = sc + LC * LCP;                    // LC x TP  x-interpolated
  T* sJ = st + LC * TP;
  const int E0x = blockIdx.x * TE, E0y = blockIdx.y * TE;
  for (int idx = threadIdx.x; idx < LC * LC; idx += blockDim.x) {
    const int ly = idx / LC, lx = idx - ly * LC;
    const int gx = node_or_wall(E0x * PC + lx, cx.N, cx.periodic);
    const int gy = node_or_wall(E0y * PC + ly, cy.N, cy.periodic);
    sc[ly * LCP + lx] = (gx >= 0 && gy >= 0) ? uc[(long)gy * cx.N + gx] : T(0);
  }
  for (int idx = threadIdx.x; idx < (PF + 1) * NPC; idx += blockDim.x) sJ[idx] = J[idx];
  __syncthreads();
  const bool lastx = E0x + TE >= fx.n, lasty = E0y + TE >= fy.n;
  const int ownx = min(TE, fx.n - E0x) * PF + ((!fx.periodic && lastx) ? 1 : 0);
  const int owny = min(TE, fy.n - E0y) * PF + ((!fy.periodic && lasty) ? 1 : 0);
  for (int idx = threadIdx.x; idx < LC * ownx; idx += blockDim.x) {
    const int ly = idx / ownx, ix = idx - ly * ownx;
    const int le = ix / PF, i = ix - le * PF;
    T t = T(0);
    if (le < TE) {
      const T* row = sc + ly * LCP + le * PC;
#pragma unroll
      for (int k = 0; k < NPC; ++k) t += sJ[i * NPC + k] * row[k];
    }
    st[ly * TP + ix] = t;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < owny * ownx; idx += blockDim.x) {
    const int jy = idx / ownx, ix = idx - jy * ownx;
    const int gi = E0x * PF + ix, gj = E0y * PF + jy;
    const long o = (long)gj * fx.N + gi;
    const bool wall = (!fx.periodic && (gi == 0 || gi == fx.N - 1)) || (!fy.periodic && (gj == 0 || gj == fy.N - 1));
    if (wall) {
      out[o] = TOut(0);
      continue;
    }
    const int le = jy / PF, j = jy - le * PF;
    const T* col = st + (le * PC) * TP + ix;
    T v = T(0);
#pragma unroll
    for (int k = 0; k < NPC; ++k) v += sJ[j * NPC + k] * col[k * TP];
    out[o] = in ? TOut(in[o] + v) : TOut(v);
  }
}

// Coarse step 1, one CTA per eigen-row a:
// T2[a][b] = (sum_j S_y[j][a] (F - mu)[j][.]) S_x[.][b] / (lam_y[a] + lam_x[b]).
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_a(CoarseView c, const T* __restrict__ f0) {
  __shared__ double srow[1024];
  __shared__ double sred[kRedThreads];
  const int a = blockIdx.x;
  double mu = 0.0;
  if (c.periodic) {
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < c.nux * c.nuy; idx += blockDim.x) {
      const int j = idx / c.nux, i = idx - j * c.nux;
      acc += (double)f0[(long)(c.firsty + j) * c.Nx + c.firstx + i];
    }
    mu = block_sum(acc, sred) / ((double)c.nux * c.nuy);
  }
  for (int i = threadIdx.x; i < c.nux; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < c.nuy; ++j)
      s += c.Sy[j * c.nuy + a] * ((double)f0[(long)(c.firsty + j) * c.Nx + c.firstx + i] - mu);
    srow[i] = s;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < c.nux; b += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < c.nux; ++i) s += srow[i] * c.Sx[i * c.nux + b];
    const bool null_pair = c.periodic && a == 0 && b == 0;
    c.T2[(long)a * c.nux + b] = null_pair ? 0.0 : s / (c.ly[a] + c.lx[b]);
  }
}

// Coarse step 2, one CTA per output row j: U[j][.] = (sum_a S_y[j][a] T2[a][.]) S_x^T,
// minus the mean of U for the periodic case.
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_b(CoarseView c, T* __restrict__ u0) {
  __shared__ double srow[1024];
  __shared__ double sred[kRedThreads];
  const int j = blockIdx.x;
  double mean = 0.0;
  if (c.periodic) {
    // mean(U) = (c_y^T T2 c_x) / N with c = S^T 1
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < c.nux * c.nuy; idx += blockDim.x) {
      const int a = idx / c.nux, b = idx - a * c.nux;
      acc += c.cy[a] * c.T2[idx] * c.cx[b];
    }
    mean = block_sum(acc, sred) / ((double)c.nux * c.nuy);
  }
  for (int b = threadIdx.x; b < c.nux; b += blockDim.x) {
    double s = 0.0;
    for (int a = 0; a < c.nuy; ++a) s += c.Sy[j * c.nuy + a] * c.T2[(long)a * c.nux + b];
    srow[b] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < c.nux; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < c.nux; ++b) s += srow[b] * c.Sx[i * c.nux + b];
    u0[(long)(c.firsty + j) * c.Nx + c.firstx + i] = T(s - mean);
  }
}

template <typename T, int PF>
cudaError_t restrict_p(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx, const DirView<T>& cy,
                       const T* J, const T* rf, T* fc, cudaStream_t s) {
  using Q = TT<PF>;
  constexpr int LN = Q::TNF + PF + 1;
  const size_t sm = sizeof(T) * (LN * (LN + 1) + LN * (Q::TNC + 2) + (PF + 1) * Q::NPC);
  cudaError_t e = allow_smem(k_restrict<T, PF>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((cx.n + Q::TE - 1) / Q::TE, (cy.n + Q::TE - 1) / Q::TE);
  k_restrict<T, PF><<<grid, 256, sm, s>>>(fx, fy, cx, cy, J, rf, fc);
  return cudaGetLastError();
}

template <typename T, typename TOut, int PF>
cudaError_t prolong_p(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx, const DirView<T>& cy,
                      const T* J, const T* uc, const T* in, TOut* out, cudaStream_t s) {
  using Q = TT<PF>;
  constexpr int LC = Q::TNC + 1;
  const size_t sm = sizeof(T) * (LC * (LC + 1) + LC * (Q::TNF + 2) + (PF + 1) * Q::NPC);
  cudaError_t e = allow_smem(k_prolong<T, TOut, PF>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((fx.n + Q::TE - 1) / Q::TE, (fy.n + Q::TE - 1) / Q::TE);
  k_prolong<T, TOut, PF><<<grid, 256, sm, s>>>(fx, fy, cx, cy, J, uc, in, out);
  return cudaGetLastError();
}

}  // namespace

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

template <typename T>
cudaError_t launch_coarse(const CoarseView& c, const T* f0, T* u0, cudaStream_t s) {
  if (c.nux > 1024 || c.nuy > 65535) return cudaErrorInvalidValue;
  k_coarse_a<T><<<c.nuy, 256, 0, s>>>(c, f0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_coarse_b<T><<<c.nuy, 256, 0, s>>>(c, u0);
  return cudaGetLastError();
}

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
