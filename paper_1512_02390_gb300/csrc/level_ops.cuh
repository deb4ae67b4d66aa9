// Bodies of the level operations of the V-cycle, one tile or one subdomain at
// a time, shared by the one-kernel-per-step launches (k_operator.cu,
// k_transfer.cu, k_schwarz.cu) and the persistent low-level cycle
// (k_lowcycle.cu): the node-centric residual of Eq. (system matrix), the grid
// transfers of Sec. 3.2 and the tensor-core (mma.sync) fast-diagonalisation
// sweep of Alg. 2 / Eq. (FDM).
#pragma once

#include <cstdint>
#include <type_traits>

#include "f32_round.h"
#include "kernels.h"

namespace sem {

// ---- level residual (operator) ------------------------------------------------
template <int P>
struct Tile {
  static constexpr int TE = tile_elems(P);           // elements per direction
  static constexpr int TN = TE * P;                  // owned nodes per direction
  static constexpr int LN = TN + P + 1;              // staged nodes per direction
  static constexpr int LP = LN + 1;                  // padded row pitch
  static constexpr int NP = P + 1;
};

// beta of this tile's problem for the fused MGCG direction (0 when unused)
__device__ __forceinline__ double fused_beta(const PcgFuse& pf, int by, int gyd) {
  if (!pf.z) return 0.0;
  const int k = by / (gyd / pf.nb);
  return pf.flags[2 * k] ? 0.0 : pf.beta[(long)k * pf.stride + pf.iter[1]];
}

// staged operand at node (gy, gx) (-1: wall, 0): u, the assembled Schwarz
// correction (E), or the MGCG direction z + beta p
template <int P, typename T>
__device__ __forceinline__ T stage_value(const T* __restrict__ u, const T* __restrict__ E, const DirView<T>& dx,
                                         const DirView<T>& dy, const PcgFuse& pf, double beta, int gy, int gx) {
  if (gx < 0 || gy < 0) return T(0);
  if (E) return window_sum_p<P>(dx, dy, E, gy, gx);
  const long o = (long)gy * dx.N + gx;
  if (pf.z) return T(fma(beta, (double)u[o], pf.z[o]));
  return u[o];
}

// per staged column (and row): its node (-1: wall) and the up to 3 windows
// holding it (count, E offset of the column / row)
template <int P>
struct StageTab {
  static constexpr int LN = Tile<P>::LN;
  static constexpr size_t BYTES = 2 * LN * (sizeof(long) * 3 + sizeof(int) * 2);
};

template <typename T, int P>
size_t apply_smem() {
  using Tl = Tile<P>;
  // + 16: the double / long tables start on a 16-byte boundary
  return sizeof(T) * (Tl::LN * Tl::LP + 2 * (Tl::TE + 1) * Tl::NP * Tl::NP + 2 * (Tl::TN + 1) +
                      (Tl::TN + 1) * Tl::TE) +
         16 + sizeof(double) * kRedThreads + StageTab<P>::BYTES;
}

// One tile (bx, by) of a (gxd x gyd) tile grid; smem: apply_smem<T, P>() bytes.
template <typename T, typename TF, int P>
__device__ __forceinline__ void apply_tile(const DirView<T>& dx, const DirView<T>& dy, const T* __restrict__ u,
                                           const TF* __restrict__ f, T* __restrict__ out, int dot,
                                           double* __restrict__ part, const T* __restrict__ E,
                                           T* __restrict__ uout, const PcgFuse& pf, int bx, int by, int gxd, int gyd,
                                           unsigned char* smem_raw) {
  using Tl = Tile<P>;
  constexpr int TE = Tl::TE, TN = Tl::TN, LN = Tl::LN, LP = Tl::LP, NP = Tl::NP;
  T* su = reinterpret_cast<T*>(smem_raw);          // LN x LP staged u
  T* sLx = su + LN * LP;                           // (TE+1) x NP x NP
  T* sLy = sLx + (TE + 1) * NP * NP;
  T* sMx = sLy + (TE + 1) * NP * NP;               // TN + 1
  T* sMy = sMx + (TN + 1);
  T* sbx = sMy + (TN + 1);                                    // [(TN + 1) x TE] left-edge x sums
  // the double / long tables start at the next 16-byte boundary; the offset
  // is a constant, so the pointers stay derived from the shared array and
  // their loads are shared-memory loads
  constexpr size_t kTabOff =
      (sizeof(T) * (LN * LP + 2 * (TE + 1) * NP * NP + 2 * (TN + 1) + (TN + 1) * TE) + 15) / 16 * 16;
  double* sred = reinterpret_cast<double*>(smem_raw + kTabOff);
  long* woff = reinterpret_cast<long*>(sred + kRedThreads);  // [2 LN][3] E offsets (columns, then rows)
  int* gnode = reinterpret_cast<int*>(woff + 2 * 3 * LN);    // [2 LN] node or -1
  int* wcnt = gnode + 2 * LN;                                // [2 LN] windows holding it

  const int ex0 = bx * TE, ey0 = by * TE;
  const int Nx = dx.N, Ny = dy.N;
  const int gx0 = ex0 * P - P, gy0 = ey0 * P - P;
  const double beta = fused_beta(pf, by, gyd);

  // staged columns and rows: node or wall, and for the assembled correction
  // the windows of Eq. (correction:global) that hold the node, in ascending
  // element order (node g = e P + j lies in the windows of e - 1 when
  // j <= n_o, of e, and of e + 1 when j >= P - n_o; index (e - e') P + j + n_o)
  for (int i = threadIdx.x; i < 2 * LN; i += blockDim.x) {
    const bool is_row = i >= LN;
    const DirView<T>& d = is_row ? dy : dx;
    const int g = node_or_wall((is_row ? gy0 - LN : gx0) + i, d.N, d.periodic, d.segN);
    gnode[i] = g;
    int n = 0;
    if (E && g >= 0) {
      const int no = dx.n_o, m = P + 1 + 2 * no;
      const long mm = (long)m * m;
      const int e = g / P, j = g - e * P;
#pragma unroll
      for (int dd = -1; dd <= 1; ++dd) {
        if ((dd < 0 && j > no) || (dd > 0 && j < P - no)) continue;
        int ee = e + dd;
        if (d.periodic) ee = ee < 0 ? ee + d.n : (ee >= d.n ? ee - d.n : ee);
        else if (ee < 0 || ee >= d.n) continue;
        const int b = j - dd * P + no;
        woff[i * 3 + n] = is_row ? (long)ee * dx.n * mm + (long)b * m : (long)ee * mm + b;
        ++n;
      }
    }
    wcnt[i] = n;
  }
  __syncthreads();
  if (E && 2 * dx.n_o < P) {
    // at most two windows per direction hold a node: the loads of SB staged
    // nodes (up to 4 windows each) are issued before any is summed, so one
    // memory latency covers them; each node sums its windows in the order
    // of the general loop below
    constexpr int SB = 2;
    for (int i0 = threadIdx.x; i0 < LN * LN; i0 += SB * blockDim.x) {
      T w[SB][4];
      int nyq[SB], nxq[SB];
#pragma unroll
      for (int q = 0; q < SB; ++q) {
        const int idx = i0 + q * blockDim.x;
        const int ly = idx / LN, lx = idx - ly * LN;
        const bool in = idx < LN * LN && gnode[lx] >= 0 && gnode[LN + ly] >= 0;
        nyq[q] = in ? wcnt[LN + ly] : 0;
        nxq[q] = in ? wcnt[lx] : 0;
#pragma unroll
        for (int iy = 0; iy < 2; ++iy)
#pragma unroll
          for (int ix = 0; ix < 2; ++ix)
            w[q][iy * 2 + ix] =
                (iy < nyq[q] && ix < nxq[q]) ? E[woff[(LN + ly) * 3 + iy] + woff[lx * 3 + ix]] : T(0);
      }
#pragma unroll
      for (int q = 0; q < SB; ++q) {
        const int idx = i0 + q * blockDim.x;
        if (idx >= LN * LN) break;
        const int ly = idx / LN, lx = idx - ly * LN;
        T v = T(0);
#pragma unroll
        for (int iy = 0; iy < 2; ++iy)
#pragma unroll
          for (int ix = 0; ix < 2; ++ix)
            if (iy < nyq[q] && ix < nxq[q]) v += w[q][iy * 2 + ix];
        su[ly * LP + lx] = v;
      }
    }
  } else {
  for (int idx = threadIdx.x; idx < LN * LN; idx += blockDim.x) {
    const int ly = idx / LN, lx = idx - ly * LN;
    const int gx = gnode[lx], gy = gnode[LN + ly];
    T v = T(0);
    if (gx >= 0 && gy >= 0) {
      if (E) {
        const int ny = wcnt[LN + ly], nx = wcnt[lx];
        for (int iy = 0; iy < ny; ++iy) {
          const T* Er = E + woff[(LN + ly) * 3 + iy];
          for (int ix = 0; ix < nx; ++ix) v += Er[woff[lx * 3 + ix]];
        }
      } else {
        v = stage_value<P>(u, E, dx, dy, pf, beta, gy, gx);  // E is null here
      }
    }
    su[ly * LP + lx] = v;
  }
  }
  // element stiffness of the tile and of its low-side neighbour (slot 0)
  for (int idx = threadIdx.x; idx < (TE + 1) * NP * NP; idx += blockDim.x) {
    const int le = idx / (NP * NP), ab = idx - le * NP * NP;
    int exx = ex0 + le - 1, eyy = ey0 + le - 1;
    if (dx.periodic) exx = (exx + dx.n) % dx.n;
    if (dy.periodic) eyy = (eyy + dy.n) % dy.n;
    sLx[idx] = (exx >= 0 && exx < dx.n) ? dx.Le[(long)exx * NP * NP + ab] : T(0);
    sLy[idx] = (eyy >= 0 && eyy < dy.n) ? dy.Le[(long)eyy * NP * NP + ab] : T(0);
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
  // x part of a node on an element's left edge (a = 0) from the element on
  // its left (that element's last stiffness row), one thread per (row,
  // element): in the node loop only two lanes of a warp need it, and the
  // whole warp would issue the 17-term sum
  for (int idx = threadIdx.x; idx < owny * TE; idx += blockDim.x) {
    const int jy = idx / TE, lex = idx - jy * TE;
    const T* Ll = sLx + lex * NP * NP + P * NP;
    const T* ul = su + (jy + P) * LP + lex * P;
    T t = T(0);
#pragma unroll
    for (int k = 0; k < NP; ++k) t += Ll[k] * ul[k];
    sbx[idx] = t;
  }
  __syncthreads();
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < ownx * owny; idx += blockDim.x) {
    // full tiles (TN or TN + 1 owned columns) divide by a constant
    const int jy = ownx == TN ? idx / TN : (ownx == TN + 1 ? idx / (TN + 1) : idx / ownx);
    const int ix = idx - jy * ownx;
    const int gi = ex0 * P + ix, gj = ey0 * P + jy;
    const long o = (long)gj * Nx + gi;
    const bool wall = gnode[ix + P] < 0 || gnode[LN + jy + P] < 0;
    T val = T(0);
    if (!wall) {
      const int lex = ix / P, a = ix - lex * P;
      const int ley = jy / P, b = jy - ley * P;
      const T* row = su + (jy + P) * LP;          // staged row of node (j, .)
      // x direction: element row a of element lex (+ left neighbour's last row)
      T xs = T(0), ys = T(0);
      {
        const T* L = sLx + (lex + 1) * NP * NP + a * NP;
        const T* uu = row + lex * P + P;
#pragma unroll
        for (int k = 0; k < NP; ++k) xs += L[k] * uu[k];
        if (a == 0 && lex < TE) xs += sbx[jy * TE + lex];
      }
      {
        const T* L = sLy + (ley + 1) * NP * NP + b * NP;
        const T* uu = su + (ley * P + P) * LP + ix + P;
#pragma unroll
        for (int k = 0; k < NP; ++k) ys += L[k] * uu[k * LP];
        if (b == 0) {
          const T* Ll = sLy + ley * NP * NP + P * NP;
          const T* ul = su + (ley * P) * LP + ix + P;
#pragma unroll
          for (int k = 0; k < NP; ++k) ys += Ll[k] * ul[k * LP];
        }
      }
      val = sMy[jy] * xs + sMx[ix] * ys;
      if (f) val = convert_to<T>(f[o]) - val;
    }
    out[o] = val;
    if (uout) uout[o] = wall ? T(0) : su[(jy + P) * LP + ix + P];
    if (dot == 1) acc += (double)su[(jy + P) * LP + ix + P] * (double)val;
    else if (dot == 2) acc += (double)val * (double)val;
  }
  if (dot) {
    const double s = block_sum_w0(acc, sred);
    if (threadIdx.x == 0) part[by * gxd + bx] = s;
  }
}


// ---- grid transfer ------------------------------------------------------------
template <int PF>
struct TT {
  static constexpr int PC = PF / 2;
  static constexpr int TE = tile_elems(PF);            // elements per tile per direction
  static constexpr int TNF = TE * PF;
  static constexpr int TNC = TE * PC;
  static constexpr int NPF = PF + 1, NPC = PC + 1;
};

// fc = I^T rf.  Fine nodes staged: [E0 pf - pf, E0 pf + TNF] per direction.
// One coarse tile (bx, by); smem: restrict_smem<T, PF>() bytes.
template <typename T, int PF>
__device__ __forceinline__ void restrict_tile(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx,
                                              const DirView<T>& cy, const T* __restrict__ J,
                                              const T* __restrict__ rf, T* __restrict__ fc, int bx, int by,
                                              unsigned char* smem_raw) {
  using Q = TT<PF>;
  constexpr int PC = Q::PC, TE = Q::TE, TNF = Q::TNF, TNC = Q::TNC, NPC = Q::NPC;
  constexpr int LN = TNF + PF + 1, LP = LN + 1, TP = TNC + 2;
  T* sr = reinterpret_cast<T*>(smem_raw);  // LN x LP fine residual
  T* st = sr + LN * LP;                     // LN x TP  x-contracted
  T* sJ = st + LN * TP;                     // NPF x NPC
  T* sbx = sJ + (PF + 1) * NPC;             // LN x TE: x sums from the element on the left
  T* sby = sbx + LN * TE;                   // TE x (TNC + 1): y sums from the element below
  const int E0x = bx * TE, E0y = by * TE;
  const int gx0 = E0x * PF - PF, gy0 = E0y * PF - PF;
  for (int idx = threadIdx.x; idx < LN * LN; idx += blockDim.x) {
    const int ly = idx / LN, lx = idx - ly * LN;
    const int gx = node_or_wall(gx0 + lx, fx.N, fx.periodic, fx.segN);
    const int gy = node_or_wall(gy0 + ly, fy.N, fy.periodic, fy.segN);
    sr[ly * LP + lx] = (gx >= 0 && gy >= 0) ? rf[(long)gy * fx.N + gx] : T(0);
  }
  for (int idx = threadIdx.x; idx < (PF + 1) * NPC; idx += blockDim.x) sJ[idx] = J[idx];
  __syncthreads();
  const bool lastx = E0x + TE >= cx.n, lasty = E0y + TE >= cy.n;
  const int ownx = min(TE, cx.n - E0x) * PC + ((!cx.periodic && lastx) ? 1 : 0);
  const int owny = min(TE, cy.n - E0y) * PC + ((!cy.periodic && lasty) ? 1 : 0);
  // A coarse node on an element's left (lower) edge, K = 0, also collects the
  // element on that side through its last coarse basis function PC.  In FP64
  // those sums come from one thread per (row, element) (in the contraction
  // loops every warp would issue them for its few K = 0 lanes, on the narrow
  // FP64 pipe), and the element's own part runs over i = 0 .. PF-1 for every
  // K: J[0][K] = 0 for K != 0 (fine node 0 is coarse node 0).  In FP32 the
  // extra passes and barriers cost more than the divergence they remove
  // (measured), so the K = 0 lanes sum both parts in place.
  constexpr bool kPass = std::is_same<T, double>::value;
  if (kPass) {
  for (int idx = threadIdx.x; idx < LN * TE; idx += blockDim.x) {
    const int ly = idx / TE, le = idx - ly * TE;
    const T* row = sr + ly * LP + le * PF + PF;
    T t = T(0);
#pragma unroll
    for (int i = 1; i < PF; ++i) t += sJ[i * NPC + PC] * row[i - PF];
    sbx[idx] = t;
  }
  __syncthreads();
  }
  // x contraction for every staged fine row
  for (int idx = threadIdx.x; idx < LN * ownx; idx += blockDim.x) {
    const int ly = idx / ownx, ic = idx - ly * ownx;
    const int le = ic / PC, K = ic - le * PC;
    const T* row = sr + ly * LP + le * PF + PF;  // fine local node 0 of element E0x + le
    T t = T(0);
    if (le < TE) {
      if (kPass) {
#pragma unroll
        for (int i = 0; i < PF; ++i) t += sJ[i * NPC + K] * row[i];
        if (K == 0) t += sbx[ly * TE + le];
      } else if (K != 0) {
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
  if (kPass) {
  for (int idx = threadIdx.x; idx < TE * ownx; idx += blockDim.x) {
    const int le = idx / ownx, ic = idx - le * ownx;
    const T* col = st + (le * PF + PF) * TP + ic;
    T t = T(0);
#pragma unroll
    for (int j = 1; j < PF; ++j) t += sJ[j * NPC + PC] * col[(j - PF) * TP];
    sby[le * (TNC + 1) + ic] = t;
  }
  __syncthreads();
  }
  for (int idx = threadIdx.x; idx < owny * ownx; idx += blockDim.x) {
    const int jc = idx / ownx, ic = idx - jc * ownx;
    const int gI = E0x * PC + ic, gJ = E0y * PC + jc;
    const bool wall = wall_node(gI, cx.N, cx.periodic, cx.segN) || wall_node(gJ, cy.N, cy.periodic, cy.segN);
    T v = T(0);
    if (!wall) {
      const int le = jc / PC, K = jc - le * PC;
      const T* col = st + (le * PF + PF) * TP + ic;
      if (kPass) {
#pragma unroll
        for (int j = 0; j < PF; ++j) v += sJ[j * NPC + K] * col[j * TP];
        if (K == 0 && le < TE) v += sby[le * (TNC + 1) + ic];
      } else if (K != 0) {
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
// One fine tile (bx, by); smem: prolong_smem<T, PF>() bytes.
// DOT (TOut double): also the z.q and z.r partials of the written values z,
// per problem, and, in the last CTA, beta and delta (PcgDot); every CTA of
// the launch runs it.
// The part of prolong_tile after the staging: sc holds the tile's coarse
// values (LC x LCP), sJ the table, st is scratch (LC x TP).
template <typename T, typename TOut, int PF, bool DOT>
__device__ __forceinline__ void prolong_finish(const DirView<T>& fx, const DirView<T>& fy, const T* sc, T* st,
                                               const T* sJ, const T* in, TOut* out, int bx, int by,
                                               const PcgDot* dot) {
  using Q = TT<PF>;
  constexpr int PC = Q::PC, TE = Q::TE, TNF = Q::TNF, TNC = Q::TNC, NPC = Q::NPC;
  constexpr int LC = TNC + 1, LCP = LC + 1, TP = TNF + 2;
  const int E0x = bx * TE, E0y = by * TE;
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
  double zq = 0.0, zr = 0.0;  // DOT: this thread's part of z.q, z.r (wall nodes: z = 0)
  for (int idx = threadIdx.x; idx < owny * ownx; idx += blockDim.x) {
    const int jy = idx / ownx, ix = idx - jy * ownx;
    const int gi = E0x * PF + ix, gj = E0y * PF + jy;
    const long o = (long)gj * fx.N + gi;
    const bool wall = wall_node(gi, fx.N, fx.periodic, fx.segN) || wall_node(gj, fy.N, fy.periodic, fy.segN);
    if (wall) {
      out[o] = TOut(0);
      continue;
    }
    const int le = jy / PF, j = jy - le * PF;
    const T* col = st + (le * PC) * TP + ix;
    T v = T(0);
#pragma unroll
    for (int k = 0; k < NPC; ++k) v += sJ[j * NPC + k] * col[k * TP];
    const TOut z = in ? convert_to<TOut>(in[o] + v) : convert_to<TOut>(v);
    out[o] = z;
    if constexpr (DOT) {
      zq += z * dot->q[o];
      zr += z * dot->r[o];
    }
  }
  if constexpr (DOT) {
    static_assert(std::is_same<TOut, double>::value, "the fused dot products take the FP64 z");
    __shared__ double sred[kRedThreads];
    __shared__ int am_last;
    const double sq = block_sum_w0(zq, sred);
    const double sr = block_sum_w0(zr, sred);
    const int kp = by / dot->gyp, G = gridDim.x * dot->gyp;
    const int c = (by - kp * dot->gyp) * gridDim.x + bx;
    if (threadIdx.x == 0) {
      dot->part[(long)kp * G + c] = sq;
      dot->part[(long)(dot->st.nb + kp) * G + c] = sr;
      __threadfence();
      am_last = atomicAdd(dot->st.ticket, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    pcg_beta_finish(dot->part, G, dot->st, sred);
  }
}

template <typename T, typename TOut, int PF, bool DOT = false>
__device__ __forceinline__ void prolong_tile(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx,
                                             const DirView<T>& cy, const T* __restrict__ J,
                                             const T* __restrict__ uc, const T* in, TOut* out, int bx, int by,
                                             unsigned char* smem_raw, const PcgDot* dot = nullptr) {
  using Q = TT<PF>;
  constexpr int PC = Q::PC, TE = Q::TE, TNF = Q::TNF, TNC = Q::TNC, NPC = Q::NPC;
  constexpr int LC = TNC + 1, LCP = LC + 1, TP = TNF + 2;
  T* sc = reinterpret_cast<T*>(smem_raw);  // LC x LCP coarse values
  T* st = sc + LC * LCP;                    // LC x TP  x-interpolated
  T* sJ = st + LC * TP;
  const int E0x = bx * TE, E0y = by * TE;
  for (int idx = threadIdx.x; idx < LC * LC; idx += blockDim.x) {
    const int ly = idx / LC, lx = idx - ly * LC;
    const int gx = node_or_wall(E0x * PC + lx, cx.N, cx.periodic, cx.segN);
    const int gy = node_or_wall(E0y * PC + ly, cy.N, cy.periodic, cy.segN);
    sc[ly * LCP + lx] = (gx >= 0 && gy >= 0) ? uc[(long)gy * cx.N + gx] : T(0);
  }
  for (int idx = threadIdx.x; idx < (PF + 1) * NPC; idx += blockDim.x) sJ[idx] = J[idx];
  __syncthreads();
  prolong_finish<T, TOut, PF, DOT>(fx, fy, sc, st, sJ, in, out, bx, by, dot);
}

// ---- the up-leg of the V-cycle in one pass ------------------------------------
// Without post-smoothing the up-leg of Alg. 3 is u_l <- u_l + I_l u_{l-1},
// l = 1 .. L, with u_0 the coarse solution.  Every level has the same element
// mesh (only the order p_l = 2^l changes) and I_l acts element by element, so
// a CTA can carry its tile of TE x TE elements (TE of the finest level) from
// level 0 up to level L in shared memory.  Level l < L needs all
// (TE p_l + 1)^2 nodes of the tile, the ones it shares with the next tile
// included: such a node is interpolated from this tile's element, through the
// end rows of J, which are exactly 0 and 1 (the GLL end points of both orders
// are -1 and 1), so it gets the value the owning tile computes.  Per node the
// arithmetic is that of prolong_tile, in the same order; results are identical
// to the level-by-level launches.

// level of order P in the chain: (TE P + 1)^2 nodes, row pitch TE P + 2
__host__ __device__ constexpr int chain_nodes(int te, int P) { return te * P + 1; }
// offset of the level of order P among the node buffers of orders 1, 2, .. P / 2
__host__ __device__ constexpr int chain_voff(int te, int P) {
  return P <= 1 ? 0 : chain_voff(te, P / 2) + chain_nodes(te, P / 2) * (chain_nodes(te, P / 2) + 1);
}
// flat index of the first staged node of the level of order P
__host__ __device__ constexpr int chain_soff(int te, int P) {
  return P <= 1 ? 0 : chain_soff(te, P / 2) + chain_nodes(te, P / 2) * chain_nodes(te, P / 2);
}
// offset of the table of order P / 2 -> P among those of orders 2, 4, .. P / 2
__host__ __device__ constexpr int chain_joff(int P) { return P <= 2 ? 0 : chain_joff(P / 2) + (P / 2 + 1) * (P / 4 + 1); }

template <int PF>
struct ChainGeo {
  static constexpr int TE = tile_elems(PF);
  static constexpr int V = chain_voff(TE, PF);                   // node buffers of orders 1 .. PF / 2
  static constexpr int NS = chain_soff(TE, PF);                  // staged nodes
  static constexpr int J = chain_joff(PF) + (PF + 1) * (PF / 2 + 1);  // tables of orders 2 .. PF
  static constexpr int ST = chain_nodes(TE, PF / 2) * (TE * PF + 2);  // x-interpolated rows (largest step)
};

template <typename T, int PF>
constexpr size_t prolong_chain_smem() {
  using G = ChainGeo<PF>;
  return sizeof(T) * (G::V + G::ST + G::J);
}

// shared-memory offset and global address of staged node q (flat over the
// levels of orders P, 2 P, .. PF / 2); addr = nullptr: wall (value 0)
template <typename T, int P, int PF>
__device__ __forceinline__ void chain_locate(const DirView<T>* cx, const DirView<T>* cy, const T* const* cu, int q,
                                             int E0x, int E0y, int& off, const T*& addr) {
  constexpr int TE = ChainGeo<PF>::TE, n = chain_nodes(TE, P);
  if constexpr (P < PF) {
    if (q < n * n) {
      constexpr int l = ilog2_c(P);
      const int ly = q / n, lx = q - ly * n;
      const DirView<T>& x = cx[l];
      const DirView<T>& y = cy[l];
      const int gx = node_or_wall(E0x * P + lx, x.N, x.periodic, x.segN);
      const int gy = node_or_wall(E0y * P + ly, y.N, y.periodic, y.segN);
      off = chain_voff(TE, P) + ly * (n + 1) + lx;
      addr = (gx >= 0 && gy >= 0) ? cu[l] + (long)gy * x.N + gx : nullptr;
      return;
    }
    chain_locate<T, 2 * P, PF>(cx, cy, cu, q - n * n, E0x, E0y, off, addr);
  }
}

// shared-memory offset (from the first table) and global address of entry q
// of the tables of orders P / 2 -> P, P -> 2 P, .. PF / 2 -> PF
template <typename T, int P, int PF>
__device__ __forceinline__ void chain_locate_J(const T* const* cJ, const T* J, int q, int& off, const T*& addr) {
  constexpr int n = (P + 1) * (P / 2 + 1);
  if constexpr (P == PF) {
    off = chain_joff(P) + q;
    addr = J + q;
  } else {
    if (q < n) {
      off = chain_joff(P) + q;
      addr = cJ[ilog2_c(P)] + q;
      return;
    }
    chain_locate_J<T, 2 * P, PF>(cJ, J, q - n, off, addr);
  }
}

// level of order P from the level below (vc) into vf, which holds u of the
// level on entry: vf <- vf + I vc on all (TE P + 1)^2 nodes of the tile
template <typename T, int P, int TE>
__device__ __forceinline__ void chain_step(const T* vc, T* vf, T* st, const T* sJ, const DirView<T>& fx,
                                           const DirView<T>& fy, int E0x, int E0y) {
  constexpr int PC = P / 2, NPC = PC + 1, LC = TE * PC + 1, LCP = LC + 1, LF = TE * P + 1, LFP = LF + 1;
  constexpr int TP = TE * P + 2;
  for (int idx = threadIdx.x; idx < LC * LF; idx += blockDim.x) {
    const int ly = idx / LF, ix = idx - ly * LF;
    const int le = min(ix / P, TE - 1), i = ix - le * P;
    const T* row = vc + ly * LCP + le * PC;
    T t = T(0);
#pragma unroll
    for (int k = 0; k < NPC; ++k) t += sJ[i * NPC + k] * row[k];
    st[ly * TP + ix] = t;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < LF * LF; idx += blockDim.x) {
    const int jy = idx / LF, ix = idx - jy * LF;
    const int le = min(jy / P, TE - 1), j = jy - le * P;
    const bool wall = wall_node(E0x * P + ix, fx.N, fx.periodic, fx.segN) ||
                      wall_node(E0y * P + jy, fy.N, fy.periodic, fy.segN);
    const T* col = st + (le * PC) * TP + ix;
    T v = T(0);
#pragma unroll
    for (int k = 0; k < NPC; ++k) v += sJ[j * NPC + k] * col[k * TP];
    T* o = vf + jy * LFP + ix;
    *o = wall ? T(0) : T(*o + v);
  }
  __syncthreads();
}

template <typename T, int P, int PF>
__device__ __forceinline__ void chain_up(const DirView<T>* cx, const DirView<T>* cy, T* sv, T* st, const T* sJ,
                                         int E0x, int E0y) {
  constexpr int TE = ChainGeo<PF>::TE;
  if constexpr (P < PF) {
    constexpr int l = ilog2_c(P);
    chain_step<T, P, TE>(sv + chain_voff(TE, P / 2), sv + chain_voff(TE, P), st, sJ + chain_joff(P), cx[l], cy[l],
                         E0x, E0y);
    chain_up<T, 2 * P, PF>(cx, cy, sv, st, sJ, E0x, E0y);
  }
}

// One tile (bx, by) of the finest level (order PF >= 4): levels 1 .. L-1 in
// shared memory, then out = in + I_L u_{L-1} as prolong_tile (with the dot
// products when DOT).  cx, cy, cu, cJ: views, vectors and tables of levels
// 0 .. L-1 (cJ[0] unused); J the finest level's table.
template <typename T, typename TOut, int PF, bool DOT>
__device__ __forceinline__ void prolong_chain_tile(const DirView<T>* cx, const DirView<T>* cy, const T* const* cu,
                                                   const T* const* cJ, const DirView<T>& fx, const DirView<T>& fy,
                                                   const T* __restrict__ J, const T* in, TOut* out, int bx, int by,
                                                   unsigned char* smem_raw, const PcgDot* dot) {
  using G = ChainGeo<PF>;
  constexpr int TE = G::TE, NS = G::NS;
  constexpr int PER = (NS + G::J + kChainThreads - 1) / kChainThreads;
  T* sv = reinterpret_cast<T*>(smem_raw);  // node buffers of orders 1 .. PF / 2
  T* st = sv + G::V;
  T* sJ = st + G::ST;                       // tables of orders 2 .. PF
  const int E0x = bx * TE, E0y = by * TE;
  // every level's nodes of the tile and every table: all loads first, then
  // the stores (one memory latency)
  T val[PER];
  int off[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int q = threadIdx.x + k * kChainThreads;
    const T* addr = nullptr;
    off[k] = -1;
    if (q < NS) {
      chain_locate<T, 1, PF>(cx, cy, cu, q, E0x, E0y, off[k], addr);
    } else if (q < NS + G::J) {
      chain_locate_J<T, 2, PF>(cJ, J, q - NS, off[k], addr);
      off[k] += G::V + G::ST;
    }
    val[k] = addr ? *addr : T(0);
  }
#pragma unroll
  for (int k = 0; k < PER; ++k)
    if (off[k] >= 0) sv[off[k]] = val[k];
  __syncthreads();
  chain_up<T, 2, PF>(cx, cy, sv, st, sJ, E0x, E0y);
  prolong_finish<T, TOut, PF, DOT>(fx, fy, sv + chain_voff(TE, PF / 2), st, sJ + chain_joff(PF), in, out, bx, by,
                                   dot);
}

template <typename T, int PF>
constexpr size_t restrict_smem() {
  using Q = TT<PF>;
  constexpr int LN = Q::TNF + PF + 1;
  constexpr int extra = std::is_same<T, double>::value ? LN * Q::TE + Q::TE * (Q::TNC + 1) : 0;  // FP64 passes
  return sizeof(T) * (LN * (LN + 1) + LN * (Q::TNC + 2) + (PF + 1) * Q::NPC + extra);
}

template <typename T, int PF>
constexpr size_t prolong_smem() {
  using Q = TT<PF>;
  constexpr int LC = Q::TNC + 1;
  return sizeof(T) * (LC * (LC + 1) + LC * (Q::TNF + 2) + (PF + 1) * Q::NPC);
}

// ---- mma.sync sweep ---------------------------------------------------------------
// One warp per subdomain: the m x m window is padded to MP x MP (MP a multiple
// of 16) in shared memory with zeros, and the four contractions of Eq. (FDM)
// run as warp-level MMAs with FP32 accumulation:
//   P1  Y[a][i] = sum_j S_y[j][a] X[j][i]          (A = S_y^T, B = X)
//   P2  X[a][b] = sum_i Y[a][i] S_x[i][b] / (lam_y[a] + lam_x[b])
//   P3  Y[j][b] = sum_a S_y[j][a] X[a][b]
//   P4  E[j][i] = w_y[j] w_x[i] sum_b Y[j][b] S_x[i][b]
// MODE 1: TF32 operands (mma m16n8k8), MODE 2: BF16 operands (mma m16n8k16).
// Padding rows/columns of S are zero, so the padded products are exact
// extensions of the m x m ones.

__device__ __forceinline__ uint32_t f2tf32(float x) { return tf32_bits_rna(__float_as_uint(x)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C (MP x MP) = A (MP x MP) * B (MP x MP), operands read from shared memory
// through accessor functors (they carry the transposition), result handed to
// an epilogue functor element by element.
template <int MODE, int MP, typename LA, typename LB, typename EP>
__device__ __forceinline__ void warp_gemm(LA la, LB lb, EP ep) {
  constexpr int MT = MP / 16, NT = MP / 8;
  constexpr int KS = MODE == 1 ? 8 : 16;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[MT][NT][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
#pragma unroll
  for (int k0 = 0; k0 < MP; k0 += KS) {
    uint32_t bf[NT][2];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int n = j * 8 + g;
      if (MODE == 1) {
        bf[j][0] = f2tf32(lb(k0 + t, n));
        bf[j][1] = f2tf32(lb(k0 + t + 4, n));
      } else {
        bf[j][0] = pack_bf16(lb(k0 + 2 * t, n), lb(k0 + 2 * t + 1, n));
        bf[j][1] = pack_bf16(lb(k0 + 2 * t + 8, n), lb(k0 + 2 * t + 9, n));
      }
    }
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      const int r = i * 16 + g;
      uint32_t af[4];
      if (MODE == 1) {
        af[0] = f2tf32(la(r, k0 + t));
        af[1] = f2tf32(la(r + 8, k0 + t));
        af[2] = f2tf32(la(r, k0 + t + 4));
        af[3] = f2tf32(la(r + 8, k0 + t + 4));
      } else {
        af[0] = pack_bf16(la(r, k0 + 2 * t), la(r, k0 + 2 * t + 1));
        af[1] = pack_bf16(la(r + 8, k0 + 2 * t), la(r + 8, k0 + 2 * t + 1));
        af[2] = pack_bf16(la(r, k0 + 2 * t + 8), la(r, k0 + 2 * t + 9));
        af[3] = pack_bf16(la(r + 8, k0 + 2 * t + 8), la(r + 8, k0 + 2 * t + 9));
      }
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        if (MODE == 1) mma_tf32(acc[i][j], af, bf[j]);
        else mma_bf16(acc[i][j], af, bf[j]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int r = i * 16 + g, c = j * 8 + 2 * t;
      ep(r, c, acc[i][j][0]);
      ep(r, c + 1, acc[i][j][1]);
      ep(r + 8, c, acc[i][j][2]);
      ep(r + 8, c + 1, acc[i][j][3]);
    }
}

constexpr int kMmaWarps = 4;

template <int MP>
struct MmaSmem {
  static constexpr int SA = MP + 4;                    // row pitch (floats)
  static constexpr int MAT = MP * SA;
  static constexpr int PER_WARP = 4 * MAT + 4 * MP;    // X, Y, S_x, S_y, lam_x, lam_y, w_x, w_y
};

// Subdomains first, first + stride, ... of one level, each by one warp; smem:
// this warp's MmaSmem<MP>::PER_WARP floats.
template <typename TIn, int MODE, int MP>
__device__ __forceinline__ void sweep_mma_warp(const DirView<float>& dx, const DirView<float>& dy,
                                               const TIn* __restrict__ r, float* __restrict__ E,
                                               const float* __restrict__ nu_inv, int nsub, int first, int stride,
                                               float* base) {
  using Q = MmaSmem<MP>;
  constexpr int SA = Q::SA;
  const int lane = threadIdx.x & 31;
  float* X = base;
  float* Y = X + Q::MAT;
  float* Sx = Y + Q::MAT;
  float* Sy = Sx + Q::MAT;
  float* lx = Sy + Q::MAT;
  float* ly = lx + MP;
  float* wx = ly + MP;
  float* wy = wx + MP;
  const int m = dx.m, mm = m * m, p = dx.p, no = dx.n_o;
  int cur_tx = -1, cur_ty = -1;  // tables currently in this warp's shared memory
  for (int sidx = first; sidx < nsub; sidx += stride) {
    const int ey = sidx / dx.n, ex = sidx - ey * dx.n;
    const int tx = dx.tab[ex], ty = dy.tab[ey];
    // window gather: every lane issues all its loads before the first store
    constexpr int PER = (MP * MP + 31) / 32;
    float xv[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = lane + 32 * q;
      const int a = idx / MP, b = idx - a * MP;
      float v = 0.f;
      if (idx < MP * MP && a < m && b < m) {
        const int gy = node_or_wall(ey * p + a - no, dy.N, dy.periodic, dy.segN);
        const int gx = node_or_wall(ex * p + b - no, dx.N, dx.periodic, dx.segN);
        if (gx >= 0 && gy >= 0) v = convert_to<float>(r[(long)gy * dx.N + gx]);
      }
      xv[q] = v;
    }
    // tables: reloaded only when this subdomain's type differs from the last
    if (tx != cur_tx) {
      const float* gSx = dx.S + (long)tx * mm;
      for (int idx = lane; idx < MP * MP; idx += 32) {
        const int a = idx / MP, b = idx - a * MP;
        Sx[a * SA + b] = (a < m && b < m) ? gSx[a * m + b] : 0.f;
      }
      for (int idx = lane; idx < MP; idx += 32) {
        lx[idx] = idx < m ? dx.lam[tx * m + idx] : 1.f;
        wx[idx] = idx < m ? dx.w[tx * m + idx] : 0.f;
      }
      cur_tx = tx;
    }
    if (ty != cur_ty) {
      const float* gSy = dy.S + (long)ty * mm;
      for (int idx = lane; idx < MP * MP; idx += 32) {
        const int a = idx / MP, b = idx - a * MP;
        Sy[a * SA + b] = (a < m && b < m) ? gSy[a * m + b] : 0.f;
      }
      for (int idx = lane; idx < MP; idx += 32) {
        ly[idx] = idx < m ? dy.lam[ty * m + idx] : 1.f;
        wy[idx] = idx < m ? dy.w[ty * m + idx] : 0.f;
      }
      cur_ty = ty;
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = lane + 32 * q;
      if (idx < MP * MP) {
        const int a = idx / MP, b = idx - a * MP;
        X[a * SA + b] = xv[q];
      }
    }
    __syncwarp();
    // P1: Y = S_y^T X
    warp_gemm<MODE, MP>([&](int row, int k) { return Sy[k * SA + row]; },
                        [&](int k, int n) { return X[k * SA + n]; },
                        [&](int row, int col, float v) { Y[row * SA + col] = v; });
    __syncwarp();
    // P2: X = (Y S_x) ./ (lam_y + lam_x)
    warp_gemm<MODE, MP>([&](int row, int k) { return Y[row * SA + k]; },
                        [&](int k, int n) { return Sx[k * SA + n]; },
                        [&](int row, int col, float v) { X[row * SA + col] = v / (ly[row] + lx[col]); });
    __syncwarp();
    // P3: Y = S_y X
    warp_gemm<MODE, MP>([&](int row, int k) { return Sy[row * SA + k]; },
                        [&](int k, int n) { return X[k * SA + n]; },
                        [&](int row, int col, float v) { Y[row * SA + col] = v; });
    __syncwarp();
    // P4: E = w_y w_x^T .* (Y S_x^T), written for the m x m window only
    const float sc = nu_inv ? nu_inv[sidx] : 1.f;
    float* Es = E + (long)sidx * mm;
    warp_gemm<MODE, MP>([&](int row, int k) { return Y[row * SA + k]; },
                        [&](int k, int n) { return Sx[n * SA + k]; },
                        [&](int row, int col, float v) {
                          if (row < m && col < m) Es[row * m + col] = wy[row] * wx[col] * v * sc;
                        });
    __syncwarp();
  }
}

}  // namespace sem
