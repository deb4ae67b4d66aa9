// The FP64 operator of Eq. (system matrix), A = M_y (x) L_x + L_y (x) M_x,
// with the element-row products evaluated exactly in integers.
//
// The FP64 pipe of this part issues about 2 FMA lanes per clock per SM; a
// 32 x 32 -> 64-bit integer multiply-add (mad.wide.s32) issues about 56.  The
// directional products y_a = sum_k L[a][k] x_k of the node-centric operator
// (the even-odd form of k_operator.cu) therefore run here on the integer pipe,
// as an error-free splitting of both operands (the idea of Ozaki, Ogita and
// Oishi's exact matrix products, with 64-bit integer instead of floating-point
// accumulation):
//   - the staged tile of u, x = X 2^-s with X an integer, |X| < 2^53: the tile's
//     largest exponent keeps all 53 mantissa bits, smaller values are rounded
//     to the same absolute step (2^-53 of the tile's bound);
//   - the element matrix, L = L_int 2^-t with |L_int| < 2^73 (per element and
//     direction, built on the host: setup.cpp fx_tables; elements with equal
//     matrices share one table), exact for the GLL stiffness matrices (their
//     entries span at most 20 binary exponents);
//   - e_k = X_k + X_{p-k}, o_k = X_k - X_{p-k}, E = L_int[a][k] + L_int[a][p-k],
//     O = L_int[a][k] - L_int[a][p-k] are exact integers; with the limbs
//     e = e1 2^25 + e0 (e0 in [0, 2^25), |e1| < 2^29) and E = E2 2^50 + E1 2^25
//     + E0 (E0, E1 in [0, 2^25), |E2| < 2^24) every limb product is below 2^54
//     and goes to the int64 accumulator of its weight (2^0, 2^25, 2^50, 2^75);
//     the even and odd sums together have p + 1 <= 33 terms, two products per
//     weight and term, so each accumulator stays below 2^60: no sum rounds or
//     overflows;
//   - 2 y_a = YE + YO and 2 y_{p-a} = YE - YO, four accumulators each, are
//     rounded to FP64 once (nearest, ties to even; fx_exact.h fx_to_f64).
// A node's value is then My[j] y_x + Mx[i] y_y in FP64, as in the other forms.
// The only roundings are the fixed-point step of x (2^-53 of the tile's
// largest |x|) and the final ones; the even-odd folding itself is exact,
// unlike its FP64 form.  The element tables (16 bytes per entry) are read with
// warp-uniform loads, which the L1 cache serves.
#include <algorithm>

#include "fx_exact.h"
#include "kernels.h"
#include "level_ops.cuh"

namespace sem {

namespace {

template <int P>
struct FxTile {
  static constexpr int H = P / 2;
  static constexpr int TE = Tile<P>::TE, TN = Tile<P>::TN, LN = Tile<P>::LN, NP = P + 1;
  static constexpr int NE = (H + 1) * (H + 1), NO = H * H, EO = NE + NO;
  static constexpr int NV = 2 * H + 1;  // e_0..e_H, o_0..o_{H-1}
  static constexpr int NT = 256;  // threads per CTA
  static constexpr int NW = NT / 32;
  static constexpr int SB = 5;  // staging loads issued together per thread
  // The staged tile without its P x P corner below and left of the tile
  // (read by neither direction): the low-side halo rows 0 .. P-1 hold only
  // the columns P .. LN-1 (pitch TW), rows P .. LN-1 all LN columns.
  static constexpr int TW = LN - P;
  static constexpr int kTop = P * TW;
  static constexpr int kTile = kTop + (LN - P) * LN;
  // The products of one direction: per row (x) or column (y) the low-side
  // neighbour's y_P, then NP values for each of the TE elements.
  static constexpr int PS = 1 + TE * NP;
  static constexpr int kProd = TN * PS;
  // staged value at tile row ly, column w + P (ly in [0, LN), w in [0, TN))
  __device__ static __forceinline__ int col_at(int ly, int w) {
    return ly < P ? ly * TW + w : kTop + (ly - P) * LN + w + P;
  }
  // slot sl's value at element node b (slot 0: only b = P)
  __device__ static __forceinline__ int prod_off(int sl, int b) { return sl == 0 ? 0 : 1 + (sl - 1) * NP + b; }
};

// Shared memory.  Two phase schedules, chosen per order by measurement:
//  - merged (p <= 8): the e/o pairs of both directions are formed from the
//    staged tile, then all products run in one pass (one barrier less, and
//    the items of both directions balance over the warps).  Region A holds
//    the staged tile, later the x and y products; region B the e/o pairs of
//    both directions.
//  - separate (p = 16, 32; the smaller footprint gives p = 32 four CTAs per
//    SM instead of three, and the merged form lost at p = 16 on 256 x 256
//    elements): e/o and products of x, then of y.  Region A holds the staged
//    tile, later the y products; region B the e/o pairs of one direction and
//    the x products.
// The block-sum scratch takes the e/o pairs' place at the end.  Then the mass
// diagonals, the per-warp exponent maxima and the per-slot table indices and
// scales.
template <int P>
struct FxSmem {
  using Q = FxTile<P>;
  static constexpr bool kMerged = P <= 8;
  static constexpr int kTile = Q::kTile;                  // staged tile (double)
  static constexpr int kProd = Q::kProd;                  // products of one direction (double)
  static constexpr int kEv = (Q::TE + 1) * Q::NV * Q::TN;  // e/o pairs of one direction (int2)
  static constexpr int kA = kMerged ? (kTile > 2 * kProd ? kTile : 2 * kProd) : kTile;
  static constexpr int kB = kMerged ? 2 * kEv : kEv + kProd;  // 8-byte words
  static_assert(kEv >= Q::NT && (kMerged || kProd <= kTile), "shared-memory regions overlap");
  static constexpr size_t kBytes =
      8 * ((size_t)kA + kB + 2 * (Q::TN + 1)) + sizeof(int) * (Q::NW + 4 * (Q::TE + 1));
};

template <int P>
size_t apply_fx_smem() {
  return FxSmem<P>::kBytes;
}

__device__ __forceinline__ int2 fx_pair(long long v) {
  int lo, hi;
  fx_limbs(v, lo, hi);
  return make_int2(lo, hi);
}

// e/o limb pairs of one direction from the staged tile su, each value taken
// to fixed point on the way (fx_of: bounded for any input, so a tile with a
// non-finite value, whose outputs are NaN, needs no special case here)
template <int P, bool XDIR>
__device__ __forceinline__ void fx_form_eo(const double* su, int emax, int2* ev) {
  using Q = FxTile<P>;
  constexpr int H = Q::H, TE = Q::TE, TN = Q::TN, LN = Q::LN, NV = Q::NV, kTop = Q::kTop;
  for (int idx = threadIdx.x; idx < (TE + 1) * H * TN; idx += blockDim.x) {
    const int w = idx % TN;
    const int q = idx / TN;
    const int sl = q / H, k = q - sl * H;
    long long xk, xm;
    if (XDIR) {  // row w + P (full width)
      const double* x = su + kTop + w * LN + sl * P;
      xk = fx_of(x[k], emax);
      xm = fx_of(x[P - k], emax);
    } else {  // column w + P
      xk = fx_of(su[Q::col_at(sl * P + k, w)], emax);
      xm = fx_of(su[Q::col_at(sl * P + P - k, w)], emax);
    }
    ev[(sl * NV + k) * TN + w] = fx_pair(xk + xm);
    ev[(sl * NV + H + 1 + k) * TN + w] = fx_pair(xk - xm);
  }
  for (int idx = threadIdx.x; idx < (TE + 1) * TN; idx += blockDim.x) {
    const int w = idx % TN, sl = idx / TN;
    ev[(sl * NV + H) * TN + w] =
        fx_pair(fx_of(XDIR ? su[kTop + w * LN + sl * P + H] : su[Q::col_at(sl * P + H, w)], emax));
  }
}

// element-row products of one direction, item idx = (slot, a, w) of
// TN (1 + TE (H + 1)); slot 0 (the low-side neighbour) only for its y_P.
// sts: the table of each slot's element, then its scale t (the zero table
// where the element does not exist).
template <int P, bool XDIR>
__device__ __forceinline__ void fx_item(const int4* __restrict__ tab, const int* sts, int emax, const int2* ev,
                                        double* dst_base, int idx) {
  using Q = FxTile<P>;
  constexpr int H = Q::H, TE = Q::TE, TN = Q::TN, EO = Q::EO, NE = Q::NE, NV = Q::NV;
  {
    const int w = idx % TN;
    const int q = idx / TN;
    const int sl = q == 0 ? 0 : 1 + (q - 1) / (H + 1);
    const int a = q == 0 ? 0 : (q - 1) % (H + 1);
    const int ts = sts[sl];
    const int4* E = tab + (long)ts * EO + a * (H + 1);
    const int4* O = tab + (long)ts * EO + NE + min(a, H - 1) * H;
    const int2* e = ev + (sl * NV) * TN + w;
    const int2* o = ev + (sl * NV + H + 1) * TN + w;
    long long e0 = 0, e1 = 0, e2 = 0, e3 = 0, o0 = 0, o1 = 0, o2 = 0, o3 = 0;
#pragma unroll
    for (int k = 0; k <= H; ++k) {
      const int4 l = __ldg(E + k);
      const int2 x = e[k * TN];
      e0 += (long long)x.x * l.x;
      e1 += (long long)x.x * l.y + (long long)x.y * l.x;
      e2 += (long long)x.x * l.z + (long long)x.y * l.y;
      e3 += (long long)x.y * l.z;
    }
    if (a < H) {  // the middle row has no odd part; uniform across a warp (w = lane)
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const int4 l = __ldg(O + k);
        const int2 x = o[k * TN];
        o0 += (long long)x.x * l.x;
        o1 += (long long)x.x * l.y + (long long)x.y * l.x;
        o2 += (long long)x.x * l.z + (long long)x.y * l.y;
        o3 += (long long)x.y * l.z;
      }
    }
    // y = (YE +- YO) 2^-(s + t + 1), s = 1075 - emax
    const int K = 1076 - emax + sts[TE + 1 + sl];
    // x: [row w][Q::prod_off], y: [Q::prod_off][column w]; slot 0 stores only y_P (a = 0)
    double* dst = XDIR ? dst_base + w * Q::PS : dst_base + w;
    constexpr int step = XDIR ? 1 : TN;
    if (a < H) dst[Q::prod_off(sl, P - a) * step] = fx_to_f64(e0 - o0, e1 - o1, e2 - o2, e3 - o3, K);
    if (sl > 0) dst[Q::prod_off(sl, a) * step] = fx_to_f64(e0 + o0, e1 + o1, e2 + o2, e3 + o3, K);
  }
}

template <int P>
__global__ void __launch_bounds__(FxTile<P>::NT) k_apply_fx(DirView<double> dx, DirView<double> dy, FxDir fx, FxDir fy,
                                                  const double* __restrict__ u, const double* __restrict__ f,
                                                  double* __restrict__ out, int dot, double* __restrict__ part,
                                                  PcgFuse pf) {
  pdl_enter();
  using Q = FxTile<P>;
  constexpr int TE = Q::TE, TN = Q::TN, LN = Q::LN, NP = Q::NP, NW = Q::NW;
  constexpr int TW = Q::TW, kTop = Q::kTop, PS = Q::PS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using S = FxSmem<P>;
  double* su = reinterpret_cast<double*>(smem_raw);  // region A: the staged tile (Q::kTile)
  int2* evx = reinterpret_cast<int2*>(su + S::kA);    // region B: e/o pairs, (TE+1) x NV x TN
  int2* evy = S::kMerged ? evx + S::kEv : evx;
  double* xb = S::kMerged ? su : reinterpret_cast<double*>(evx + S::kEv);  // [row][Q::prod_off]
  double* yb = S::kMerged ? su + S::kProd : su;                            // [Q::prod_off][col]
  double* sred = reinterpret_cast<double*>(evx);  // NT doubles, once the products are formed
  double* sMx = su + S::kA + S::kB;
  double* sMy = sMx + (TN + 1);
  int* semax = reinterpret_cast<int*>(sMy + (TN + 1));
  int* stab = semax + NW;  // per direction: TE + 1 tables, TE + 1 scales

  const int ex0 = blockIdx.x * TE, ey0 = blockIdx.y * TE;
  const int Nx = dx.N, Ny = dy.N;
  const int gx0 = ex0 * P - P, gy0 = ey0 * P - P;
  const double beta = fused_beta(pf, blockIdx.y, gridDim.y);
  // staging: the operand (z + beta p with the fused direction update, else
  // u) on the tile and its low-side halo, without the P x P corner (shared
  // offset idx: Q::col_at's layout).  The loads of kSB nodes are issued
  // before their stores (one memory latency per batch).
  int emax = 0;  // largest exponent field of the staged values
  constexpr int NT = Q::NT, kNS = (Q::kTile + NT - 1) / NT, kSB = Q::SB;
#pragma unroll
  for (int b0 = 0; b0 < kNS; b0 += kSB) {
    double va[kSB], vb[kSB];
#pragma unroll
    for (int j = 0; j < kSB; ++j) {
      const int idx = threadIdx.x + (b0 + j) * NT;
      va[j] = 0.0;
      vb[j] = 0.0;
      if (b0 + j < kNS && idx < Q::kTile) {
        int ly, lx;
        if (idx < kTop) {
          ly = idx / TW;
          lx = P + idx - ly * TW;
        } else {
          ly = (idx - kTop) / LN;
          lx = idx - kTop - ly * LN;
          ly += P;
        }
        const int gx = node_or_wall(gx0 + lx, Nx, dx.periodic, dx.segN);
        const int gy = node_or_wall(gy0 + ly, Ny, dy.periodic, dy.segN);
        if (gx >= 0 && gy >= 0) {
          const long o = (long)gy * Nx + gx;
          va[j] = u[o];
          if (pf.z) vb[j] = pf.z[o];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kSB; ++j) {
      const int idx = threadIdx.x + (b0 + j) * NT;
      if (b0 + j >= kNS || idx >= Q::kTile) continue;
      const double v = pf.z ? fma(beta, va[j], vb[j]) : va[j];  // as stage_value
      su[idx] = v;
      emax = max(emax, (__double2hiint(v) >> 20) & 0x7ff);
    }
  }
  for (int idx = threadIdx.x; idx <= TN; idx += blockDim.x) {
    const int gx = ex0 * P + idx, gy = ey0 * P + idx;
    sMx[idx] = gx < Nx ? dx.Mg[gx] : 0.0;
    sMy[idx] = gy < Ny ? dy.Mg[gy] : 0.0;
  }
  if (threadIdx.x < 2 * (TE + 1)) {
    // the table and scale of each slot's element (slot sl: element e0 - 1 + sl,
    // in [-1, n + TE - 2]; a periodic mesh has n >= 3 and TE <= 4, so one wrap
    // maps it into [0, n); "element" n is the zero table)
    const bool ydir = threadIdx.x > TE;
    const int sl = ydir ? threadIdx.x - (TE + 1) : threadIdx.x;
    const DirView<double>& d = ydir ? dy : dx;
    const FxDir& fd = ydir ? fy : fx;
    int el = (ydir ? ey0 : ex0) - 1 + sl;
    if (d.periodic) el = el < 0 ? el + d.n : (el >= d.n ? el - d.n : el);
    if (el < 0 || el >= d.n) el = d.n;
    const int ts = __ldg(fd.slot + el);
    stab[(ydir ? 2 * (TE + 1) : 0) + sl] = ts;
    stab[(ydir ? 3 : 1) * (TE + 1) + sl] = __ldg(fd.t + ts);
  }
  emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
  if ((threadIdx.x & 31) == 0) semax[threadIdx.x >> 5] = emax;
  __syncthreads();
#pragma unroll
  for (int w = 0; w < NW; ++w) emax = max(emax, semax[w]);
  const bool finite = emax < 0x7ff;
  const bool lastx = ex0 + TE >= dx.n, lasty = ey0 + TE >= dy.n;
  const int ownx = min(TE, dx.n - ex0) * P + ((!dx.periodic && lastx) ? 1 : 0);
  const int owny = min(TE, dy.n - ey0) * P + ((!dy.periodic && lasty) ? 1 : 0);
  // the owned staged values (for the dot product): the y products overwrite the tile
  constexpr int KOWN = ((TN + 1) * (TN + 1) + NT - 1) / NT;
  double own[KOWN];
#pragma unroll
  for (int q = 0; q < KOWN; ++q) {
    const int idx = threadIdx.x + NT * q;
    own[q] = 0.0;
    if (idx < ownx * owny) {
      const int jy = idx / ownx, ix = idx - jy * ownx;
      own[q] = su[kTop + jy * LN + ix + P];
    }
  }
  const int4* tabx = reinterpret_cast<const int4*>(fx.tab);
  const int4* taby = reinterpret_cast<const int4*>(fy.tab);
  constexpr int XI = TN * (1 + TE * (Q::H + 1));  // product items per direction
  if constexpr (S::kMerged) {
    fx_form_eo<P, true>(su, emax, evx);
    fx_form_eo<P, false>(su, emax, evy);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * XI; idx += NT) {
      if (idx < XI) fx_item<P, true>(tabx, stab, emax, evx, xb, idx);
      else fx_item<P, false>(taby, stab + 2 * (TE + 1), emax, evy, yb, idx - XI);
    }
    __syncthreads();
  } else {
    fx_form_eo<P, true>(su, emax, evx);
    __syncthreads();
    for (int idx = threadIdx.x; idx < XI; idx += NT) fx_item<P, true>(tabx, stab, emax, evx, xb, idx);
    __syncthreads();
    fx_form_eo<P, false>(su, emax, evy);
    __syncthreads();
    for (int idx = threadIdx.x; idx < XI; idx += NT) fx_item<P, false>(taby, stab + 2 * (TE + 1), emax, evy, yb, idx);
    __syncthreads();
  }

  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < KOWN; ++q) {
    const int idx = threadIdx.x + NT * q;
    if (idx >= ownx * owny) break;
    const int jy = idx / ownx, ix = idx - jy * ownx;
    const int gi = ex0 * P + ix, gj = ey0 * P + jy;
    const long o = (long)gj * Nx + gi;
    const bool wall = wall_node(gi, Nx, dx.periodic, dx.segN) || wall_node(gj, Ny, dy.periodic, dy.segN);
    double val = 0.0;
    if (!wall) {
      const int lex = ix / P, a = ix - lex * P;
      const int ley = jy / P, b = jy - ley * P;
      // slot lex + 1's values; a = 0 adds the left slot's y_P (Q::prod_off:
      // 1 + (lex - 1) NP + P, or 0 for slot 0)
      const double* xr = xb + jy * PS + 1 + lex * NP;
      double xs = xr[a];
      if (a == 0) xs += xr[P - NP];
      const double* yc = yb + (1 + ley * NP) * TN + ix;
      double ys = yc[b * TN];
      if (b == 0) ys += yc[(P - NP) * TN];
      val = sMy[jy] * xs + sMx[ix] * ys;
      if (!finite) val = __longlong_as_double(0x7FF8000000000000LL);
      if (f) val = f[o] - val;
    }
    out[o] = val;
    if (dot == 1) acc += own[q] * val;
    else if (dot == 2) acc += val * val;
  }
  if (dot) {
    const double s = block_sum_w0(acc, sred);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

template <int P>
cudaError_t apply_fx_p(const DirView<double>& dx, const DirView<double>& dy, const FxDir& fx, const FxDir& fy,
                       const double* u, const double* f, double* out, int dot, double* part, int* nparts,
                       cudaStream_t s, const PcgFuse& pf) {
  using Q = FxTile<P>;
  dim3 grid((dx.n + Q::TE - 1) / Q::TE, (dy.n + Q::TE - 1) / Q::TE);
  if (dot && (int)(grid.x * grid.y) > kMaxPartials) return cudaErrorInvalidConfiguration;
  if (nparts) *nparts = grid.x * grid.y;
  const size_t sm = apply_fx_smem<P>();
  cudaError_t e = allow_smem(k_apply_fx<P>, sm);
  if (e != cudaSuccess) return e;
  e = launch_pdl(k_apply_fx<P>, grid, dim3(Q::NT), sm, s, dx, dy, fx, fy, u, f, out, dot, part, pf);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply_fx(const DirView<double>& dx, const DirView<double>& dy, const FxDir& fx,
                            const FxDir& fy, const double* u, const double* f, double* out, int dot, double* part,
                            int* nparts, cudaStream_t s, PcgFuse pf) {
  if (!fx.tab || !fx.t || !fx.slot || !fy.tab || !fy.t || !fy.slot || dx.p != dy.p) return cudaErrorInvalidValue;
  switch (dx.p) {
    case 4: return apply_fx_p<4>(dx, dy, fx, fy, u, f, out, dot, part, nparts, s, pf);
    case 8: return apply_fx_p<8>(dx, dy, fx, fy, u, f, out, dot, part, nparts, s, pf);
    case 16: return apply_fx_p<16>(dx, dy, fx, fy, u, f, out, dot, part, nparts, s, pf);
    case 32: return apply_fx_p<32>(dx, dy, fx, fy, u, f, out, dot, part, nparts, s, pf);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sem
