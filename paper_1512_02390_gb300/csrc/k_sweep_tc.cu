// Weighted additive Schwarz sweep on the fifth-generation tensor cores
// (tcgen05, sm_103a): the fast-diagonalisation local solve of Sec. 3.1,
// Eq. (FDM), E_s = W_s (S_y (x) S_x) Lambda^{-1} (S_y^T (x) S_x^T) R_s r, for a
// STACK of subdomains per MMA.
//
// Subdomains with the same factor tables (S_x, S_y, Lambda, w; all interior
// elements of a uniform mesh share them) are grouped G = floor(128 / m) at a
// time; their m x m windows are stacked into the 128 rows of one accumulator
// (one TMEM lane per row, one CTA thread per lane).  Every product of the FDM
// is then a right multiplication of the stack by a shared m x m table:
//
//   G1  C1[(s,a)][bh] = sum_b  X_s[a][b]     S_x[b][bh]       (x transform)
//   G2  C2[(s,bh)][ah] = sum_a C1[(s,a)][bh]  S_y[a][ah]      (y transform; A = per-subdomain transpose of C1)
//       C2 /= lambda_y[ah] + lambda_x[bh]
//   G3  C3[(s,bh)][a] = sum_ah C2[(s,bh)][ah] S_y[a][ah]      (inverse y transform; A = C2)
//   G4  E_s[a][b]     = sum_bh C3[(s,bh)][a]  S_x[b][bh]      (inverse x transform; A = transpose of C3)
//       E_s[a][b]    *= w_y[a] w_x[b] / nu_bar_s
//
// A (the stack) and B (a table) sit in shared memory in the K-major,
// no-swizzle canonical layout (8-row x 16-byte core matrices; LBO = stride of
// core matrices along K, SBO = stride of 8-row groups); one elected thread
// issues tcgen05.mma, tcgen05.commit arrives on an mbarrier, and the 128
// threads read the accumulator back with tcgen05.ld and write the next A
// operand.  TF32 (kind::tf32) or BF16 (kind::f16) operands, FP32 accumulation.
//
// Every wait on the tensor cores is bounded: a CTA whose wait runs out sets
// *err, stops issuing, waits (bounded) for what it issued, frees its TMEM and
// returns.

#include "k_sweep_tc.cuh"

namespace sem {

namespace {

// NPC = NP / 16: the accumulator row is held in registers (constant indices)
template <typename TIn, int MODE, int NPC>
__global__ void __launch_bounds__(kTcThreads) k_sweep_tc(DirView<float> dx, DirView<float> dy,
                                                         const TIn* __restrict__ r, float* __restrict__ E,
                                                         const float* __restrict__ nu_inv, TcWork wk, TcLay L) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sB = smem + L.a_bytes;  // tables B1 = S_x^T, B2 = S_y^T, B3 = S_y, B4 = S_x (N x K rows)
  float* lxs = reinterpret_cast<float*>(sB + 4 * L.b_bytes);
  float* lys = lxs + 64;
  float* wxs = lys + 64;
  float* wys = wxs + 64;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  __shared__ int s_flag;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t bar = smem_addr(&mbar);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tbase)),
                 "r"(L.cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // zero the stack once: padded rows and K columns stay zero for every stage
  for (int i = t; i < (int)(L.a_bytes / 4); i += kTcThreads) reinterpret_cast<uint32_t*>(sA)[i] = 0u;
  bool ok = tc_sync(true);
  const uint32_t tmem = tbase;
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t a_s = smem_addr(sA);
  const int m = L.m, mm = m * m, G = L.G, NP = NPC * 16, KP = L.KP;
  const int p = dx.p, no = dx.n_o, Nx = dx.N;
  const int rows = G * m;
  // this thread's stack row: subdomain slot s, local index j (a or bh)
  const int s_me = t / m, j_me = t - s_me * m;
  const int per = (wk.ngroups + gridDim.x - 1) / gridDim.x;
  const int g0 = blockIdx.x * per, g1 = min(wk.ngroups, g0 + per);
  int cur_tx = -1, cur_ty = -1;
  uint32_t phase = 0;
  float v[16];  // accumulator columns are read 16 at a time
  for (int g = g0; g < g1 && ok; ++g) {
    const int* sub = wk.sub + (long)g * G;
    const int first = sub[0];
    const int tx = dx.tab[first % dx.n], ty = dy.tab[first / dx.n];
    if (tx != cur_tx || ty != cur_ty) {
      // the previous MMAs have completed: the tables may be overwritten
      const float* Sx = dx.S + (long)tx * mm;
      const float* Sy = dy.S + (long)ty * mm;
      for (int idx = t; idx < NP * KP; idx += kTcThreads) {
        const int n = idx / KP, k = idx - n * KP;
        const bool in = n < m && k < m;
        const uint32_t o = op_off<MODE>(n, k, L);
        op_put<MODE>(sB, o, in ? Sx[k * m + n] : 0.f);
        op_put<MODE>(sB + L.b_bytes, o, in ? Sy[k * m + n] : 0.f);
        op_put<MODE>(sB + 2 * L.b_bytes, o, in ? Sy[n * m + k] : 0.f);
        op_put<MODE>(sB + 3 * L.b_bytes, o, in ? Sx[n * m + k] : 0.f);
      }
      for (int i = t; i < 64; i += kTcThreads) {
        lxs[i] = i < m ? dx.lam[tx * m + i] : 1.f;
        lys[i] = i < m ? dy.lam[ty * m + i] : 1.f;
        wxs[i] = i < m ? dx.w[tx * m + i] : 0.f;
        wys[i] = i < m ? dy.w[ty * m + i] : 0.f;
      }
      cur_tx = tx;
      cur_ty = ty;
    }
    // gather R_s r into the stack.  Lane l of every warp first finds the
    // window origin of slots l and l + 32 (flag 1: window inside the grid and
    // clear of stacked-problem walls, no per-node checks; 2: needs them;
    // 0: empty slot); then warp w takes window rows w, w + 4, ... and lane b
    // reads node b of the row (consecutive lanes, consecutive nodes).
    int oy0 = 0, ox0 = 0, fl0 = 0, oy1 = 0, ox1 = 0, fl1 = 0;
    {
      auto origin = [&](int s, int& oy, int& ox, int& fl) {
        const int sidx = s < G ? sub[s] : -1;
        if (sidx < 0) return;
        const int ey = sidx / dx.n, ex = sidx - ey * dx.n;
        oy = ey * p - no;
        ox = ex * p - no;
        // every node of the window an unknown: inside the walls, and no
        // stacked-problem wall (multiple of segN) in [o, o + m - 1]
        const bool in_y = oy > 0 && oy + m - 1 < dy.N - 1 &&
                          (dy.segN == 0 || (oy - 1) / dy.segN == (oy + m - 1) / dy.segN);
        const bool in_x = ox > 0 && ox + m - 1 < dx.N - 1 &&
                          (dx.segN == 0 || (ox - 1) / dx.segN == (ox + m - 1) / dx.segN);
        fl = (in_x && in_y && !dx.periodic && !dy.periodic) ? 1 : 2;
      };
      origin(lane, oy0, ox0, fl0);
      origin(lane + 32, oy1, ox1, fl1);
    }
    if (m <= 32) {
      // four rows per batch: all loads of a batch are issued before its stores
      int s = 0, a = warp;  // row = s m + a, advanced by 4 rows at a time
      while (a >= m) a -= m, ++s;
      for (int row = warp; row < rows; row += 4 * (kTcThreads / 32)) {
        float xv[4];
        uint32_t ro[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rq = row + q * (kTcThreads / 32);
          const int src = s & 31;
          const bool hi = s >= 32;
          const int oy = __shfl_sync(0xffffffffu, hi ? oy1 : oy0, src);
          const int ox = __shfl_sync(0xffffffffu, hi ? ox1 : ox0, src);
          const int fl = __shfl_sync(0xffffffffu, hi ? fl1 : fl0, src);
          ro[q] = rq < rows ? row_off(rq, L.sbo) : 0xffffffffu;
          xv[q] = 0.f;
          if (rq < rows && lane < m && fl != 0) {
            int gy = oy + a, gx = ox + lane;
            if (fl == 2) {
              gy = node_or_wall(gy, dy.N, dy.periodic, dy.segN);
              gx = node_or_wall(gx, Nx, dx.periodic, dx.segN);
            }
            if (gx >= 0 && gy >= 0) xv[q] = convert_to<float>(r[(long)gy * Nx + gx]);
          }
          a += kTcThreads / 32;
          while (a >= m) a -= m, ++s;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (ro[q] != 0xffffffffu && lane < m) op_put<MODE>(sA, ro[q] + k_off<MODE>(lane), xv[q]);
      }
    } else {
      int s = 0, a = warp;  // row = s m + a, advanced by 4 rows per step
      while (a >= m) a -= m, ++s;
      for (int row = warp; row < rows; row += kTcThreads / 32) {
        const int src = s & 31;
        const bool hi = s >= 32;
        const int oy = __shfl_sync(0xffffffffu, hi ? oy1 : oy0, src);
        const int ox = __shfl_sync(0xffffffffu, hi ? ox1 : ox0, src);
        const int fl = __shfl_sync(0xffffffffu, hi ? fl1 : fl0, src);
        const uint32_t ro = row_off(row, L.sbo);
        int gy = oy + a;
        if (fl == 2) gy = node_or_wall(gy, dy.N, dy.periodic, dy.segN);
        for (int b = lane; b < m; b += 32) {
          float x = 0.f;
          if (fl == 1) {
            x = convert_to<float>(r[(long)gy * Nx + ox + b]);
          } else if (fl == 2 && gy >= 0) {
            const int gx = node_or_wall(ox + b, Nx, dx.periodic, dx.segN);
            if (gx >= 0) x = convert_to<float>(r[(long)gy * Nx + gx]);
          }
          op_put<MODE>(sA, ro + k_off<MODE>(b), x);
        }
        a += kTcThreads / 32;
        while (a >= m) a -= m, ++s;
      }
    }
    ok = tc_sync(ok);
    if (!ok) break;
    // G1: C1 = X S_x
    ok = tc_step<MODE>(tmem, a_s, smem_addr(sB), L, bar, phase, &s_flag);
    if (ok) {
      // A2[(s, bh)][a] = C1[(s, a)][bh]
      const uint32_t ko = k_off<MODE>(j_me);
#pragma unroll
      for (int c = 0; c < NPC; ++c) {
        tmem_ld16(taddr + c * 16, v);
        tmem_wait_ld();
        if (t < rows) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c * 16 + i < m) op_put<MODE>(sA, row_off(s_me * m + c * 16 + i, L.sbo) + ko, v[i]);
        }
      }
    }
    ok = tc_sync(ok);
    if (!ok) break;
    // G2: C2 = A2 S_y, then / (lambda_y + lambda_x)
    ok = tc_step<MODE>(tmem, a_s, smem_addr(sB + L.b_bytes), L, bar, phase, &s_flag);
    if (ok) {
      const float lx = lxs[j_me];
      unsigned char* ro = sA + row_off(t, L.sbo);
#pragma unroll
      for (int c = 0; c < NPC; ++c) {
        tmem_ld16(taddr + c * 16, v);
        tmem_wait_ld();
        if (t < rows) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int ah = c * 16 + i;
            if (ah < m) op_put<MODE>(ro, k_off<MODE>(ah), __fdividef(v[i], lys[ah] + lx));
          }
        }
      }
    }
    ok = tc_sync(ok);
    if (!ok) break;
    // G3: C3 = C2 S_y^T
    ok = tc_step<MODE>(tmem, a_s, smem_addr(sB + 2 * L.b_bytes), L, bar, phase, &s_flag);
    if (ok) {
      // A4[(s, a)][bh] = C3[(s, bh)][a]
      const uint32_t ko = k_off<MODE>(j_me);
#pragma unroll
      for (int c = 0; c < NPC; ++c) {
        tmem_ld16(taddr + c * 16, v);
        tmem_wait_ld();
        if (t < rows) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c * 16 + i < m) op_put<MODE>(sA, row_off(s_me * m + c * 16 + i, L.sbo) + ko, v[i]);
        }
      }
    }
    ok = tc_sync(ok);
    if (!ok) break;
    // G4: E = A4 S_x^T, weighted
    ok = tc_step<MODE>(tmem, a_s, smem_addr(sB + 3 * L.b_bytes), L, bar, phase, &s_flag);
    if (ok) {
      const int sidx = t < rows ? sub[s_me] : -1;
      const float sc = (sidx >= 0 && nu_inv) ? nu_inv[sidx] : 1.f;
      const float wy = wys[j_me];
      float* Es = E + (long)max(sidx, 0) * mm + j_me * m;
#pragma unroll
      for (int c = 0; c < NPC; ++c) {
        tmem_ld16(taddr + c * 16, v);
        tmem_wait_ld();
        if (sidx >= 0) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int b = c * 16 + i;
            if (b < m) Es[b] = wy * wxs[b] * v[i] * sc;
          }
        }
      }
    }
    ok = tc_sync(ok);
  }
  if (!ok && t == 0) {
    atomicExch(wk.err, 1);
    // let the commit still in flight land before the accumulator is freed
    tc_wait(bar, phase ^ 1u);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L.cols));
  }
}

template <int MODE>
TcLay tc_layout(int m) {
  TcLay L{};
  constexpr int ES = MODE == 1 ? 4 : 2, KS = MODE == 1 ? 8 : 16;
  L.m = m;
  L.G = kTcThreads / m;
  L.NP = (m + 15) / 16 * 16;
  L.KP = (m + KS - 1) / KS * KS;
  L.cols = L.NP <= 32 ? 32 : 64;
  const int chunks = L.KP * ES / 16;
  L.lbo = kLbo;
  L.sbo = (uint32_t)chunks * L.lbo;
  L.a_bytes = (kTcThreads / 8) * L.sbo;
  L.b_bytes = (uint32_t)(L.NP / 8) * L.sbo;
  return L;
}

template <typename TIn, int MODE, int NPC>
cudaError_t sweep_tc_launch(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E,
                            const float* nu_inv, const TcWork& wk, const TcLay& L, cudaStream_t s) {
  const size_t sm = L.a_bytes + 4 * (size_t)L.b_bytes + 4 * 64 * sizeof(float);
  // TMEM: at most 512 / cols CTAs of this kernel may be resident on one SM
  const size_t sm_min = (size_t)(228 * 1024) / (512 / L.cols) + 1;
  const size_t smem = std::max(sm, L.cols > 32 ? sm_min : sm);
  cudaError_t e = allow_smem(k_sweep_tc<TIn, MODE, NPC>, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(wk.ngroups, resident_grid(k_sweep_tc<TIn, MODE, NPC>, smem, L.cols));
  e = launch_pdl(k_sweep_tc<TIn, MODE, NPC>, dim3(grid), dim3(kTcThreads), smem, s, dx, dy, r, E, nu_inv, wk, L);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename TIn, int MODE>
cudaError_t sweep_tc_mode(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E,
                          const float* nu_inv, const TcWork& wk, cudaStream_t s) {
  if (dx.m != dy.m || dx.m > 64 || dx.m < 2 || wk.G != kTcThreads / dx.m || wk.ngroups <= 0 || !wk.sub || !wk.err)
    return cudaErrorInvalidValue;
  cudaError_t e = sweep_tcm_lo<TIn>(dx, dy, r, E, MODE, nu_inv, wk, s);
  if (e == cudaErrorNotSupported) e = sweep_tcm_p16<TIn>(dx, dy, r, E, MODE, nu_inv, wk, s);
  if (e == cudaErrorNotSupported) e = sweep_tcm_p32<TIn>(dx, dy, r, E, MODE, nu_inv, wk, s);
  if (e != cudaErrorNotSupported) return e;
  const TcLay L = tc_layout<MODE>(dx.m);
  switch (L.NP / 16) {
    case 1: return sweep_tc_launch<TIn, MODE, 1>(dx, dy, r, E, nu_inv, wk, L, s);
    case 2: return sweep_tc_launch<TIn, MODE, 2>(dx, dy, r, E, nu_inv, wk, L, s);
    case 3: return sweep_tc_launch<TIn, MODE, 3>(dx, dy, r, E, nu_inv, wk, L, s);
    default: return sweep_tc_launch<TIn, MODE, 4>(dx, dy, r, E, nu_inv, wk, L, s);
  }
}

}  // namespace

template <typename TIn>
cudaError_t launch_sweep_tc(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E, int mode,
                            const float* nu_inv, const TcWork& wk, cudaStream_t s) {
  if (mode == 1) return sweep_tc_mode<TIn, 1>(dx, dy, r, E, nu_inv, wk, s);
  if (mode == 2) return sweep_tc_mode<TIn, 2>(dx, dy, r, E, nu_inv, wk, s);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_sweep_tc<float>(const DirView<float>&, const DirView<float>&, const float*, float*, int,
                                            const float*, const TcWork&, cudaStream_t);
template cudaError_t launch_sweep_tc<double>(const DirView<float>&, const DirView<float>&, const double*, float*,
                                             int, const float*, const TcWork&, cudaStream_t);

}  // namespace sem
