// Shared pieces of the tcgen05 Schwarz sweeps (k_sweep_tc.cu and the
// k_sweep_tcm_*.cu translation units, which instantiate the compile-time
// window kernel for disjoint sets of window sizes so that they compile in
// parallel).
//
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
#pragma once

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "f32_round.h"
#include "kernels.h"

namespace sem {

// The compile-time-window sweeps of one set of window sizes m (mode: 1 TF32,
// 2 BF16 operands); cudaErrorNotSupported when m is not in the set.
//   lo:  m = 5 ... 17 odd (the levels p = 2, 4, 8; FP32 right sides only)
//   p16: m = 19, 21, 23 (p = 16, n_o = 1, 2, 3)
//   p32: m = 35, 37, 39 (p = 32, n_o = 1, 2, 3; FP32 and FP64 right sides in
//        two translation units)
template <typename TIn>
cudaError_t sweep_tcm_lo(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E, int mode,
                             const float* nu_inv, const TcWork& wk, cudaStream_t s);
template <typename TIn>
cudaError_t sweep_tcm_p16(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E, int mode,
                             const float* nu_inv, const TcWork& wk, cudaStream_t s);
template <typename TIn>
cudaError_t sweep_tcm_p32(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E, int mode,
                             const float* nu_inv, const TcWork& wk, cudaStream_t s);

namespace {

constexpr int kTcThreads = 128;          // one thread per accumulator row / TMEM lane
constexpr long long kTcWaitCycles = 1LL << 31;  // about one second at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
  return d;
}

// instruction descriptor: D FP32, A/B TF32 (MODE 1) or BF16 (MODE 2), both
// K-major, M = 128, N = n
template <int MODE>
__device__ __forceinline__ uint32_t tc_idesc(int n) {
  const uint32_t fmt = MODE == 1 ? 2u : 1u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcThreads >> 4) << 24);
}

template <int MODE>
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  if (MODE == 1)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// bounded wait for phase `parity` of the mbarrier
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kTcWaitCycles) return false;
  }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Operand geometry of one level (host-computed): N padded to NP (multiple of
// 16: M = 128 needs N % 16 == 0), K padded to KP (multiple of the K step:
// 8 for TF32, 16 for BF16), `chunks` 16-byte core-matrix columns along K.
struct TcLay {
  int m, G, NP, KP, cols;      // cols: TMEM columns allocated (power of two >= 32)
  uint32_t lbo, sbo;           // bytes
  uint32_t a_bytes, b_bytes;   // the stack operand; one table operand
};

// core matrices 144 bytes apart along K (a 16-byte gap): writes of
// consecutive K by consecutive threads then fall in distinct banks
constexpr uint32_t kLbo = 144;

// byte offset of stack / table row `row` and of column k within a row
__device__ __forceinline__ uint32_t row_off(int row, uint32_t sbo) { return (row & 7) * 16 + (row >> 3) * sbo; }
template <int MODE>
__device__ __forceinline__ uint32_t k_off(int k) {
  constexpr int ES = MODE == 1 ? 4 : 2;
  return ((k * ES) & 15) + ((k * ES) >> 4) * kLbo;
}
template <int MODE>
__device__ __forceinline__ uint32_t op_off(int row, int k, const TcLay& L) {
  return row_off(row, L.sbo) + k_off<MODE>(k);
}

// TF32 operand bits, round to nearest, ties away from zero (f32_round.h:
// two integer operations)
__device__ __forceinline__ uint32_t round_tf32(float x) { return tf32_bits_rna(__float_as_uint(x)); }

template <int MODE>
__device__ __forceinline__ void op_put(unsigned char* base, uint32_t off, float v) {
  if (MODE == 1) *reinterpret_cast<uint32_t*>(base + off) = round_tf32(v);
  else *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

// One block-wide step between operand writes and the next MMA: make the
// generic-proxy shared-memory writes visible to the tensor cores, order the
// TMEM reads before the next MMA, and agree on `ok`.
__device__ __forceinline__ bool tc_sync(bool ok) {
  fence_async_smem();
  fence_before();
  const bool all = __syncthreads_and(ok ? 1 : 0) != 0;
  fence_after();
  return all;
}

// D (TMEM) = A (stack) * B^T (table), K = KP; issued by thread 0
template <int MODE>
__device__ __forceinline__ void tc_gemm(uint32_t tmem, uint32_t a, uint32_t b, const TcLay& L, uint32_t bar) {
  constexpr int KS = MODE == 1 ? 8 : 16;  // 32 bytes of K per instruction = 2 core matrices
  const uint32_t idesc = tc_idesc<MODE>(L.NP);
  for (int kb = 0; kb < L.KP / KS; ++kb) {
    const uint32_t step = (uint32_t)kb * 2u * L.lbo;
    tc_mma<MODE>(tmem, tc_desc(a + step, L.lbo, L.sbo), tc_desc(b + step, L.lbo, L.sbo), idesc, kb > 0 ? 1u : 0u);
  }
  tc_commit(bar);
}

// One product of the stack: thread 0 issues it and waits (bounded) for its
// commit; the other threads wait at the barrier, spending no issue slots on
// polling.  Returns the CTA-uniform completion flag.
template <int MODE>
__device__ __forceinline__ bool tc_step(uint32_t tmem, uint32_t a, uint32_t b, const TcLay& L, uint32_t bar,
                                        uint32_t& phase, volatile int* flag) {
  if (threadIdx.x == 0) {
    tc_gemm<MODE>(tmem, a, b, L, bar);
    *flag = tc_wait(bar, phase) ? 1 : 0;
  }
  phase ^= 1u;
  __syncthreads();
  fence_after();
  return *flag != 0;
}

// ---- compile-time window size, row-linear operands ---------------------------
// The kernel above computes every operand offset at run time from the 8-row
// core-matrix layout; for the window sizes of the finest levels the size is a
// template parameter and the operands use the row-linear K-major layout:
// element (row r, column k) sits at byte (k / EPC) * LBO + 16 r + (k % EPC) * ES
// (EPC elements of ES bytes per 16-byte core-matrix row).  The 8-row core
// matrices of one K chunk are contiguous (SBO = 128), the K chunks LBO apart
// (16 bytes more than a chunk, which spreads the chunks over the banks).  A
// transposed write (G1, G3) is then a per-thread base plus an immediate, the
// scaled rewrite of G2 writes whole 16-byte chunks, 1 / (lambda_y + lambda_x)
// comes from a table built with the factors, and w_x is folded into the last
// table (B4 = diag(w_x) S_x).
template <int M, int MODE>
struct TcGeo {
  static constexpr int ES = MODE == 1 ? 4 : 2;
  static constexpr int EPC = 16 / ES;
  static constexpr int KS = MODE == 1 ? 8 : 16;
  static constexpr int G = kTcThreads / M;
  static constexpr int ROWS = G * M;
  static constexpr int NP = (M + 15) / 16 * 16;
  static constexpr int NPC = NP / 16;
  static constexpr int KP = (M + KS - 1) / KS * KS;
  static constexpr int KC = KP / EPC;
  static constexpr uint32_t SBO = 128;
  static constexpr uint32_t LBO_A = kTcThreads * 16 + 16;
  static constexpr uint32_t LBO_B = NP * 16 + 16;
  static constexpr uint32_t A_BYTES = KC * LBO_A;
  static constexpr uint32_t B_BYTES = KC * LBO_B;
  // the stack buffer also stages the G output blocks of M x M floats
  static constexpr uint32_t STAGE_BYTES = (uint32_t)(G * M * M * sizeof(float));
  static constexpr uint32_t A_REGION = ((A_BYTES > STAGE_BYTES ? A_BYTES : STAGE_BYTES) + 15u) / 16u * 16u;
  static constexpr int PAD_CHUNK = M / EPC;  // first K chunk that holds padding columns
  static constexpr int COLS = NP <= 32 ? 32 : 64;
  static constexpr int CW = (M + 31) / 32;  // gather passes over a window row (one column per lane)
  // windows beyond 32 (p = 32) hold three subdomains per stack and about
  // 60 KB of shared memory: three CTAs per SM, more registers per thread
  static constexpr int MIN_CTAS = M <= 32 ? 8 : 3;
  static constexpr size_t SMEM = A_REGION + 4 * (size_t)B_BYTES + (size_t)(M * M + M) * sizeof(float);
  static_assert(M <= 48 && ROWS <= kTcThreads && KP >= M, "window size outside the row-linear kernel");
  __host__ __device__ static constexpr uint32_t off_a(int r, int k) {
    return (uint32_t)(k / EPC) * LBO_A + (uint32_t)r * 16u + (uint32_t)(k % EPC) * ES;
  }
  __host__ __device__ static constexpr uint32_t off_b(int n, int k) {
    return (uint32_t)(k / EPC) * LBO_B + (uint32_t)n * 16u + (uint32_t)(k % EPC) * ES;
  }
};

// D (TMEM) = A * B^T over K = KP, issued by thread 0; then the commit
template <class Q, int MODE>
__device__ __forceinline__ void tcm_gemm(uint32_t tmem, uint32_t a, uint32_t b, uint32_t bar) {
  const uint32_t idesc = tc_idesc<MODE>(Q::NP);
#pragma unroll
  for (int kb = 0; kb < Q::KP / Q::KS; ++kb)
    tc_mma<MODE>(tmem, tc_desc(a + (uint32_t)kb * 2u * Q::LBO_A, Q::LBO_A, Q::SBO),
                 tc_desc(b + (uint32_t)kb * 2u * Q::LBO_B, Q::LBO_B, Q::SBO), idesc, kb > 0 ? 1u : 0u);
  tc_commit(bar);
}

template <class Q, int MODE>
__device__ __forceinline__ bool tcm_step(uint32_t tmem, uint32_t a, uint32_t b, uint32_t bar, uint32_t& phase,
                                         volatile int* flag) {
  if (threadIdx.x == 0) {
    tcm_gemm<Q, MODE>(tmem, a, b, bar);
    *flag = tc_wait(bar, phase) ? 1 : 0;
  }
  phase ^= 1u;
  __syncthreads();
  fence_after();
  return *flag != 0;
}

// 16 bytes of operand row: EPC consecutive K entries
template <int MODE>
__device__ __forceinline__ void op_put16(unsigned char* p, const float* x) {
  uint4 u;
  if (MODE == 1) {
    u.x = round_tf32(x[0]); u.y = round_tf32(x[1]); u.z = round_tf32(x[2]); u.w = round_tf32(x[3]);
  } else {
    __nv_bfloat162 h0 = __floats2bfloat162_rn(x[0], x[1]), h1 = __floats2bfloat162_rn(x[2], x[3]);
    __nv_bfloat162 h2 = __floats2bfloat162_rn(x[4], x[5]), h3 = __floats2bfloat162_rn(x[6], x[7]);
    u.x = *reinterpret_cast<uint32_t*>(&h0); u.y = *reinterpret_cast<uint32_t*>(&h1);
    u.z = *reinterpret_cast<uint32_t*>(&h2); u.w = *reinterpret_cast<uint32_t*>(&h3);
  }
  *reinterpret_cast<uint4*>(p) = u;
}

template <typename TIn, int MODE, int M>
__global__ void __launch_bounds__(kTcThreads, TcGeo<M, MODE>::MIN_CTAS) k_sweep_tcm(DirView<float> dx, DirView<float> dy,
                                                             const TIn* __restrict__ r, float* __restrict__ E,
                                                             const float* __restrict__ nu_inv, TcWork wk) {
  using Q = TcGeo<M, MODE>;
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sB = smem + Q::A_REGION;  // B1 = S_x^T, B2 = S_y^T, B3 = S_y, B4 = diag(w_x) S_x (N x K rows)
  float* inv = reinterpret_cast<float*>(sB + 4 * Q::B_BYTES);  // [ah * M + bh] = 1 / (lambda_y[ah] + lambda_x[bh])
  float* wys = inv + M * M;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  __shared__ int s_flag;
  // metadata of kChunk stacks at a time, loaded once per chunk: the slots'
  // subdomains [gi * G + s], their 1 / nu_bar_s (1 for the Poisson
  // operator) and each stack's table pair tx | ty << 16
  constexpr int kChunk = 16;
  __shared__ int s_sub[kChunk * Q::G];
  __shared__ float s_scale[kChunk * Q::G];
  __shared__ int s_tab[kChunk];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t bar = smem_addr(&mbar);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tbase)),
                 "r"(Q::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // zero the stack once: rows >= ROWS and K columns >= M stay zero
  for (int i = t; i < (int)(Q::A_BYTES / 16); i += kTcThreads) reinterpret_cast<uint4*>(sA)[i] = make_uint4(0, 0, 0, 0);
  bool ok = tc_sync(true);
  const uint32_t tmem = tbase;
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t a_s = smem_addr(sA), b_s = smem_addr(sB);
  const int s_me = t / M, j_me = t - s_me * M;  // this thread's stack row (slot, local index)
  const bool row_ok = t < Q::ROWS;
  // transposed writes: element (row s_me M + c, column j_me) = tr + 16 c
  const uint32_t tr = Q::off_a(s_me * M, j_me);
  // gather writes: element (row s M + warp + 4 i, column lane + 32 c) = g_base[c] + 16 (s M + 4 i)
  uint32_t g_base[Q::CW];
#pragma unroll
  for (int c = 0; c < Q::CW; ++c) g_base[c] = Q::off_a(warp, min(lane + 32 * c, M - 1));
  const int p = dx.p, no = dx.n_o, Nx = dx.N;
  const int per = (wk.ngroups + gridDim.x - 1) / gridDim.x;
  const int g0 = blockIdx.x * per, g1 = min(wk.ngroups, g0 + per);
  int cur_tx = -1, cur_ty = -1;
  uint32_t phase = 0;
  for (int c0 = g0; c0 < g1 && ok; c0 += kChunk) {
  const int cn = min(kChunk, g1 - c0);
  __syncthreads();  // the previous chunk's last epilogue has read s_sub / s_scale
  for (int i = t; i < cn * Q::G; i += kTcThreads) s_sub[i] = wk.sub[(long)c0 * Q::G + i];
  __syncthreads();
  for (int i = t; i < cn * Q::G; i += kTcThreads) {
    const int v = s_sub[i];
    s_scale[i] = (v >= 0 && nu_inv) ? nu_inv[v] : 1.f;
  }
  for (int i = t; i < cn; i += kTcThreads) {
    const int first = s_sub[i * Q::G];  // slot 0 of a stack is never empty
    s_tab[i] = dx.tab[first % dx.n] | (dy.tab[first / dx.n] << 16);
  }
  __syncthreads();
  for (int gi = 0; gi < cn && ok; ++gi) {
    const int* sub = s_sub + gi * Q::G;
    const int tx = s_tab[gi] & 0xffff, ty = s_tab[gi] >> 16;
    if (tx != cur_tx || ty != cur_ty) {
      __syncthreads();  // the previous stack's epilogues have read inv / wys
      const float* Sx = dx.S + (long)tx * M * M;
      const float* Sy = dy.S + (long)ty * M * M;
      const float* wx = dx.w + (long)tx * M;
      // every load of this thread first, then the stores: one memory latency
      constexpr int TI = (Q::NP * Q::KP + kTcThreads - 1) / kTcThreads;
      constexpr int LI = (M * M + kTcThreads - 1) / kTcThreads;
      float b1[TI], b2[TI], b3[TI], b4[TI], ly[LI], lx[LI];
#pragma unroll
      for (int q = 0; q < TI; ++q) {
        const int idx = t + q * kTcThreads;
        const int n = idx / Q::KP, k = idx - n * Q::KP;
        const bool in = idx < Q::NP * Q::KP && n < M && k < M;
        b1[q] = in ? Sx[k * M + n] : 0.f;
        b2[q] = in ? Sy[k * M + n] : 0.f;
        b3[q] = in ? Sy[n * M + k] : 0.f;
        b4[q] = in ? wx[n] * Sx[n * M + k] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < LI; ++q) {
        const int i = t + q * kTcThreads;
        const int ah = i / M, bh = i - ah * M;
        ly[q] = i < M * M ? dy.lam[(long)ty * M + ah] : 1.f;
        lx[q] = i < M * M ? dx.lam[(long)tx * M + bh] : 0.f;
      }
      const float wy_t = t < M ? dy.w[(long)ty * M + t] : 0.f;
#pragma unroll
      for (int q = 0; q < TI; ++q) {
        const int idx = t + q * kTcThreads;
        if (idx < Q::NP * Q::KP) {
          const int n = idx / Q::KP, k = idx - n * Q::KP;
          const uint32_t o = Q::off_b(n, k);
          op_put<MODE>(sB, o, b1[q]);
          op_put<MODE>(sB + Q::B_BYTES, o, b2[q]);
          op_put<MODE>(sB + 2 * Q::B_BYTES, o, b3[q]);
          op_put<MODE>(sB + 3 * Q::B_BYTES, o, b4[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < LI; ++q) {
        const int i = t + q * kTcThreads;
        if (i < M * M) inv[i] = 1.f / (ly[q] + lx[q]);
      }
      if (t < M) wys[t] = wy_t;
      cur_tx = tx;
      cur_ty = ty;
    }
    // window origins: lane l < G of every warp finds slot l (flag 1: window
    // inside the walls and clear of stacked-problem walls; 2: per-node checks;
    // 0: empty slot)
    int oy_l = 0, ox_l = 0, fl_l = 0;
    if (lane < Q::G) {
      const int sidx = sub[lane];
      if (sidx >= 0) {
        const int ey = sidx / dx.n, ex = sidx - ey * dx.n;
        oy_l = ey * p - no;
        ox_l = ex * p - no;
        const bool in_y = oy_l > 0 && oy_l + M - 1 < dy.N - 1 &&
                          (dy.segN == 0 || (oy_l - 1) / dy.segN == (oy_l + M - 1) / dy.segN);
        const bool in_x = ox_l > 0 && ox_l + M - 1 < Nx - 1 &&
                          (dx.segN == 0 || (ox_l - 1) / dx.segN == (ox_l + M - 1) / dx.segN);
        fl_l = (in_x && in_y && !dx.periodic && !dy.periodic) ? 1 : 2;
      }
    }
    // gather R_s r: warp w takes window rows w, w + 4, ... of every slot, lane
    // b nodes b, b + 32, ... of the row; the loads of SB slots at a time are
    // all issued before their stores, so one memory latency covers SB slots
    constexpr int NA = (M + 3) / 4;
    constexpr int SB = Q::CW > 1 ? 1 : (Q::G + 1) / 2;
#pragma unroll
    for (int s0 = 0; s0 < Q::G; s0 += SB) {
      TIn xv[SB][Q::CW][NA];
#pragma unroll
      for (int ds = 0; ds < SB; ++ds) {
        const int s = s0 + ds;
        const int src = s < Q::G ? s : 0;
        const int oy = __shfl_sync(0xffffffffu, oy_l, src);
        const int ox = __shfl_sync(0xffffffffu, ox_l, src);
        const int fl = s < Q::G ? __shfl_sync(0xffffffffu, fl_l, src) : 0;
#pragma unroll
        for (int c = 0; c < Q::CW; ++c) {
          const int col = lane + 32 * c;
          if (fl == 1) {
            // window inside the walls (warp-uniform): lanes past the window
            // read its last column again and do not store
            const TIn* rp = r + (long)(oy + warp) * Nx + ox + min(col, M - 1);
            const long step = 4L * Nx;
#pragma unroll
            for (int i = 0; i < NA; ++i)
              xv[ds][c][i] = (i + 1 < NA || warp + 4 * i < M) ? rp[i * step] : TIn(0);
          } else {
#pragma unroll
            for (int i = 0; i < NA; ++i) {
              const int a = warp + 4 * i;
              xv[ds][c][i] = TIn(0);
              if (a < M && col < M && fl != 0) {
                const int gy = node_or_wall(oy + a, dy.N, dy.periodic, dy.segN);
                const int gx = node_or_wall(ox + col, Nx, dx.periodic, dx.segN);
                if (gx >= 0 && gy >= 0) xv[ds][c][i] = r[(long)gy * Nx + gx];
              }
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < Q::CW; ++c) {
        if (lane + 32 * c < M) {
#pragma unroll
          for (int ds = 0; ds < SB; ++ds) {
            const int s = s0 + ds;
#pragma unroll
            for (int i = 0; i < NA; ++i)
              if (s < Q::G && (i + 1 < NA || warp + 4 * i < M))
                op_put<MODE>(sA, g_base[c] + (uint32_t)(s * M + 4 * i) * 16u, convert_to<float>(xv[ds][c][i]));
          }
        }
      }
    }
    ok = tc_sync(ok);
    if (!ok) break;
    // G1: C1 = X S_x;  A2[(s, bh)][a] = C1[(s, a)][bh]
    ok = tcm_step<Q, MODE>(tmem, a_s, b_s, bar, phase, &s_flag);
    if (ok) {
#pragma unroll
      for (int c = 0; c < Q::NPC; ++c) {
        float v[16];
        tmem_ld16(taddr + c * 16, v);
        tmem_wait_ld();
        if (row_ok) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c * 16 + i < M) op_put<MODE>(sA, tr + (uint32_t)(c * 16 + i) * 16u, v[i]);
        }
      }
    }
    ok = tc_sync(ok);
    if (!ok) break;
    // G2: C2 = A2 S_y, then / (lambda_y[ah] + lambda_x[bh]) into the own row
    ok = tcm_step<Q, MODE>(tmem, a_s, b_s + Q::B_BYTES, bar, phase, &s_flag);
    if (ok) {
      const float* iv = inv + j_me;
      unsigned char* row = sA + (uint32_t)t * 16u;
#pragma unroll
      for (int c = 0; c < Q::NPC; ++c) {
        float v[16];
        tmem_ld16(taddr + c * 16, v);
        tmem_wait_ld();
        if (row_ok) {
#pragma unroll
          for (int q = 0; q < 16 / Q::EPC; ++q) {
            const int k0 = c * 16 + q * Q::EPC;
            if (k0 < Q::KP) {
              float x[Q::EPC];
#pragma unroll
              for (int e = 0; e < Q::EPC; ++e) {
                const int ah = k0 + e;
                x[e] = ah < M ? v[q * Q::EPC + e] * iv[ah * M] : 0.f;
              }
              op_put16<MODE>(row + (uint32_t)(k0 / Q::EPC) * Q::LBO_A, x);
            }
          }
        }
      }
    }
    ok = tc_sync(ok);
    if (!ok) break;
    // G3: C3 = C2 S_y^T;  A4[(s, a)][bh] = C3[(s, bh)][a]
    ok = tcm_step<Q, MODE>(tmem, a_s, b_s + 2 * Q::B_BYTES, bar, phase, &s_flag);
    if (ok) {
#pragma unroll
      for (int c = 0; c < Q::NPC; ++c) {
        float v[16];
        tmem_ld16(taddr + c * 16, v);
        tmem_wait_ld();
        if (row_ok) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c * 16 + i < M) op_put<MODE>(sA, tr + (uint32_t)(c * 16 + i) * 16u, v[i]);
        }
      }
    }
    ok = tc_sync(ok);
    if (!ok) break;
    // G4: E_s[a][b] = w_y[a] / nu_bar_s * sum_bh A4[(s, a)][bh] w_x[b] S_x[b][bh]
    ok = tcm_step<Q, MODE>(tmem, a_s, b_s + 3 * Q::B_BYTES, bar, phase, &s_flag);
    if (ok) {
      // the weighted rows go to the free stack buffer as the E blocks
      // [s][a][b]; warp w then copies blocks w, w + 4, ... to E with
      // consecutive lanes on consecutive floats
      float* stage = reinterpret_cast<float*>(sA);
      const float f = row_ok ? wys[j_me] * s_scale[gi * Q::G + s_me] : 0.f;
#pragma unroll
      for (int c = 0; c < Q::NPC; ++c) {
        float v[16];
        tmem_ld16(taddr + c * 16, v);
        tmem_wait_ld();
        if (row_ok) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c * 16 + i < M) stage[t * M + c * 16 + i] = v[i] * f;
        }
      }
      __syncthreads();
#pragma unroll
      for (int sl = warp; sl < Q::G; sl += kTcThreads / 32) {
        const int sidx = sub[sl];
        if (sidx >= 0) {
          float* Es = E + (long)sidx * (M * M);
          const float* src = stage + sl * (M * M);
#pragma unroll
          for (int i = lane; i < M * M; i += 32) Es[i] = src[i];
        }
      }
      __syncthreads();
      // the staged floats overwrote the zero K padding of the stack operand
      // (as BF16 pairs they can read as NaN); the next gather's barrier
      // orders this before the next product
      for (int i = t; i < (Q::KC - Q::PAD_CHUNK) * kTcThreads; i += kTcThreads)
        *reinterpret_cast<uint4*>(sA + (uint32_t)(Q::PAD_CHUNK + i / kTcThreads) * Q::LBO_A +
                                  (uint32_t)(i % kTcThreads) * 16u) = make_uint4(0, 0, 0, 0);
    }
  }
  }
  if (!ok && t == 0) {
    atomicExch(wk.err, 1);
    tc_wait(bar, phase ^ 1u);  // let a commit still in flight land before the accumulator is freed
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Q::COLS));
  }
}

// CTAs of a kernel that are resident on the whole GPU at once: the SM count
// times the per-SM limit set by threads, registers, shared memory (with the
// per-block reservation) and TMEM columns (`cols` per CTA of 512)
template <class K>
int resident_grid(K kernel, size_t smem, int cols) {
  int dev = 0, sms = 152, smem_sm = 228 * 1024, reserved = 1024;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 152 * 4;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
    return 152 * 4;
  const int by_threads = 2048 / kTcThreads;
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;  // allocation unit: 256 registers per warp
  const int by_regs = regs_warp > 0 ? 65536 / (regs_warp * (kTcThreads / 32)) : by_threads;
  const int by_smem = (int)((size_t)smem_sm / (smem + fa.sharedSizeBytes + (size_t)reserved));
  const int by_tmem = 512 / cols;
  return sms * std::max(1, std::min(std::min(by_threads, by_regs), std::min(by_smem, by_tmem)));
}

template <typename TIn, int MODE, int M>
cudaError_t sweep_tcm_launch(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E,
                             const float* nu_inv, const TcWork& wk, cudaStream_t s) {
  using Q = TcGeo<M, MODE>;
  // TMEM: at most 512 / COLS CTAs may be resident on one SM
  const size_t smem = std::max(Q::SMEM, Q::COLS > 32 ? (size_t)(228 * 1024) / (512 / Q::COLS) + 1 : Q::SMEM);
  cudaError_t e = allow_smem(k_sweep_tcm<TIn, MODE, M>, smem);
  if (e != cudaSuccess) return e;
  static const int cap = resident_grid(k_sweep_tcm<TIn, MODE, M>, smem, Q::COLS);
  const int grid = std::min(wk.ngroups, cap);
  e = launch_pdl(k_sweep_tcm<TIn, MODE, M>, dim3(grid), dim3(kTcThreads), smem, s, dx, dy, r, E, nu_inv, wk);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

// the compile-time kernel for the window sizes Ms: the one that matches m
template <typename TIn, int... Ms>
cudaError_t sweep_tcm_set(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E, int mode,
                          const float* nu_inv, const TcWork& wk, cudaStream_t s) {
  if (mode != 1 && mode != 2) return cudaErrorInvalidValue;
  cudaError_t e = cudaErrorNotSupported;
  (void)((dx.m == Ms && ((e = mode == 1 ? sweep_tcm_launch<TIn, 1, Ms>(dx, dy, r, E, nu_inv, wk, s)
                                        : sweep_tcm_launch<TIn, 2, Ms>(dx, dy, r, E, nu_inv, wk, s)),
                         true)) || ...);
  return e;
}

}  // namespace sem
