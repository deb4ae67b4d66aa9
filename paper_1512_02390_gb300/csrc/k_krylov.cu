// FP64 vector kernels of the inexact MG-preconditioned CG, Alg. 4.
//
// Reductions are deterministic: a producer kernel writes one partial sum per
// CTA; every CTA of the consumer kernel sums the same partials in the same
// fixed order, so all CTAs agree bit for bit on the scalar (alpha, beta,
// delta) without an extra launch or atomics.  Per-iteration scalars are kept
// in history arrays indexed by the iteration count, so a kernel that reads
// delta_{i-1} never races with the one that writes delta_i.
#include "f32_round.h"
#include "kernels.h"

namespace sem {

namespace {

constexpr int kElemGrid = 4 * 152;

// Elements per thread and pass of the MGCG vector loops (CTAs of kB =
// kRedThreads threads, the block size of every launch below): thread t of
// CTA c takes elements base + j kB (j < kU) with base = lo + c kU kB + t,
// and issues the loads of all kU before using any: one memory round trip per
// pass of kU (on vectors beyond L2, 16.8 M nodes, the vector kernels took
// 11 % less time than with one element per trip; at 1 M nodes the FP64 pipe
// bounds them either way).
constexpr int kU = 4;
constexpr int kB = kRedThreads;

__device__ __forceinline__ long pass_base(long lo) { return lo + (long)blockIdx.x * (kB * kU) + threadIdx.x; }
__device__ __forceinline__ long pass_step() { return (long)gridDim.x * (kB * kU); }

__device__ __forceinline__ bool bad(double x) { return !(fabs(x) <= 1.7976931348623157e308); }

__device__ __forceinline__ void segment(const PcgState& st, long n, int k, long& lo, long& hi) {
  lo = (long)k * st.seg_len;
  hi = (k == st.nb - 1) ? n : lo + st.seg_len;
}

// The vector part of k_update_ur_check over nodes [lo, hi): [HAS_Z: p = z +
// beta p, stored]; u += alpha p; r -= alpha q; [HAS_R32: FP32 copy of r];
// returns this thread's part of ||r||^2
template <bool HAS_Z, bool HAS_R32>
__device__ __forceinline__ double update_ur(long lo, long hi, double alpha, double beta, double* __restrict__ u,
                                            double* __restrict__ r, double* __restrict__ p,
                                            const double* __restrict__ q, const double* __restrict__ z,
                                            float* __restrict__ r32) {
  double acc = 0.0;
  for (long i0 = pass_base(lo); i0 < hi; i0 += pass_step()) {
    double pv[kU], zv[kU], uv[kU], rv[kU], qv[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const long i = i0 + j * kB;
      const bool in = i < hi;
      pv[j] = in ? p[i] : 0.0;
      zv[j] = (HAS_Z && in) ? z[i] : 0.0;
      uv[j] = in ? u[i] : 0.0;
      rv[j] = in ? r[i] : 0.0;
      qv[j] = in ? q[i] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const long i = i0 + j * kB;
      if (i < hi) {
        double pi = pv[j];
        if constexpr (HAS_Z) {
          pi = fma(beta, pv[j], zv[j]);  // the operator staged the same value
          p[i] = pi;
        }
        u[i] = uv[j] + alpha * pi;
        const double ri = rv[j] - alpha * qv[j];
        r[i] = ri;
        if constexpr (HAS_R32) r32[i] = f32_from_f64_rn(ri);  // integer ALU, not the FP64 pipe
        acc += ri * ri;
      }
    }
  }
  return acc;
}

// Iteration i = iter[0], problem k = blockIdx.y (skipped once done):
// [z != null: p = z + beta p with beta = beta_k,iter[1], the direction update
// of Alg. 4 fused here and into the operator that formed q]
// alpha_k = delta_k,i-1 / (p.q)_k;  u += alpha p;  r -= alpha q;  then the
// last CTA reduces every problem's ||r||^2 in fixed order, records the
// scalars, sets done / status (convergence ||r|| <= r_max, breakdown, i_max),
// advances the counter and, inside a graph, sets the WHILE condition to
// "some problem still iterating".  npq: partials of p.q per problem.
// (256, 4): at most 64 registers, so the 4 x 152 CTAs of the grid are resident at once
__global__ void __launch_bounds__(256, 4) k_update_ur_check(long n, double* __restrict__ u, double* __restrict__ r,
                                                         double* __restrict__ p, const double* __restrict__ q,
                                                         const double* __restrict__ part_pq, int npq, PcgState st,
                                                         double* __restrict__ part_rr, int i_max,
                                                         cudaGraphConditionalHandle cond, int use_cond,
                                                         const double* __restrict__ z, float* __restrict__ r32) {
  pdl_enter();
  __shared__ double sred[kRedThreads];
  __shared__ double s_alpha;
  __shared__ int am_last;
  if (*st.active == 0) {  // nothing left (zero or invalid start of every problem)
    if (use_cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  const int k = blockIdx.y;
  const int it = st.iter[0];
  const bool live = st.flags[2 * k] == 0;
  double acc = 0.0;
  if (live) {
    const double pq = sum_partials(part_pq + (long)k * npq, npq, sred);
    // one division per CTA: a double division is a sequence of FP64-pipe
    // operations, and this kernel is bound by that pipe
    if (threadIdx.x == 0) {
      s_alpha = st.delta[(long)k * st.stride + it - 1] / pq;
      if (blockIdx.x == 0) {
        st.pq[(long)k * st.stride + it] = pq;
        st.alpha[(long)k * st.stride + it] = s_alpha;
      }
    }
    __syncthreads();
    const double alpha = s_alpha;
    long lo, hi;
    segment(st, n, k, lo, hi);
    const double beta = z ? st.beta[(long)k * st.stride + st.iter[1]] : 0.0;
    if (z) {
      acc = r32 ? update_ur<true, true>(lo, hi, alpha, beta, u, r, p, q, z, r32)
                : update_ur<true, false>(lo, hi, alpha, beta, u, r, p, q, z, r32);
    } else {
      acc = r32 ? update_ur<false, true>(lo, hi, alpha, beta, u, r, p, q, z, r32)
                : update_ur<false, false>(lo, hi, alpha, beta, u, r, p, q, z, r32);
    }
  }
  const double s = block_sum_w0(acc, sred);
  if (threadIdx.x == 0) {
    part_rr[(long)k * gridDim.x + blockIdx.x] = s;
    __threadfence();
    const unsigned ticket = atomicAdd(st.ticket, 1u);
    am_last = ticket == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  int active = 0;
  for (int kk = 0; kk < st.nb; ++kk) {
    const double rr = sum_partials_cg(part_rr + (long)kk * gridDim.x, gridDim.x, sred);
    if (threadIdx.x == 0 && st.flags[2 * kk] == 0) {
      const long o = (long)kk * st.stride + it;
      st.rr[o] = rr;
      int done = 0, status = 0;
      if (bad(rr) || bad(st.alpha[o]) || !(st.pq[o] > 0.0)) {
        done = 1;
        status = 2;  // SEM_BREAKDOWN
      } else if (sqrt(rr) <= st.rmax[kk]) {
        done = 1;
      } else if (it >= i_max) {
        done = 1;
        status = 1;  // SEM_NOT_CONVERGED
      }
      st.flags[2 * kk] = done;
      st.flags[2 * kk + 1] = status;
      st.iters[kk] = it;
      if (!done) ++active;
    }
  }
  if (threadIdx.x == 0) {
    *st.active = active;
    st.iter[1] = it;      // index for the rest of this iteration (beta, delta)
    st.iter[0] = it + 1;  // next iteration's update
    *st.ticket = 0u;
    if (use_cond) cudaGraphSetConditional(cond, active ? 1u : 0u);
  }
}

// i = iter[1], problem k: partials of z.q (q = A p of iteration i) and z.r;
// the last CTA reduces every live problem's partials in fixed order and
// records beta_i = z^T (r_i - r_{i-1}) / delta_{i-1} in the form
// (i == 1 ? z^T r : -alpha_i z^T q) / delta_{i-1} (r_i - r_{i-1} = -alpha_i q,
// and r_old = 0 before the first update, Alg. 4), and delta_i = z^T r.
__global__ void __launch_bounds__(256) k_dot2_beta(long n, const double* __restrict__ z,
                                                   const double* __restrict__ r, const double* __restrict__ q,
                                                   double* __restrict__ part, PcgState st) {
  pdl_enter();
  __shared__ double sred[kRedThreads];
  __shared__ int am_last;
  const int k = blockIdx.y;
  double a = 0.0, b = 0.0;
  if (st.flags[2 * k] == 0) {
    long lo, hi;
    segment(st, n, k, lo, hi);
    for (long i0 = pass_base(lo); i0 < hi; i0 += pass_step()) {
      double zv[kU], qv[kU], rv[kU];
#pragma unroll
      for (int j = 0; j < kU; ++j) {
        const long i = i0 + j * kB;
        const bool in = i < hi;
        zv[j] = in ? z[i] : 0.0;
        qv[j] = in ? q[i] : 0.0;
        rv[j] = in ? r[i] : 0.0;
      }
#pragma unroll
      for (int j = 0; j < kU; ++j) {
        a += zv[j] * qv[j];
        b += zv[j] * rv[j];
      }
    }
  }
  const double sa = block_sum_w0(a, sred);
  const double sb = block_sum_w0(b, sred);
  if (threadIdx.x == 0) {
    part[(long)k * gridDim.x + blockIdx.x] = sa;
    part[(long)(st.nb + k) * gridDim.x + blockIdx.x] = sb;
    __threadfence();
    const unsigned ticket = atomicAdd(st.ticket, 1u);
    am_last = ticket == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  pcg_beta_finish(part, gridDim.x, st, sred);
}

// per problem k: part[k G + c] = sum z.(r - r_old), part[(nb + k) G + c] = sum z.r
__global__ void __launch_bounds__(256) k_dot2(long n, const double* __restrict__ z, const double* __restrict__ r,
                                              const double* __restrict__ r_old, double* __restrict__ part,
                                              PcgState st) {
  pdl_enter();
  __shared__ double sred[kRedThreads];
  const int k = blockIdx.y;
  long lo, hi;
  segment(st, n, k, lo, hi);
  double a = 0.0, b = 0.0;
  for (long i0 = pass_base(lo); i0 < hi; i0 += pass_step()) {
    double zv[kU], rv[kU], ov[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const long i = i0 + j * kB;
      const bool in = i < hi;
      zv[j] = in ? z[i] : 0.0;
      rv[j] = in ? r[i] : 0.0;
      ov[j] = in ? r_old[i] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      a += zv[j] * (rv[j] - ov[j]);
      b += zv[j] * rv[j];
    }
  }
  const double sa = block_sum_w0(a, sred);
  const double sb = block_sum_w0(b, sred);
  if (threadIdx.x == 0) {
    part[(long)k * gridDim.x + blockIdx.x] = sa;
    part[(long)(st.nb + k) * gridDim.x + blockIdx.x] = sb;
  }
}

// i = iter[1], problem k (live only): beta = z.(r - r_old) / delta_{i-1};
// delta_i = z.r;  p = z + beta p;  r_old = r
__global__ void __launch_bounds__(256) k_update_p(long n, const double* __restrict__ z, double* __restrict__ p,
                                                  const double* __restrict__ r, double* __restrict__ r_old,
                                                  const double* __restrict__ part, int np, PcgState st) {
  pdl_enter();
  __shared__ double sred[kRedThreads];
  __shared__ double s_beta;
  const int k = blockIdx.y;
  if (st.flags[2 * k]) return;
  const int it = st.iter[1];
  const double zd = sum_partials(part + (long)k * np, np, sred);
  const double zr = sum_partials(part + (long)(st.nb + k) * np, np, sred);
  if (threadIdx.x == 0) {  // one division per CTA (FP64-pipe bound kernel)
    s_beta = zd / st.delta[(long)k * st.stride + it - 1];
    if (blockIdx.x == 0) {
      st.beta[(long)k * st.stride + it] = s_beta;
      st.delta[(long)k * st.stride + it] = zr;
    }
  }
  __syncthreads();
  const double beta = s_beta;
  long lo, hi;
  segment(st, n, k, lo, hi);
  for (long i0 = pass_base(lo); i0 < hi; i0 += pass_step()) {
    double zv[kU], pv[kU], rv[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const long i = i0 + j * kB;
      const bool in = i < hi;
      zv[j] = in ? z[i] : 0.0;
      pv[j] = in ? p[i] : 0.0;
      rv[j] = in ? r[i] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const long i = i0 + j * kB;
      if (i < hi) {
        p[i] = zv[j] + beta * pv[j];
        r_old[i] = rv[j];
      }
    }
  }
}

// start of Alg. 4 per problem: p = z (= MG(0, r_0)), delta_0 = p.r, r_old = 0,
// rr_0 (nrr residual partials per problem), r_max
__global__ void __launch_bounds__(256) k_start(long n, const double* __restrict__ z, const double* __restrict__ r,
                                               double* __restrict__ p, double* __restrict__ r_old,
                                               const double* __restrict__ part_zr, int nzr,
                                               const double* __restrict__ part_rr, int nrr, PcgState st,
                                               double tol) {
  pdl_enter();
  __shared__ double sred[kRedThreads];
  const int k = blockIdx.y;
  const double zr = sum_partials(part_zr + (long)(st.nb + k) * nzr, nzr, sred);
  const double rr = sum_partials(part_rr + (long)k * nrr, nrr, sred);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st.delta[(long)k * st.stride] = zr;
    st.rr[(long)k * st.stride] = rr;
    st.rmax[k] = tol * sqrt(rr);
    const bool broken = bad(rr) || bad(zr);
    const int done = (broken || rr == 0.0) ? 1 : 0;
    st.flags[2 * k] = done;
    st.flags[2 * k + 1] = broken ? 2 : 0;
    st.iters[k] = 0;
    atomicAdd(st.active, done ? 0 : 1);
  }
  long lo, hi;
  segment(st, n, k, lo, hi);
  for (long i = lo + blockIdx.x * (long)blockDim.x + threadIdx.x; i < hi; i += (long)gridDim.x * blockDim.x) {
    p[i] = z[i];
    r_old[i] = 0.0;
  }
}

// reset the lockstep counters before k_start
__global__ void k_reset(PcgState st) {
  pdl_enter();
  st.iter[0] = 1;
  st.iter[1] = 0;
  *st.ticket = 0u;
  *st.active = 0;
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_convert(long n, const TA* __restrict__ a, TB* __restrict__ b) {
  pdl_enter();
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    b[i] = convert_to<TB>(a[i]);
}

__global__ void __launch_bounds__(256) k_axpy(long n, double alpha, const double* __restrict__ x,
                                              double* __restrict__ y) {
  pdl_enter();
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] += alpha * x[i];
}

__global__ void __launch_bounds__(256) k_sub_mean(long n, double* __restrict__ b, const double* __restrict__ part,
                                                  int np, double count) {
  pdl_enter();
  __shared__ double sred[kRedThreads];
  __shared__ double s_mu;
  const double sum = sum_partials(part, np, sred);
  if (threadIdx.x == 0) s_mu = sum / count;  // one division per CTA
  __syncthreads();
  const double mu = s_mu;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) b[i] -= mu;
}

__global__ void __launch_bounds__(256) k_norm2(long n, const double* __restrict__ x, double* __restrict__ part) {
  pdl_enter();
  __shared__ double sred[kRedThreads];
  double a = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    a += x[i] * x[i];
  const double s = block_sum_w0(a, sred);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// problem k of nmem: (rows + 1) x Nx nodes, walls (first / last row and
// column) written as 0
__global__ void __launch_bounds__(256) k_stack_in(const double* const* __restrict__ srcs, const double* one,
                                                  double* __restrict__ stack, int rows, int Nx, long seg_len) {
  pdl_enter();
  const int k = blockIdx.y;
  const double* src = srcs ? srcs[k] : one;
  const long per = (long)(rows + 1) * Nx;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < per; i += (long)gridDim.x * blockDim.x) {
    const int row = (int)(i / Nx), col = (int)(i - (long)row * Nx);
    const bool wall = row == 0 || row == rows || col == 0 || col == Nx - 1;
    stack[(long)k * seg_len + i] = wall ? 0.0 : src[i];
  }
}

__global__ void __launch_bounds__(256) k_stack_out(const double* __restrict__ stack, double* const* __restrict__ dsts,
                                                   double* one, int rows, int Nx, long seg_len) {
  pdl_enter();
  const int k = blockIdx.y;
  double* dst = dsts ? dsts[k] : one;
  const long per = (long)(rows + 1) * Nx;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < per; i += (long)gridDim.x * blockDim.x)
    dst[i] = stack[(long)k * seg_len + i];
}

}  // namespace

cudaError_t launch_stack_in(const double* const* srcs, const double* one, double* stack, int nmem, int rows, int Nx,
                            long seg_len, cudaStream_t s) {
  const long per = (long)(rows + 1) * Nx;
  dim3 grid((unsigned)std::max<long>(1, std::min<long>((per + 255) / 256, 1024)), nmem);
  {
    const cudaError_t e_ = launch_pdl(k_stack_in, dim3(grid), dim3(256), 0, s, srcs, one, stack, rows, Nx, seg_len);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_stack_out(const double* stack, double* const* dsts, double* one, int nmem, int rows, int Nx,
                             long seg_len, cudaStream_t s) {
  const long per = (long)(rows + 1) * Nx;
  dim3 grid((unsigned)std::max<long>(1, std::min<long>((per + 255) / 256, 1024)), nmem);
  {
    const cudaError_t e_ = launch_pdl(k_stack_out, dim3(grid), dim3(256), 0, s, stack, dsts, one, rows, Nx, seg_len);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

int elementwise_grid(long n) { return (int)std::max<long>(1, std::min<long>((n + 255) / 256, kElemGrid)); }

int chunk_grid(const PcgState& st) {
  const long per = st.seg_len;
  const int g = (int)std::max<long>(1, std::min<long>((per + 255) / 256, std::max(4, kElemGrid / st.nb)));
  return std::min(g, kMaxPartials / std::max(1, 2 * st.nb));
}

cudaError_t launch_pcg_update_ur_check(long n, double* u, double* r, double* p, const double* q,
                                       const double* part_pq, int npq, PcgState st, double* part_rr, int i_max,
                                       cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s,
                                       const double* z, float* r32) {
  dim3 grid(chunk_grid(st), st.nb);
  {
    const cudaError_t e_ = launch_pdl(k_update_ur_check, dim3(grid), dim3(kB), 0, s, n, u, r, p, q, part_pq, npq, st, part_rr, i_max, cond, use_cond, z, r32);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_dot2_beta(long n, const double* z, const double* r, const double* q, double* part, PcgState st,
                             cudaStream_t s) {
  dim3 grid(chunk_grid(st), st.nb);
  {
    const cudaError_t e_ = launch_pdl(k_dot2_beta, dim3(grid), dim3(kB), 0, s, n, z, r, q, part, st);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_dot2(long n, const double* z, const double* r, const double* r_old, double* part, PcgState st,
                        cudaStream_t s) {
  dim3 grid(chunk_grid(st), st.nb);
  {
    const cudaError_t e_ = launch_pdl(k_dot2, dim3(grid), dim3(kB), 0, s, n, z, r, r_old, part, st);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_pcg_update_p(long n, const double* z, double* p, const double* r, double* r_old,
                                const double* part, PcgState st, cudaStream_t s) {
  dim3 grid(chunk_grid(st), st.nb);
  {
    const cudaError_t e_ = launch_pdl(k_update_p, dim3(grid), dim3(kB), 0, s, n, z, p, r, r_old, part, grid.x, st);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_pcg_start(long n, const double* z, const double* r, double* p, double* r_old,
                             const double* part_zr, const double* part_rr, int nrr, PcgState st, double tol,
                             cudaStream_t s) {
  {
    const cudaError_t e_ = launch_pdl(k_reset, dim3(1), dim3(1), 0, s, st);
    if (e_ != cudaSuccess) return e_;
  }
  dim3 grid(chunk_grid(st), st.nb);
  {
    const cudaError_t e_ = launch_pdl(k_start, dim3(grid), dim3(256), 0, s, n, z, r, p, r_old, part_zr, grid.x, part_rr, nrr, st, tol);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

template <typename TA, typename TB>
cudaError_t launch_convert(long n, const TA* a, TB* b, cudaStream_t s) {
  {
    const cudaError_t e_ = launch_pdl(k_convert<TA, TB>, dim3(elementwise_grid(n)), dim3(256), 0, s, n, a, b);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(long, const double*, float*, cudaStream_t);
template cudaError_t launch_convert<float, double>(long, const float*, double*, cudaStream_t);

cudaError_t launch_axpy(long n, double alpha, const double* x, double* y, cudaStream_t s) {
  {
    const cudaError_t e_ = launch_pdl(k_axpy, dim3(elementwise_grid(n)), dim3(256), 0, s, n, alpha, x, y);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_sub_mean(long n, double* b, const double* part, int np, cudaStream_t s) {
  {
    const cudaError_t e_ = launch_pdl(k_sub_mean, dim3(elementwise_grid(n)), dim3(256), 0, s, n, b, part, np, (double)n);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_norm2(long n, const double* x, double* part, cudaStream_t s) {
  {
    const cudaError_t e_ = launch_pdl(k_norm2, dim3(elementwise_grid(n)), dim3(256), 0, s, n, x, part);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

}  // namespace sem
