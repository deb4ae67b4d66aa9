// FP64 vector kernels of the inexact MG-preconditioned CG, Alg. 4.
//
// Reductions are deterministic: a producer kernel writes one partial sum per
// CTA; every CTA of the consumer kernel sums the same partials in the same
// fixed order, so all CTAs agree bit for bit on the scalar (alpha, beta,
// delta) without an extra launch or atomics.  Per-iteration scalars are kept
// in history arrays indexed by the iteration count, so a kernel that reads
// delta_{i-1} never races with the one that writes delta_i.
#include "kernels.h"

namespace sem {

namespace {

constexpr int kElemGrid = 4 * 152;

__device__ __forceinline__ bool bad(double x) { return !(fabs(x) <= 1.7976931348623157e308); }

// Sum of n partials written by other CTAs of the same launch (read through
// L2, fixed order): used by the last CTA of a launch.
__device__ __forceinline__ double sum_partials_cg(const double* part, int n, double* sbuf) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(part + i);
  return block_sum(v, sbuf);
}

// Iteration i = iter[0]:  alpha = delta_{i-1} / (p.q);  u += alpha p;
// r -= alpha q;  then the last CTA to finish reduces ||r||^2 in fixed order,
// records the scalars, sets done / status (convergence ||r|| <= r_max,
// breakdown, i_max), advances the counter and, inside a graph, sets the
// condition of the enclosing WHILE node.
__global__ void __launch_bounds__(256) k_update_ur_check(long n, double* __restrict__ u, double* __restrict__ r,
                                                         const double* __restrict__ p, const double* __restrict__ q,
                                                         const double* __restrict__ part_pq, int npq, PcgState st,
                                                         double* __restrict__ part_rr, int i_max,
                                                         cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double sred[kRedThreads];
  __shared__ int am_last;
  if (st.flags[0]) {  // finished before this iteration (zero or invalid start)
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  const int it = st.iter[0];
  const double pq = sum_partials(part_pq, npq, sred);
  const double alpha = st.delta[it - 1] / pq;
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    u[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    acc += ri * ri;
  }
  const double s = block_sum(acc, sred);
  if (threadIdx.x == 0) {
    part_rr[blockIdx.x] = s;
    __threadfence();
    const unsigned ticket = atomicAdd(st.ticket, 1u);
    am_last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  const double rr = sum_partials_cg(part_rr, gridDim.x, sred);
  if (threadIdx.x == 0) {
    st.pq[it] = pq;
    st.alpha[it] = alpha;
    st.rr[it] = rr;
    int done = 0, status = 0;
    if (bad(rr) || bad(alpha) || !(pq > 0.0)) {
      done = 1;
      status = 2;  // SEM_BREAKDOWN
    } else if (sqrt(rr) <= st.rmax[0]) {
      done = 1;
    } else if (it >= i_max) {
      done = 1;
      status = 1;  // SEM_NOT_CONVERGED
    }
    st.flags[0] = done;
    st.flags[1] = status;
    st.iter[1] = it;      // index for the rest of this iteration (beta, delta)
    st.iter[2] = it;      // iterations completed
    st.iter[0] = it + 1;  // next iteration's update
    *st.ticket = 0u;
    if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
  }
}

// part[2 cta] = sum z.(r - r_old), part[2 cta + 1] = sum z.r
__global__ void __launch_bounds__(256) k_dot2(long n, const double* __restrict__ z, const double* __restrict__ r,
                                              const double* __restrict__ r_old, double* __restrict__ part) {
  __shared__ double sred[kRedThreads];
  double a = 0.0, b = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double zi = z[i], ri = r[i];
    a += zi * (ri - r_old[i]);
    b += zi * ri;
  }
  const double sa = block_sum(a, sred);
  const double sb = block_sum(b, sred);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sa;
    part[gridDim.x + blockIdx.x] = sb;
  }
}

// i = iter[1]:  beta = z.(r - r_old) / delta_{i-1};  delta_i = z.r;
// p = z + beta p;  r_old = r
__global__ void __launch_bounds__(256) k_update_p(long n, const double* __restrict__ z, double* __restrict__ p,
                                                  const double* __restrict__ r, double* __restrict__ r_old,
                                                  const double* __restrict__ part, int np, PcgState st) {
  __shared__ double sred[kRedThreads];
  const int it = st.iter[1];
  const double zd = sum_partials(part, np, sred);
  const double zr = sum_partials(part + np, np, sred);
  const double beta = zd / st.delta[it - 1];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st.beta[it] = beta;
    st.delta[it] = zr;
  }
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    p[i] = z[i] + beta * p[i];
    r_old[i] = r[i];
  }
}

// start of Alg. 4: p = z (= MG(0, r_0)), delta_0 = p.r, r_old = 0, rr_0, r_max
__global__ void __launch_bounds__(256) k_start(long n, const double* __restrict__ z, const double* __restrict__ r,
                                               double* __restrict__ p, double* __restrict__ r_old,
                                               const double* __restrict__ part_zr, int nzr,
                                               const double* __restrict__ part_rr, int nrr, PcgState st,
                                               double tol) {
  __shared__ double sred[kRedThreads];
  const double zr = sum_partials(part_zr + nzr, nzr, sred);
  const double rr = sum_partials(part_rr, nrr, sred);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st.delta[0] = zr;
    st.rr[0] = rr;
    st.rmax[0] = tol * sqrt(rr);
    const bool broken = bad(rr) || bad(zr);
    st.flags[0] = (broken || rr == 0.0) ? 1 : 0;
    st.flags[1] = broken ? 2 : 0;
    st.iter[0] = 1;
    st.iter[1] = 0;
    st.iter[2] = 0;
    *st.ticket = 0u;
  }
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    p[i] = z[i];
    r_old[i] = 0.0;
  }
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_convert(long n, const TA* __restrict__ a, TB* __restrict__ b) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    b[i] = TB(a[i]);
}

__global__ void __launch_bounds__(256) k_axpy(long n, double alpha, const double* __restrict__ x,
                                              double* __restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] += alpha * x[i];
}

__global__ void __launch_bounds__(256) k_sub_mean(long n, double* __restrict__ b, const double* __restrict__ part,
                                                  int np, double count) {
  __shared__ double sred[kRedThreads];
  const double mu = sum_partials(part, np, sred) / count;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) b[i] -= mu;
}

__global__ void __launch_bounds__(256) k_norm2(long n, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sred[kRedThreads];
  double a = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    a += x[i] * x[i];
  const double s = block_sum(a, sred);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

}  // namespace

int elementwise_grid(long n) { return (int)std::max<long>(1, std::min<long>((n + 255) / 256, kElemGrid)); }

cudaError_t launch_pcg_update_ur_check(long n, double* u, double* r, const double* p, const double* q,
                                       const double* part_pq, int npq, PcgState st, double* part_rr, int i_max,
                                       cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
  k_update_ur_check<<<elementwise_grid(n), 256, 0, s>>>(n, u, r, p, q, part_pq, npq, st, part_rr, i_max, cond,
                                                        use_cond);
  return cudaGetLastError();
}

cudaError_t launch_dot2(long n, const double* z, const double* r, const double* r_old, double* part,
                        cudaStream_t s) {
  k_dot2<<<elementwise_grid(n), 256, 0, s>>>(n, z, r, r_old, part);
  return cudaGetLastError();
}

cudaError_t launch_pcg_update_p(long n, const double* z, double* p, const double* r, double* r_old,
                                const double* part, int np, PcgState st, cudaStream_t s) {
  k_update_p<<<elementwise_grid(n), 256, 0, s>>>(n, z, p, r, r_old, part, np, st);
  return cudaGetLastError();
}

cudaError_t launch_pcg_start(long n, const double* z, const double* r, double* p, double* r_old,
                             const double* part_zr, int nzr, const double* part_rr, int nrr, PcgState st,
                             double tol, cudaStream_t s) {
  k_start<<<elementwise_grid(n), 256, 0, s>>>(n, z, r, p, r_old, part_zr, nzr, part_rr, nrr, st, tol);
  return cudaGetLastError();
}

template <typename TA, typename TB>
cudaError_t launch_convert(long n, const TA* a, TB* b, cudaStream_t s) {
  k_convert<TA, TB><<<elementwise_grid(n), 256, 0, s>>>(n, a, b);
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(long, const double*, float*, cudaStream_t);
template cudaError_t launch_convert<float, double>(long, const float*, double*, cudaStream_t);

cudaError_t launch_axpy(long n, double alpha, const double* x, double* y, cudaStream_t s) {
  k_axpy<<<elementwise_grid(n), 256, 0, s>>>(n, alpha, x, y);
  return cudaGetLastError();
}

cudaError_t launch_sub_mean(long n, double* b, const double* part, int np, cudaStream_t s) {
  k_sub_mean<<<elementwise_grid(n), 256, 0, s>>>(n, b, part, np, (double)n);
  return cudaGetLastError();
}

cudaError_t launch_norm2(long n, const double* x, double* part, cudaStream_t s) {
  k_norm2<<<elementwise_grid(n), 256, 0, s>>>(n, x, part);
  return cudaGetLastError();
}

}  // namespace sem
