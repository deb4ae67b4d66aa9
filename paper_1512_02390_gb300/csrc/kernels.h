// Host launchers of the CUDA kernels (one translation unit per kernel family).
// Every launcher enqueues on `s` and returns the launch status.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace sem {

// Number of partial sums a reduction-producing launch writes (one per CTA).
constexpr int kMaxPartials = 1 << 17;
// Elements per direction of one operator / grid-transfer tile at order P:
// 32 x 32 owned nodes for P >= 16, 16 x 16 for P <= 8 (the lower levels are
// small and latency-bound: more, smaller CTAs).
__host__ __device__ constexpr int tile_elems(int P) { return P >= 32 ? 1 : (P <= 8 ? 16 / P : 32 / P); }
__host__ __device__ constexpr int ilog2_c(int p) { return p <= 1 ? 0 : 1 + ilog2_c(p / 2); }

// ---- sum-factorised operator (Eq. (system matrix)), k_operator.cu --------
// The MGCG direction update of Alg. 4 fused into the FP64 operator: the
// operand is z + beta_k p, beta_k = beta[k * stride + iter[1]] of the tile's
// problem k (0 once the problem is done), formed with the same fma as the
// vector update that stores p.  z == nullptr: the plain operand.
struct PcgFuse {
  const double* z = nullptr;
  const double* beta = nullptr;
  const int* flags = nullptr;
  const int* iter = nullptr;
  int stride = 0, nb = 1;
};

// eo: -1 the even-odd form in FP64 only, 0 never, 1 for P >= 4 in any type.
// out = A u (f == nullptr) or out = f - A u.  dot: 0 none, 1 part[cta] = sum
// u.out, 2 part[cta] = sum out.out over the CTA's nodes.  *nparts receives
// the number of partials written.  With E != nullptr the input u is not read:
// it is assembled on the fly as the Schwarz correction sum_s R_s^T E[s] (the
// scatter of Alg. 2 fused into the residual) and written to uout.
template <typename T, typename TF>
cudaError_t launch_apply(const DirView<T>& dx, const DirView<T>& dy, const T* u, const TF* f,
                         T* out, int dot, double* part, int* nparts, cudaStream_t s, const T* E = nullptr,
                         T* uout = nullptr, PcgFuse pf = PcgFuse(), int eo = -1);

// The FP64 operator of Eq. (system matrix) evaluated exactly in integer
// arithmetic (an error-free splitting in the manner of Ozaki et al.): each CTA
// writes its staged tile of u as 53-bit fixed point (one power-of-two scale per
// tile); the element matrices come as exact fixed-point integers (one scale per
// element and direction); the even-odd products (E = L[a][k] + L[a][p-k],
// O = L[a][k] - L[a][p-k], exact in integers) are accumulated exactly in
// 64-bit integers (6 mad.wide.s32 per term, on the integer pipe), and each
// directional sum sum_k L[i][k] u_k is rounded to FP64 once.  FxDir holds, per
// direction, the tables of setup.h fx_tables: per distinct element matrix
// E[a][k], a, k = 0..p/2 (entry k = p/2: 2 L[a][p/2]), then O[a][k], a, k <
// p/2, each entry four ints (l0, l1, l2, 0) = l2 2^50 + l1 2^25 + l0, and per
// element the index of its table; "element" n maps to an all-zero table
// (missing neighbours).
struct FxDir {
  const int* tab;   // k + 1 distinct tables of ((p/2+1)^2 + (p/2)^2) x 4 ints, the last all zero
  const int* t;     // k + 1: L_int = L * 2^t[table]
  const int* slot;  // n + 1: element e's table (slot[n]: the zero table)
};
// out = A u (f == nullptr) or f - A u, FP64 (p in {4, 8, 16, 32}); dot and pf
// as for launch_apply (no fused scatter).  A tile holding a non-finite value
// writes NaN on its nodes.
cudaError_t launch_apply_fx(const DirView<double>& dx, const DirView<double>& dy, const FxDir& fx,
                            const FxDir& fy, const double* u, const double* f, double* out, int dot, double* part,
                            int* nparts, cudaStream_t s, PcgFuse pf = PcgFuse());

// Variable-diffusivity operator B(nu) (Sec. 4.3): element data of one level.
template <typename T>
struct VarView {
  const T* Gx;  // n_e x (p+1)^2: w_j w_i J nu (2/h_x)^2
  const T* Gy;  // n_e x (p+1)^2: w_j w_i J nu (2/h_y)^2
  const T* D;   // (p+1)^2 differentiation matrix
  T* E;         // n_e x (p+1)^2 scratch: element-local products
};
// out = B u (f == nullptr) or f - B u; element-local weak form then a
// deterministic node gather; dot as for launch_apply.
template <typename T>
cudaError_t launch_apply_var(const DirView<T>& dx, const DirView<T>& dy, const VarView<T>& v, const T* u, const T* f,
                             T* out, int dot, double* part, int* nparts, cudaStream_t s);

// b = (M_y (x) M_x) f_nodal, walls 0; part[cta] = sum of b (for the periodic
// mean projection).
cudaError_t launch_mass(const DirView<double>& dx, const DirView<double>& dy, const double* f,
                        double* b, double* part, int* nparts, cudaStream_t s);

// ---- weighted additive Schwarz sweep (Alg. 2), k_schwarz.cu ---------------
// E[s] = W_s A_ss^{-1} R_s r for every subdomain s (element-blocked m x m).
// mode: 0 SIMT in T, 1 tensor cores TF32, 2 tensor cores BF16 (T = float).
// nu_inv (may be null): 1 / nu_bar_s per subdomain (Eq. (subproblem:solution)).
// spw: tensor-core modes, about spw subdomains per warp (grid size).
template <typename T, typename TIn>
cudaError_t launch_sweep(const DirView<T>& dx, const DirView<T>& dy, const TIn* r, T* E, int mode,
                         const T* nu_inv, cudaStream_t s, int spw = 1);
// Work list of the tensor-core (tcgen05) sweep of one level: groups of up to
// G = floor(128 / m) subdomains sharing their factor tables (same table id in
// x and in y); every group's first slot is used.
struct TcWork {
  const int* sub = nullptr;  // ngroups x G subdomain indices ey * n_x + ex (-1: empty slot)
  int ngroups = 0, G = 0;
  int* err = nullptr;        // set to 1 by a CTA whose wait on the tensor cores ran out
};
// The sweep of launch_sweep (mode 1 TF32, 2 BF16) with stacks of G subdomains
// per tcgen05 MMA (k_sweep_tc.cu).
template <typename TIn>
cudaError_t launch_sweep_tc(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E, int mode,
                            const float* nu_inv, const TcWork& wk, cudaStream_t s);
// u = (accum ? u : 0) + sum_s R_s^T E[s]  (deterministic node-centric sum).
template <typename T, typename TOut>
cudaError_t launch_scatter(const DirView<T>& dx, const DirView<T>& dy, const T* E, TOut* u,
                           bool accum, cudaStream_t s);

// ---- multiplicative Schwarz sweep (Alg. 1), k_mult.cu ---------------------
// Colour classes per direction of the parallel order (0: no valid colouring,
// a periodic mesh with n < 3).
int mult_colours(int n, bool periodic);
// Dynamic shared memory of one k_mult CTA at order p, window m, element size tsize.
size_t mult_smem_bytes(int p, int m, size_t tsize);
// One sweep of Alg. 1 over the level (u in place, right side f): the colour
// classes in increasing order, or decreasing when reverse; one launch per
// non-empty class (*launches receives the count).  Local solves in T.
template <typename T, typename TU, typename TF>
cudaError_t launch_mult_sweep(const DirView<T>& dx, const DirView<T>& dy, TU* u, const TF* f, bool reverse,
                              cudaStream_t s, int* launches);

// ---- grid transfer (Sec. 3.2), k_transfer.cu ------------------------------
// fc = I^T rf from order pf to pf/2 on the same mesh (coarse walls 0).
template <typename T>
cudaError_t launch_restrict(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx,
                            const DirView<T>& cy, const T* J, const T* rf, T* fc, cudaStream_t s);
// out = in + I uc (in may alias out; in == nullptr means 0).
template <typename T, typename TOut>
cudaError_t launch_prolong(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx,
                           const DirView<T>& cy, const T* J, const T* uc, const T* in, TOut* out,
                           cudaStream_t s);

// ---- coarse solve u0 = A_0^+ f0 by global fast diagonalisation ------------
struct CoarseView {
  int nux, nuy, firstx, firsty, Nx, Ny, periodic;
  int batch;       // stacked independent problems (coarse blocks)
  int block_rows;  // node rows between consecutive blocks
  const double *Sx, *Sy, *lx, *ly, *cx, *cy;
  const float *Sx32, *Sy32, *lx32, *ly32, *cx32, *cy32;  // FP32 copies (the FP32 coarse kernel)
  double* T1;  // batch x nuy x nux scratch (also holds S_y T2)
  double* T2;  // batch x nuy x nux scratch
};
// FP64: four multi-CTA products; FP32 with at most 64 x 64 unknowns: one
// cluster of 8 CTAs per problem runs all four
template <typename T>
cudaError_t launch_coarse(const CoarseView& c, const T* f0, T* u0, cudaStream_t s);
inline int coarse_launches(const CoarseView& c, bool fp32) { return (fp32 && c.nux <= 64 && c.nuy <= 64) ? 1 : 4; }
// u0 = Binv f0 over the Dirichlet unknowns with a dense FP64 inverse (variable nu)
template <typename T>
cudaError_t launch_coarse_dense(const CoarseView& c, const double* Binv, const T* f0, T* u0, cudaStream_t s);

// ---- persistent low-level V-cycle (Alg. 3 below the upper levels), k_lowcycle.cu
struct LowLevel {
  DirView<float> x, y;
  const float* J;  // interpolation from level l-1 to l (l >= 1)
  float *u, *f, *r, *E;
};
struct LowCycle {
  int top;             // highest level handled, p_top in {2, 4, 8}
  LowLevel lev[4];     // levels 0 .. top
  CoarseView coarse;   // FP32 tables, at most 64 x 64 unknowns per problem
  float* cw;           // coarse scratch, coarse.batch x 64 x 64
  unsigned* bar;       // grid barrier [arrivals, generation]; arrivals 0 between launches
  int* err;            // set to 1 when a barrier wait gave up
};
// Levels top .. 1: one Schwarz step from zero (mma.sync sweep, mode 1 TF32 /
// 2 BF16, m <= 16), residual with the scatter fused, restriction; the coarse
// solve; prolongations back to level top.  One cooperative launch; *grid
// receives its CTA count.
cudaError_t launch_low_cycle(const LowCycle& c, int mode, int top_p, int* grid, cudaStream_t s);

// ---- Krylov vector kernels (Alg. 4), k_krylov.cu -------------------------
// MGCG state of nb independent problems stacked in one node grid (nb = 1 for a
// single solve).  Problem k owns nodes [k seg_len, (k+1) seg_len) (the last
// one runs to the end); its scalars live at k * stride + i.
struct PcgState {
  int nb;            // problems
  int stride;        // i_max + 2: length of each problem's scalar history
  long seg_len;      // nodes per problem segment
  double* alpha;     // [nb][stride] per-iteration scalars
  double* beta;
  double* delta;
  double* pq;
  double* rr;
  double* rmax;      // [nb] threshold on ||r||
  int* flags;        // [nb][2]: done, status
  int* iters;        // [nb] iterations completed
  int* iter;         // [2]: index of the next update, index of the current beta (lockstep)
  unsigned* ticket;  // CTA completion counter of the fused update / check
  int* active;       // problems still iterating
};

// Polak-Ribiere step of Alg. 4 for every live problem k, from G partials of
// z.q (part[k G ..]) and of z.r (part[(nb + k) G ..]) per problem, by the last
// CTA of the launch that wrote them: beta_i = z.(r - r_old) / delta_{i-1}
// with r - r_old = -alpha_i q (z.r itself at i = 1, where r_old = 0), and
// delta_i = z.r; then the CTA counter is reset for the next launch.
__device__ __forceinline__ void pcg_beta_finish(const double* part, int G, const PcgState& st, double* sred) {
  const int it = st.iter[1];
  for (int kk = 0; kk < st.nb; ++kk) {
    const double zq = sum_partials_cg(part + (long)kk * G, G, sred);
    const double zr = sum_partials_cg(part + (long)(st.nb + kk) * G, G, sred);
    if (threadIdx.x == 0 && st.flags[2 * kk] == 0) {
      const long o = (long)kk * st.stride + it;
      const double num = it == 1 ? zr : -st.alpha[o] * zq;
      st.beta[o] = num / st.delta[o - 1];
      st.delta[o] = zr;
    }
  }
  if (threadIdx.x == 0) *st.ticket = 0u;
}

// z.q and z.r of Alg. 4's direction update, fused into the kernel that writes
// z = MG(r).  The nb problems are stacked along y, gyp tile rows each (no tile
// straddles two): the CTA in tile row by belongs to problem k = by / gyp and
// is number c of its G = gridDim.x gyp; it writes part[k G + c] and
// part[(nb + k) G + c]; the last CTA to finish runs pcg_beta_finish
// (2 nb G <= kMaxPartials).
struct PcgDot {
  const double* q;
  const double* r;
  double* part;
  PcgState st;
  int gyp;
};

// out = in + I uc as launch_prolong (double z; in may alias out), plus the
// fused z.q, z.r and beta of `dot`.  cudaErrorInvalidConfiguration when the
// tile grid needs more than kMaxPartials / 2 partials.
// CTAs (tiles) of the prolongation to order p of an nx x ny element mesh
long prolong_ctas(int p, int nx, int ny);
template <typename T>
cudaError_t launch_prolong_dot(const DirView<T>& fx, const DirView<T>& fy, const DirView<T>& cx,
                               const DirView<T>& cy, const T* J, const T* uc, const T* in, double* out,
                               const PcgDot& dot, cudaStream_t s);

// The up-leg of the V-cycle without post-smoothing (Alg. 3) in one launch:
// u_l + I_l u_{l-1} for l = 1 .. L-1 (u_0 the coarse solution), then
// out = in + I_L u_{L-1} on the finest level L (order fx.p = 2^L, table J),
// with the z.q, z.r and beta of *dot when dot != nullptr.  Each CTA carries
// its tile of elements through the levels in shared memory (the mesh is the
// same on every level); u_1 .. u_{L-1} are read, not written.  Results are
// those of the level-by-level launches, bit for bit.  fx.p in {4, 8, 16, 32}.
constexpr int kChainLevels = 6;    // levels 0 .. 5 (orders 1 .. 32)
constexpr int kChainThreads = 256;
template <typename T>
struct ProlongChain {
  DirView<T> x[kChainLevels], y[kChainLevels];  // level l: order 2^l
  const T* u[kChainLevels];                      // u_0 .. u_{L-1}
  const T* J[kChainLevels];                      // J[l]: order 2^(l-1) -> 2^l (l >= 1)
};
template <typename T>
cudaError_t launch_prolong_chain(const ProlongChain<T>& c, const DirView<T>& fx, const DirView<T>& fy, const T* J,
                                 const T* in, double* out, const PcgDot* dot, cudaStream_t s);

int elementwise_grid(long n);
// CTAs per problem of the batched vector kernels (grid = (chunks, nb))
int chunk_grid(const PcgState& st);
// z != nullptr: first p = z + beta_i p (beta_i from launch_dot2_beta), stored;
// r32 != nullptr: the updated residual is also written rounded to FP32 (the
// right side of a mixed-precision V-cycle)
cudaError_t launch_pcg_update_ur_check(long n, double* u, double* r, double* p, const double* q,
                                       const double* part_pq, int npq, PcgState st, double* part_rr, int i_max,
                                       cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s,
                                       const double* z = nullptr, float* r32 = nullptr);
// i = iter[1]: per problem beta_i = z^T (r - r_old) / delta_{i-1} with
// r - r_old = -alpha_i q (r_old = 0 at i = 1) and delta_i = z^T r, reduced by
// the last CTA and stored in the scalar histories
cudaError_t launch_dot2_beta(long n, const double* z, const double* r, const double* q, double* part, PcgState st,
                             cudaStream_t s);
cudaError_t launch_dot2(long n, const double* z, const double* r, const double* r_old,
                        double* part, PcgState st, cudaStream_t s);
cudaError_t launch_pcg_update_p(long n, const double* z, double* p, const double* r, double* r_old,
                                const double* part, PcgState st, cudaStream_t s);
// nrr: residual partials per problem (from the operator launch)
cudaError_t launch_pcg_start(long n, const double* z, const double* r, double* p, double* r_old,
                             const double* part_zr, const double* part_rr, int nrr, PcgState st, double tol,
                             cudaStream_t s);
template <typename TA, typename TB>
cudaError_t launch_convert(long n, const TA* a, TB* b, cudaStream_t s);
cudaError_t launch_axpy(long n, double alpha, const double* x, double* y, cudaStream_t s);
cudaError_t launch_sub_mean(long n, double* b, const double* part, int np, cudaStream_t s);
cudaError_t launch_norm2(long n, const double* x, double* part, cudaStream_t s);
// Copy nmem problem grids of (rows + 1) x Nx nodes into / out of a stack in
// which problem k starts at node k * seg_len; wall nodes of the stack are 0.
// srcs / dsts: DEVICE arrays of nmem pointers, or null to use `one`.
cudaError_t launch_stack_in(const double* const* srcs, const double* one, double* stack, int nmem, int rows, int Nx,
                            long seg_len, cudaStream_t s);
cudaError_t launch_stack_out(const double* stack, double* const* dsts, double* one, int nmem, int rows, int Nx,
                             long seg_len, cudaStream_t s);

}  // namespace sem
