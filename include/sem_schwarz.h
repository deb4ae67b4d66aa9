/*
 * sem_schwarz.h - C ABI of the GB300 library for the hybrid Schwarz/multigrid
 * spectral-element Poisson solver of J. Stiller, "Nonuniformly weighted Schwarz
 * smoothers for spectral element multigrid" (J. Sci. Comput.).
 *
 * The library solves the 2D spectral-element system A u = f of Sec. 2
 * (Eq. (discrete), Eq. (system matrix): A = M_y (x) L_x + L_y (x) M_x on a
 * Cartesian mesh of n_x x n_y elements of order p) with
 *   - the weighted additive Schwarz smoother of Sec. 3.1 (Alg. 2),
 *   - the p-multigrid V-cycle of Sec. 3.2 (Alg. 3),
 *   - the inexact multigrid-preconditioned CG (MGCG) of Sec. 3.3 (Alg. 4).
 *
 * Conventions shared by every call
 * --------------------------------
 *  Vectors.  A field is the full node grid of the finest level, row-major with
 *    x fastest: ny_nodes rows of nx_nodes doubles (sem_sizes).  With Dirichlet
 *    walls the grid includes the wall nodes; their input values are ignored and
 *    the library writes 0 there.  Periodic grids have n_x p x n_y p nodes.
 *    Unless a call says otherwise, vector pointers are DEVICE pointers owned by
 *    the caller, valid on the handle's device, 8-byte aligned, non-overlapping.
 *  Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls marked "async" only enqueue work on that stream; calls
 *    marked "sync" return after the work has finished.
 *  Ownership.  The handle owns every workspace; no call allocates device memory
 *    after sem_create returns.  Handles are not thread-safe: one host thread and
 *    one stream at a time per handle.
 *  Errors.  Every call returns a sem_status.  Nothing aborts and no exception
 *    crosses the ABI.  sem_last_error() gives a message for the calling thread.
 *    There is no CPU fallback: without a usable CUDA device sem_create fails.
 */
#ifndef SEM_SCHWARZ_H
#define SEM_SCHWARZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sem_status {
  SEM_OK = 0,
  SEM_NOT_CONVERGED = 1, /* i_max reached before the residual test passed     */
  SEM_BREAKDOWN = 2,     /* p^T q <= 0, or a NaN/Inf in a reduction           */
  SEM_TIMEOUT = 3,       /* a bounded device wait gave up                     */
  SEM_BAD_ARG = 4,       /* invalid configuration or argument                 */
  SEM_CUDA_ERROR = 5,    /* a CUDA runtime call failed                         */
  SEM_OOM = 6            /* device allocation failed in sem_create           */
} sem_status;

/* Weight functions of Table (weighting), Sec. 3.1.  SEM_W_ARITH is the
 * arithmetic mean W = R_s C^+ R_s^T; SEM_W_IDENTITY is W = I (classical
 * additive Schwarz). */
typedef enum sem_weight {
  SEM_W_LINEAR = 1,
  SEM_W_CUBIC = 3,
  SEM_W_QUINTIC = 5,
  SEM_W_SEPTIC = 7,
  SEM_W_TOPHAT = 100,
  SEM_W_ARITH = 101,
  SEM_W_IDENTITY = 102,
  SEM_W_LEARNED = 103   /* per-interface (s, kt) from sem_config.learned_x/y */
} sem_weight;

/* Overlap n_{o,l} per level (Sec. 4): a fixed count, floor(p_l/8),
 * ceil(p_l/8) or ceil(p_l/2); always capped at p_l - 1. */
typedef enum sem_overlap_rule {
  SEM_OVERLAP_FIXED = 0,
  SEM_OVERLAP_FLOOR8 = 1,
  SEM_OVERLAP_CEIL8 = 2,
  SEM_OVERLAP_CEIL2 = 3
} sem_overlap_rule;

/* Smoother of the V-cycle (Sec. 3.1, Alg. 3).
 *   SEM_SMOOTH_ADDITIVE  weighted additive Schwarz, Alg. 2 (the default).
 *   SEM_SMOOTH_MULT      multiplicative Schwarz, Alg. 1: the subdomains one
 *                        after another, the residual recomputed before each
 *                        local solve, the local solution added on the
 *                        element's own closed node set without weights; the
 *                        order of every second sweep reversed.  The
 *                        subdomains are visited by colour classes (element
 *                        indices modulo q per direction: q = 3 with Dirichlet
 *                        walls, the smallest divisor q >= 3 of n when
 *                        periodic), a class at a time, instead of the paper's
 *                        lexicographic order: members of a class do not
 *                        interact, so each class is one parallel launch.
 *                        Poisson operator (nu_kind 0), FP64 or FP32
 *                        precision, one problem (not batched), n >= 3 per
 *                        direction when periodic; the weight setting is
 *                        unused. */
typedef enum sem_smoother {
  SEM_SMOOTH_ADDITIVE = 0,
  SEM_SMOOTH_MULT = 1
} sem_smoother;

/* Arithmetic of the multigrid preconditioner.  The outer MGCG iteration, the
 * operator application q = A p, the coarse solve and all dot products are
 * FP64 in every mode.
 *   SEM_PREC_FP64   the plain method, FP64 throughout.
 *   SEM_PREC_FP32   V-cycle (residuals, transfers, FDM) in FP32.
 *   SEM_PREC_TF32   as FP32, FDM contractions on tensor cores with TF32
 *                   operands and FP32 accumulation.
 *   SEM_PREC_BF16   as FP32, FDM contractions on tensor cores with BF16
 *                   operands and FP32 accumulation. */
typedef enum sem_precision {
  SEM_PREC_FP64 = 0,
  SEM_PREC_FP32 = 1,
  SEM_PREC_TF32 = 2,
  SEM_PREC_BF16 = 3
} sem_precision;

typedef struct sem_config {
  int32_t nx, ny;          /* elements per direction (>= 2)                      */
  int32_t p;               /* polynomial order, a power of two in [2, 32]        */
  int32_t periodic;        /* 1: periodic in x and y; 0: homogeneous Dirichlet   */
  double lx, ly;           /* domain [0, lx] x [0, ly] (uniform meshes)          */
  const double* x_edges;   /* optional host array of nx+1 increasing x edges     */
  const double* y_edges;   /* optional host array of ny+1 increasing y edges     */
  int32_t overlap_rule;    /* sem_overlap_rule                                   */
  int32_t overlap;         /* n_o for SEM_OVERLAP_FIXED                          */
  int32_t weight;          /* sem_weight                                         */
  int32_t ns1, ns2;        /* pre-/post-smoothing steps per level (Alg. 3)       */
  int32_t variable_cycle;  /* 1: n_{s,l} doubles per coarser level (Sec. 4.2)    */
  int32_t precision;       /* sem_precision                                      */
  double tol;              /* MGCG stops when ||r_i|| <= tol * ||r_0||           */
  int32_t i_max;           /* MGCG iteration limit                               */
  /* Variable diffusivity (Sec. 4.3, Eq. (diffusion)): -div(nu grad u) = f.
   * nu_kind 0: Poisson (nu = 1).  1: nu = 1 + (a-1)(1/2 + 1/2 sin 2 pi x cos 2 pi y),
   * contrast a.  2: nu = 1 + a sin 2 pi (x-b) sin 2 pi (y-b) (the paper's study).
   * nu is evaluated at the GLL nodes of every level; the residual uses B(nu),
   * the local solves are divided by the element mean nu_bar_s
   * (Eq. (subproblem:solution)) and the coarse problem is solved with a dense
   * FP64 inverse of B_0(nu) (periodic meshes: its pseudo-inverse, at most
   * 32 x 32 elements). */
  int32_t nu_kind;
  double nu_a, nu_b;
  /* SEM_W_LEARNED: optional HOST arrays [level 0..L][interface 0..n][2] of
   * (s, kt) per interface line (interface i between elements i-1 and i;
   * entries of wall interfaces are ignored).  The transition of Eq. (weight
   * function) at the interface has half width s delta_O min(h_left, h_right)/2
   * (s in (0, 1]) and shape degree kt in [1, 7], a convex blend of the
   * neighbouring odd degrees of Table (weighting).  Both sides of an
   * interface use the same pair, so the weights keep the partition of unity. */
  const double* learned_x;
  const double* learned_y;
  int32_t smoother;        /* sem_smoother (default SEM_SMOOTH_ADDITIVE)          */
  /* SEM_W_LEARNED with learned_x and learned_y both NULL: optional HOST array
   * of SEM_MLP_PARAMS floats, the parameters of the weight network (layout
   * below).  sem_create then computes the interface features
   * (sem_learned_features), runs the network's forward kernel on the device
   * and uses its (s, kt) outputs as learned_x / learned_y. */
  const float* mlp_params;
} sem_config;

typedef struct sem_result {
  int32_t iterations;      /* i at exit of Alg. 4 (or V-cycles of sem_mg_solve)   */
  int32_t status;          /* sem_status of the solve                            */
  double res0;             /* ||r_0||_2                                          */
  double res;              /* ||r_i||_2 at exit (recursively updated residual)   */
  double rbar;             /* log10(res0 / res) / iterations (Sec. 4)            */
} sem_result;

typedef struct sem_handle sem_handle;

/* Fill *cfg with defaults: 4x4 Dirichlet unit square, p = 4, n_o = 1, w_5,
 * additive smoother, MG(1,0) steps, FP64, tol 1e-10, i_max 200. */
void sem_default_config(sem_config* cfg);

/* Set up a solver (sync).  Host FP64 set-up of Sec. 2 and Sec. 3: GLL nodes,
 * element matrices, generalised eigenpairs of the restricted 1D pairs for the
 * fast-diagonalisation inverse (Eq. (FDM)), weights (Eq. (weight function)),
 * interpolation I_l, coarse factors; then allocates all device workspace on
 * the current CUDA device and uploads the tables.
 * Errors: SEM_BAD_ARG (invalid cfg, *out untouched), SEM_OOM, SEM_CUDA_ERROR. */
int sem_create(const sem_config* cfg, sem_handle** out);

/* Free everything the handle owns (sync).  NULL is ignored. */
void sem_destroy(sem_handle* h);

/* Node-grid layout of the finest level (host, no device work).  Any output
 * pointer may be NULL.  n_unknowns excludes Dirichlet wall nodes. */
int sem_sizes(const sem_handle* h, int64_t* n_unknowns, int64_t* nx_nodes, int64_t* ny_nodes);

/* Node coordinates of the finest level (host): x[nx_nodes], y[ny_nodes],
 * caller-owned HOST arrays. */
int sem_coords(const sem_handle* h, double* x, double* y);

/* b = M_2D f with M_2D = M_y (x) M_x, the GLL-quadrature mass (Sec. 2); the
 * discrete right side of Eq. (discrete) for nodal source values f (async).
 * Periodic grids: b is projected to zero mean (the range of A, Sec. 3.2). */
int sem_mass(sem_handle* h, const double* f_nodal, double* b, void* stream);

/* Au = A u, Eq. (system matrix), FP64, sum-factorised (async). */
int sem_apply(sem_handle* h, const double* u, double* Au, void* stream);

/* n_it sweeps of the weighted additive Schwarz method on the finest level,
 * Alg. 2: r = f - A u; u += sum_s R_s^T W A_ss^{-1} R_s r (async).  u is
 * updated in place.  Runs in the handle's precision (FP64 storage of u). */
int sem_smooth(sem_handle* h, double* u, const double* f, int32_t n_it, void* stream);

/* One multigrid V-cycle, Alg. 3 MultigridCycle(u, f, n_s), u in place (async). */
int sem_vcycle(sem_handle* h, double* u, const double* f, void* stream);

/* Stand-alone multigrid iteration MG(ns1, ns2) (sync): V-cycles until
 * ||f - A u|| <= tol ||f - A u_0|| or i_max cycles.  If history != NULL it
 * receives the residual norms of cycles 0..iterations (HOST array of
 * history_len doubles). */
int sem_mg_solve(sem_handle* h, double* u, const double* f, sem_result* res,
                 double* history, int32_t history_len, void* stream);

/* Inexact MG-preconditioned CG, Alg. 4 (sync): from the caller's u (in place)
 * until ||r_i|| <= tol ||r_0|| or i_max iterations; beta by the Polak-Ribiere
 * form z^T (r - r_old) / delta.  history as in sem_mg_solve (norms ||r_i||,
 * i = 0..iterations).  Returns res->status. */
int sem_pcg_solve(sem_handle* h, double* u, const double* f, sem_result* res,
                  double* history, int32_t history_len, void* stream);

/* Host-only inspection of the set-up tables of one level (no device work;
 * works without a GPU).  Fills *info; every array pointer may be NULL, else it
 * is a caller-owned HOST array of the size given by info (call once with NULL
 * arrays to get the sizes):
 *   tab_x[nx]                  subdomain table id of each element column
 *   S_x[n_tables_x * m * m]    padded eigenvectors (row = window slot a, the
 *                              element-local node a - n_o; column = eigen-slot)
 *   lam_x[n_tables_x * m]      eigenvalues (padding slots hold 1)
 *   w_x[n_tables_x * m]        1D weights (padding slots hold 0)
 *   coords_x[nx_nodes]         node coordinates
 * The x direction is reported; y is built by the same code.
 * Errors: SEM_BAD_ARG for an invalid cfg or level. */
typedef struct sem_level_info {
  int32_t p, n_o, m, n_tables_x, nx_nodes;
} sem_level_info;
int sem_inspect_level(const sem_config* cfg, int32_t level, sem_level_info* info, int32_t* tab_x,
                      double* S_x, double* lam_x, double* w_x, double* coords_x);

/* Host-only: the 1D GLL set of order p that every level is built from
 * (Sec. 2): nodes xi[p+1] and quadrature weights w[p+1] on [-1, 1], the
 * differentiation matrix D[(p+1)^2] (row-major, D[i*(p+1) + j] = phi_j'(xi_i))
 * and the reference stiffness L_ref[(p+1)^2], L_ref_ij = sum_q w_q D_qi D_qj
 * (an element of width h has stiffness (2/h) L_ref and mass (h/2) w).  Each
 * entry is the correctly rounded double of its exact value: the set is
 * computed in double-double arithmetic and rounded once.  Caller-owned HOST
 * arrays; any pointer may be NULL.  No device work (works without a GPU).
 * Errors: SEM_BAD_ARG for p < 1 or p > 64. */
int sem_gll_tables(int32_t p, double* xi, double* w, double* D, double* L_ref);

/* Kernel classes of the tracing counters. */
typedef enum sem_kernel_class {
  SEM_K_APPLY_FP64 = 0, /* FP64 operator / residual on the finest level (Eq. (system matrix)) */
  SEM_K_APPLY_MG = 1,   /* level residuals inside the V-cycle                               */
  SEM_K_SWEEP = 2,      /* gather + FDM + weights of Alg. 2                                 */
  SEM_K_SCATTER = 3,    /* R_s^T sum of Alg. 2                                              */
  SEM_K_RESTRICT = 4,   /* I_l^T                                                            */
  SEM_K_PROLONG = 5,    /* I_l                                                              */
  SEM_K_COARSE = 6,     /* A_0^+ (four kernels per solve)                                   */
  SEM_K_VECTOR = 7,     /* MGCG vector updates, dots, conversions                           */
  SEM_K_LOW_CYCLE = 8,  /* the levels p_l <= 8 and the coarse solve in one persistent kernel */
  SEM_K_NCLASS = 9
} sem_kernel_class;

/* Tracing.  sem_profile resets the per-class kernel-launch counters of the
 * handle and switches CUDA-event timing of every launch on (enable = 1) or off
 * (0).  With timing on, each launch is bracketed by two events on its stream
 * (adds a little host overhead).  sem_profile_read (sync on the recorded
 * events) fills ms[SEM_K_NCLASS] with the summed device time and
 * launches[SEM_K_NCLASS] with the kernel counts since sem_profile; either
 * pointer may be NULL (HOST arrays). */
int sem_profile(sem_handle* h, int32_t enable);
int sem_profile_read(sem_handle* h, double* ms, int64_t* launches);
/* The timed launches since sem_profile of one V-cycle level (1..L: the
 * level's smoothing, residual, restriction to level - 1 and prolongation
 * from level - 1; 0: the coarse solve; -1: everything outside the V-cycle,
 * e.g. the outer FP64 operator and MGCG vector updates), per class as in
 * sem_profile_read; only launches timed with profiling on are counted. */
int sem_profile_read_level(sem_handle* h, int32_t level, double* ms, int64_t* launches);

/* ---- launch-shape autotuning --------------------------------------------------
 * Not in the paper: launch choices per level l = 1..log2(p) that change the
 * speed of Alg. 3 (fuse and spw leave the results bitwise the same; tc changes
 * only the rounding order of the reduced-precision local solves):
 *   fuse  with one pre-smoothing step, the down-sweep of the V-cycle writes the
 *         Schwarz corrections E_s, and ONE residual kernel assembles
 *         u_l = sum_s R_s^T E_s itself (Eq. (correction:global), same order of
 *         summation as the scatter kernel), writes u_l and r_l = f_l - A_l u_l.
 *         Saves a launch and a pass over u_l; costs re-assembly of u_l at the
 *         halos of the residual's tiles (worth it at small p_l only).
 *   tc    reduced-precision sweep (TF32 / BF16): 1 = on the tcgen05 tensor
 *         cores, floor(128 / m) subdomains that share their factor tables
 *         stacked per MMA (available where the stacks are at least half
 *         full: uniform or one-direction-stretched meshes); 0 = mma.sync with
 *         one subdomain per warp at a time.
 *   spw   mma.sync sweep: subdomains per warp (sets the grid size; a warp
 *         that loops reuses its factor tables).
 *   eo    form of the level residual: -1 the even-odd sum factorisation in
 *         FP64 and the plain one in FP32, 0 plain, 1 even-odd (p_l >= 4); the
 *         two forms round differently (the results agree to the precision).
 * Defaults (no tuning): fuse 0, tc 1 where available, spw 1, eo -1.  sem_autotune (sync) times every
 * candidate on the handle's own level vectors (best of 3 x 10 steps, CUDA
 * events) and keeps the fastest; with cache_path != NULL it first looks each
 * level up in that JSON-lines file (key: device name, p_l, n_o, precision,
 * operator kind, element grid) and stores what it measured.  Tuning or setting
 * a level discards the captured solve graph; the next solve captures a new one.
 * It overwrites the level work vectors and the MGCG residual (no solve may be
 * in flight on the handle). */
typedef struct sem_level_tune {
  int32_t fuse;         /* 0 or 1 */
  int32_t spw;          /* 1..64 */
  int32_t tc;           /* 0 or 1 */
  int32_t tc_available; /* sem_get_tune: 1 if the level has tcgen05 stacks (ignored by sem_set_tune) */
  int32_t eo;           /* -1, 0 or 1 */
  double us;            /* measured time of the level's down-sweep step (microseconds; 0 if not timed) */
} sem_level_tune;
int sem_autotune(sem_handle* h, const char* cache_path, void* stream);
/* The lower part of the V-cycle as ONE persistent cooperative kernel (not in
 * the paper): on levels 1 .. min(log2(p) - 1, 3) one Schwarz step from zero
 * (tensor-core sweep, scatter fused into the residual), the restrictions, the
 * FP32 coarse solve and the prolongations, with grid barriers instead of kernel
 * boundaries.  Available for the TF32 / BF16 modes of the Poisson operator with
 * one pre-smoothing step and no post-smoothing, windows m <= 16 and coarse
 * grids of at most 64 x 64 unknowns.  Off by default: measured on one GB300 it
 * loses to the per-level kernels replayed from the solve graph (64 x 64, p = 16:
 * 2.69 against 2.31 ms per solve; 14 grid barriers at 2 CTAs per SM cost more
 * than the launch gaps they remove); sem_autotune turns it on where it wins.
 * A grid barrier that waits more than about a second makes the next
 * synchronous solve return SEM_TIMEOUT.  sem_set_low_cycle(h, 1) fails with
 * SEM_BAD_ARG where it is not available; both calls discard the captured graph. */
int sem_set_low_cycle(sem_handle* h, int32_t enable);
int sem_get_low_cycle(const sem_handle* h, int32_t* available, int32_t* enabled);
/* The up-leg of the V-cycle (Alg. 3) in ONE launch.  With no post-smoothing
 * on any level the up-leg is u_l <- u_l + I_l u_{l-1}, l = 1 .. L, and every
 * level has the same element mesh, so one kernel takes each tile of elements
 * from the coarse solution through all levels in shared memory and writes only
 * the finest level's z (with the fused dot products of the MGCG update where
 * the level-by-level path has them).  Results are identical, bit for bit, to
 * the level-by-level prolongations (the end rows of the interpolation tables
 * are exactly 0 and 1, so a node shared by two tiles gets the same value from
 * either); u_1 .. u_{L-1} are left as the down-leg wrote them.  Available when
 * p >= 4 and ns2 = 0 (also under variable_cycle); on by default; not used
 * while the persistent low-level cycle is on.  sem_set_fused_prolongation(h,
 * 1) fails with SEM_BAD_ARG where it is not available; both calls discard the
 * captured graph. */
int sem_set_fused_prolongation(sem_handle* h, int32_t enable);
int sem_get_fused_prolongation(const sem_handle* h, int32_t* available, int32_t* enabled);
/* The FP64 operator of Eq. (system matrix) (the outer MGCG operator of
 * Alg. 4, sem_apply, the residuals of sem_mg_solve) evaluated exactly in
 * integer arithmetic.  Each tile of u becomes 53-bit fixed point with one
 * power-of-two scale; each element matrix becomes exact 75-bit fixed point
 * (built once at sem_create; exact while an element's entries span at most 20
 * binary exponents, as the GLL stiffness matrices do); the even-odd products
 * are summed exactly in 64-bit integers on the integer pipe (the GPU's FP64
 * pipe is ~30x slower than its 32-bit integer multiply-add) and each
 * directional sum is rounded to FP64 once, to nearest.  The only other
 * rounding is the fixed-point step of u (2^-53 of a tile's largest |u|), so
 * the result is at least as accurate as the FP64 evaluation.  Available for the
 * Poisson operator at p >= 4 when every element matrix is centro-symmetric
 * (uniform and stretched meshes); on by default.  A tile that holds a
 * non-finite value writes NaN on its nodes.  sem_set_fixed_point_operator(h,
 * 1) fails with SEM_BAD_ARG where it is not available; both calls discard the
 * captured graph. */
int sem_set_fixed_point_operator(sem_handle* h, int32_t enable);
int sem_get_fixed_point_operator(const sem_handle* h, int32_t* available, int32_t* enabled);
int sem_get_tune(const sem_handle* h, int32_t level, sem_level_tune* t);
int sem_set_tune(sem_handle* h, int32_t level, const sem_level_tune* t);

/* Allocation-free Schwarz correction.  The paper has no counterpart: this is a
 * deployment variant of the weighted additive correction
 *     u += sum_s R_s^T W A_ss^{-1} R_s r
 * for callers that cannot call cudaMalloc: code that runs inside a host
 * framework which owns the device memory through its own pool and forbids
 * other allocators, code with a fixed memory budget, and latency-critical
 * loops in which cudaMalloc/cudaFree would synchronise the device.  It needs
 * no sem_handle and allocates nothing (no cudaMalloc, cudaFree or allocating
 * library call); the caller passes every input and output.
 *
 * Tables (one per direction, DEVICE arrays owned by the caller, in the layout
 * sem_inspect_level reports for level log2(p)): tab[n] table id per element,
 * S[tables * m * m], lam[tables * m], w[tables * m], m = p + 1 + 2 n_o.  The
 * two directions must agree on p, n_o and periodic.  r and u are DEVICE node
 * grids of (n_y p [+1]) x (n_x p [+1]) doubles as for the other calls; u is
 * updated in place (async on `stream`).
 *
 * Scratch: the element-blocked corrections (n_x n_y m^2 doubles) live in one
 * static device array of 2^21 doubles (16 MiB) that every GPU loading this
 * library holds until the process exits.  Larger problems are rejected with
 * SEM_BAD_ARG and a message giving the size needed, and so are windows whose
 * FP64 local solve (8 (4 m^2 + 4 m) bytes) exceeds the device's shared memory
 * per block.  The first call on a device (with that device current) looks up
 * the array's device address with cudaGetSymbolAddress and keeps it; make
 * that first call before any stream capture.  cudaDeviceReset frees the array
 * with the context: after a reset of a device, do not call this function on it
 * again in the same process.  All
 * calls share the array and it keeps the last call's contents (every entry a
 * call reads is first written by the same call, so nothing needs clearing);
 * calls that overlap on the GPU, e.g. on two streams at once, race on it.
 * Errors: SEM_BAD_ARG, SEM_CUDA_ERROR (message in sem_last_error). */
typedef struct sem_sweep_tables {
  int32_t n;           /* elements in this direction                            */
  int32_t p;           /* polynomial order (power of two in [2, 32])            */
  int32_t n_o;         /* overlap layers, 0 <= n_o <= p - 1                     */
  int32_t periodic;    /* 1 periodic, 0 Dirichlet walls                         */
  const int32_t* tab;  /* DEVICE: n table ids                                   */
  const double* S;     /* DEVICE: tables x m x m padded eigenvectors            */
  const double* lam;   /* DEVICE: tables x m eigenvalues                        */
  const double* w;     /* DEVICE: tables x m weights                            */
} sem_sweep_tables;
int sem_schwarz_correction_noalloc(const sem_sweep_tables* x, const sem_sweep_tables* y, const double* r,
                                   double* u, void* stream);

/* ---- learned weights: the MLP of the interface-line parameters -------------
 * Not in the paper: a small FP32 network (4 -> 64 -> 64 -> 2, ReLU) maps the
 * features of an interface line to the parameters (s, kt) of
 * SEM_W_LEARNED, trained on convergence rates that the plain method measures
 * in parameter sweeps; the quintic weights w_5 (s = 1, kt = 5) stay the
 * fallback.  Parameter vector: SEM_MLP_PARAMS floats, W1 (64x4), b1 (64),
 * W2 (64x64), b2 (64), W3 (2x64), b3 (2), row-major.  All pointers are DEVICE
 * pointers; calls are async on `stream`.  Loss L = (1/2N) sum (o - t)^2.
 * Errors: SEM_BAD_ARG, SEM_CUDA_ERROR. */
#define SEM_MLP_PARAMS 4610
/* Features per interface line (host, no device work), written for every
 * level 0..L and interface 0..n of each direction ([level][interface][4]):
 * log2(p_l)/5, delta_O/2, log2(AR)/5 with AR the largest element aspect
 * ratio next to the line, log10(rho)/2 with rho the largest ratio of element
 * mean diffusivities across the line.  Caller-owned HOST arrays. */
int sem_learned_features(const sem_config* cfg, float* feat_x, float* feat_y);
/* Y[n][2] = network outputs for X[n][4]; transform = 1 maps them to
 * (s, kt) = (0.25 + 0.75 sigmoid(o0), 1 + 6 sigmoid(o1)). */
int sem_mlp_forward(const float* params, const float* X, int32_t n, float* Y, int32_t transform, void* stream);
/* Learned weights from the network, on an existing handle (sync): the
 * handle is rebuilt as if sem_create had been called with its configuration,
 * weight SEM_W_LEARNED and mlp_params = params (HOST array of SEM_MLP_PARAMS
 * floats): interface features, one forward pass of the network on the device,
 * (s, kt) per interface line and level, new weight tables.  The handle keeps
 * its address; its captured solve graph and launch tuning are discarded.
 * Errors: SEM_BAD_ARG (a handle of a batch, variable-cycle options that the
 * learned weights do not support), SEM_CUDA_ERROR, SEM_OOM; on an error the
 * handle is unchanged. */
int sem_mlp_load(sem_handle* h, const float* params);
/* Bytes of the caller-provided workspace for n samples. */
int64_t sem_mlp_workspace_bytes(int32_t n);
/* grad[SEM_MLP_PARAMS] and *loss (DEVICE) of the mean-squared loss against
 * targets T[n][2] (backpropagation, deterministic reduction over samples). */
int sem_mlp_loss_grad(const float* params, const float* X, const float* T, int32_t n, float* grad, float* loss,
                      void* workspace, void* stream);
/* `steps` full-batch Adam steps (lr, beta = 0.9 / 0.999, eps 1e-8) from step
 * count step0; adam_m / adam_v hold the moments (zero at the start);
 * loss_hist (DEVICE, may be NULL) receives the loss before each step. */
int sem_mlp_train(float* params, float* adam_m, float* adam_v, const float* X, const float* T, int32_t n,
                  int32_t steps, float lr, int32_t step0, float* loss_hist, void* workspace, void* stream);

/* ---- batched solves ----------------------------------------------------------
 * Not in the paper: many independent problems solved by Alg. 4 at once.
 * Problems with identical uniform Dirichlet Poisson configurations (same mesh,
 * p, overlap, weights, precision, tol, i_max) are stacked along y into one
 * grid separated by wall rows, so every level kernel serves the whole group;
 * each problem keeps its own MGCG scalars, residual test and iteration count.
 * Other configurations form groups of one.  From the second sem_batch_solve
 * on, all groups run as parallel branches of ONE captured CUDA graph (one
 * launch; a WHILE node per group loops until its last problem converged).
 * The batch owns all workspace; sem_batch_solve allocates nothing. */
typedef struct sem_batch sem_batch;
/* Set up n problems (sync).  Periodic problems are rejected (SEM_BAD_ARG). */
int sem_batch_create(const sem_config* cfgs, int32_t n, sem_batch** out);
void sem_batch_destroy(sem_batch* b);
/* Groups formed and total unknowns (host). */
int sem_batch_info(const sem_batch* b, int32_t* groups, int64_t* unknowns);
/* Solve all problems (sync): u[k], f[k] are the DEVICE node grids of problem k
 * (layout of a single sem_create of cfgs[k]); u in place; res[n] HOST results.
 * Returns the largest status over the problems. */
int sem_batch_solve(sem_batch* b, double* const* u, const double* const* f, sem_result* res, void* stream);
/* Kernel launches of the batch since creation (tracing, host). */
int sem_batch_launches(const sem_batch* b, int64_t* launches);
/* sem_autotune for every group of the batch (sync); the next sem_batch_solve
 * captures a new batch graph. */
int sem_batch_autotune(sem_batch* b, const char* cache_path, void* stream);

/* Name of a status code. */
const char* sem_status_string(int32_t status);

/* Last error message of the calling thread ("" if none). */
const char* sem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SEM_SCHWARZ_H */
