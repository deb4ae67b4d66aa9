/*
 * sem_schwarz3d.h - C ABI of the three-dimensional extension of the hybrid
 * Schwarz/multigrid spectral-element Poisson solver (J. Stiller, "Nonuniformly
 * weighted Schwarz smoothers for spectral element multigrid").  The paper's
 * concluding section names the extension to three space dimensions as future
 * work; the method carries over one dimension up:
 *   - the operator of Eq. (system matrix) becomes
 *     A = M_z (x) M_y (x) L_x + M_z (x) L_y (x) M_x + L_z (x) M_y (x) M_x
 *     on an n_x x n_y x n_z Cartesian mesh of elements of order p;
 *   - the extended-element subdomains of Sec. 3.1 are tensor products of the
 *     1D windows, their inverse A_ss^{-1} the fast-diagonalisation product of
 *     Eq. (FDM) with three contractions on each side, the weights of
 *     Eq. (weight function) W = W_z (x) W_y (x) W_x;
 *   - Alg. 2 (weighted additive Schwarz), Alg. 3 (p-multigrid V-cycle with
 *     I_l = P_z (x) P_y (x) P_x) and Alg. 4 (MGCG) are unchanged.
 *
 * Conventions are those of sem_schwarz.h (status codes, sem_result, streams,
 * caller-owned DEVICE vectors, no CPU fallback).  A field is the full node
 * grid of the finest level, nz_nodes x ny_nodes x nx_nodes doubles, x
 * fastest; Dirichlet wall nodes are included (ignored on input, 0 on output).
 * The handle owns all workspace; no call allocates after sem3_create.
 */
#ifndef SEM_SCHWARZ3D_H
#define SEM_SCHWARZ3D_H

#include <stdint.h>

#include "sem_schwarz.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sem3_config {
  int32_t nx, ny, nz;      /* elements per direction (>= 2)                       */
  int32_t p;               /* polynomial order, a power of two in [2, 16]         */
  int32_t periodic;        /* 1: periodic in x, y and z; 0: homogeneous Dirichlet */
  double lx, ly, lz;       /* domain [0, lx] x [0, ly] x [0, lz]                  */
  int32_t overlap_rule;    /* sem_overlap_rule                                    */
  int32_t overlap;         /* n_o for SEM_OVERLAP_FIXED                           */
  int32_t weight;          /* sem_weight, not SEM_W_LEARNED                       */
  int32_t ns1, ns2;        /* pre-/post-smoothing steps per level (Alg. 3)        */
  int32_t precision;       /* SEM_PREC_FP64, or SEM_PREC_FP32 for the V-cycle     */
  double tol;              /* MGCG stops when ||r_i|| <= tol ||r_0||              */
  int32_t i_max;           /* MGCG iteration limit                                */
} sem3_config;

typedef struct sem3_handle sem3_handle;

/* Defaults: 4 x 4 x 4 Dirichlet unit cube, p = 4, n_o = 1, w_5, MG(1,0), FP64,
 * tol 1e-10, i_max 200. */
void sem3_default_config(sem3_config* cfg);

/* Set up a solver on the current CUDA device (sync): the 1D tables of every
 * direction and level (Sec. 2, Sec. 3.1), interpolation, coarse factors, and
 * all device workspace.  The m^3 window of the finest level must fit one
 * CTA's shared memory (m = p + 1 + 2 n_o <= 23 in FP64).
 * Errors: SEM_BAD_ARG, SEM_OOM, SEM_CUDA_ERROR. */
int sem3_create(const sem3_config* cfg, sem3_handle** out);
void sem3_destroy(sem3_handle* h);
/* Node-grid layout of the finest level; any pointer may be NULL (host). */
int sem3_sizes(const sem3_handle* h, int64_t* n_unknowns, int64_t* nx_nodes, int64_t* ny_nodes,
               int64_t* nz_nodes);
/* Node coordinates x[nx_nodes], y[ny_nodes], z[nz_nodes] (HOST arrays). */
int sem3_coords(const sem3_handle* h, double* x, double* y, double* z);
/* b = (M_z (x) M_y (x) M_x) f for nodal f (async); periodic: projected to zero mean. */
int sem3_mass(sem3_handle* h, const double* f_nodal, double* b, void* stream);
/* Au = A u, FP64 (async). */
int sem3_apply(sem3_handle* h, const double* u, double* Au, void* stream);
/* n_it sweeps of Alg. 2 on the finest level, u in place (async), in the
 * handle's precision. */
int sem3_smooth(sem3_handle* h, double* u, const double* f, int32_t n_it, void* stream);
/* One V-cycle of Alg. 3, u in place (async). */
int sem3_vcycle(sem3_handle* h, double* u, const double* f, void* stream);
/* Alg. 4 from the caller's u (in place) until ||r_i|| <= tol ||r_0|| or i_max
 * (sync: the host reads the dot products of every iteration).  history
 * (HOST, may be NULL) receives ||r_i||, i = 0..iterations. */
int sem3_pcg_solve(sem3_handle* h, double* u, const double* f, sem_result* res, double* history,
                   int32_t history_len, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SEM_SCHWARZ3D_H */
