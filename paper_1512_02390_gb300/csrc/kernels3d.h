// Host launchers of the kernels of the three-dimensional extension (k_3d.cu).
// Every launcher enqueues on `s` and returns the launch status.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace sem {

// The three directions of one level.
template <typename T>
struct Dir3 {
  DirView<T> x, y, z;
};

// Coarse (p = 1) fast diagonalisation: the unknowns form a compact
// nu[2] x nu[1] x nu[0] grid starting at node first[] of the N[] node grid;
// S[d] (nu x nu, columns M-orthonormal eigenvectors) and lam[d] per direction;
// singular: periodic in all directions (mode (0,0,0) dropped, mean removed).
template <typename T>
struct Coarse3 {
  int nu[3], first[3], N[3];
  int singular;
  const T* S[3];
  const T* lam[3];
};

// Partial sums written by launch3_dot (at most).
constexpr int kDot3Parts = 1024;

// out = A u (f null) or f - A u, Eq. (system matrix) in 3D.
template <typename T, typename TF>
cudaError_t launch3_apply(const Dir3<T>& d, const T* u, const TF* f, T* out, cudaStream_t s);
// b = (M_z (x) M_y (x) M_x) f_nodal, walls 0.
template <typename T>
cudaError_t launch3_mass(const Dir3<T>& d, const T* fn, T* b, cudaStream_t s);
// Dynamic shared memory of one subdomain of the 3D sweep with window m.
template <typename T>
size_t sweep3_smem_bytes(int m);
// u = (accum ? u : 0) + sum_s R_s^T W_s A_ss^{-1} R_s r (E: n_e m^3 scratch).
template <typename T, typename TOut>
cudaError_t launch3_sweep(const Dir3<T>& d, const T* r, T* E, TOut* u, bool accum, cudaStream_t s);
// out = in + I uc (in may alias out, or be null for 0).
template <typename T, typename TOut>
cudaError_t launch3_prolong(const Dir3<T>& f, const Dir3<T>& c, const T* J, const T* uc, const T* in, TOut* out,
                            cudaStream_t s);
// fc = I^T rf (Ec: n_e (p_c + 1)^3 scratch).
template <typename T>
cudaError_t launch3_restrict(const Dir3<T>& f, const Dir3<T>& c, const T* J, const T* rf, T* Ec, T* fc,
                             cudaStream_t s);
// u0 = A_0^+ f0 on the coarse node grid (w1, w2: compact scratch).
template <typename T>
cudaError_t launch3_coarse(const Coarse3<T>& cv, T* w1, T* w2, T* f0, T* u0, cudaStream_t s);
// part[0 .. *nparts) = per-CTA partial sums of a . b (fixed grid, fixed order).
cudaError_t launch3_dot(const double* a, const double* b, long n, double* part, int* nparts, cudaStream_t s);
// y = a x + b y (x null: y = b y).
cudaError_t launch3_axpby(long n, double a, const double* x, double b, double* y, cudaStream_t s);
template <typename TA, typename TB>
cudaError_t launch3_convert(long n, const TA* a, TB* b, cudaStream_t s);

}  // namespace sem
