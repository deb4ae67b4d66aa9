// Host-side FP64 set-up of the Schwarz/multigrid solver: 1D spectral basics
// (Sec. 2), subdomain factors and weights (Sec. 3.1), interpolation and coarse
// factors (Sec. 3.2).  Runs once per handle; the results are uploaded as small
// device tables.
#pragma once

#include <string>
#include <vector>

namespace sem {

struct Mesh1D {
  int n = 0;                  // elements
  bool periodic = false;
  std::vector<double> edges;  // n + 1 increasing coordinates
  int seg = 0;                // > 0: a Dirichlet wall every seg elements (stacked problems)
  double h(int e) const { return edges[e + 1] - edges[e]; }
  int nodes(int p) const { return periodic ? n * p : n * p + 1; }
  // neighbour of element e on side -1/+1; -1 at a Dirichlet wall
  int neighbour(int e, int side) const {
    int f = e + side;
    if (seg > 0 && f >= 0 && f < n && f / seg != e / seg) return -1;
    if (f >= 0 && f < n) return f;
    if (!periodic) return -1;
    return (f % n + n) % n;
  }
  // is global node g (order p) a Dirichlet wall node?
  bool wall(int g, int p) const {
    if (periodic) return false;
    return g <= 0 || g >= n * p || (seg > 0 && g % (seg * p) == 0);
  }
};

// GLL nodes and weights on [-1, 1] (Sec. 2), computed in double-double
// arithmetic and rounded once: the correctly rounded values.
void gll(int p, std::vector<double>& xi, std::vector<double>& w);
// The GLL differentiation matrix D[i*(p+1) + j] = phi_j'(xi_i), correctly rounded.
void gll_deriv(int p, std::vector<double>& D);
// Lagrange basis on nodes xi evaluated at points x: out[i*n + k] = phi_k(x_i).
void lagrange_eval(const std::vector<double>& xi, const std::vector<double>& x,
                   std::vector<double>& out);
// 1D element mass (GLL diagonal, p+1) and stiffness ((p+1)^2) of width h:
// M = (h/2) w and L = (2/h) Lhat, Lhat_ij = sum_q w_q D_qi D_qj correctly
// rounded, each scaled with one double multiplication.
void element_matrices(int p, double h, std::vector<double>& M, std::vector<double>& L);
// Symmetric-definite eigenproblem A s = lambda diag(b) s by cyclic Jacobi on
// diag(b)^{-1/2} A diag(b)^{-1/2}.  S (n x n, row-major, columns = vectors with
// S^T diag(b) S = I), lam ascending.  Returns false if Jacobi did not converge.
bool gen_eig_diag(int n, const std::vector<double>& A, const std::vector<double>& b,
                  std::vector<double>& S, std::vector<double>& lam);

// Shape function phi_kappa of Eq. (shape function) for weight id kappa.
double shape_phi(int kappa, double x);
// Shape function of continuous degree kt in [1, 7]: the convex blend of the
// two neighbouring odd degrees of Table (weighting), sgn outside (-1, 1).
double shape_phi_blend(double kt, double x);

// Factors of the extended-element subdomains of one direction of one level,
// padded to the interior window size m = p + 1 + 2 n_o.  Window slot a holds
// element-local node k = a - n_o; slots outside the mesh (Dirichlet walls)
// have zero rows in S, zero weight, and their eigen-slots carry lam = 1.
struct SubTable {
  std::vector<double> S;    // m x m, S[a*m + b] = b-th eigenvector at slot a
  std::vector<double> lam;  // m
  std::vector<double> w;    // m, 1D weights (Eq. (weight function))
};

struct Dir1D {
  int n = 0, p = 0, n_o = 0, m = 0, N = 0;
  bool periodic = false;
  std::vector<double> Me;     // n x (p+1): element mass diagonals
  std::vector<double> Le;     // n x (p+1)^2: element stiffness
  std::vector<double> Mglob;  // N: assembled mass diagonal (walls included)
  std::vector<double> coords; // N
  std::vector<int> tab;       // n: subdomain table id per element
  std::vector<SubTable> tables;
};

// Build one direction of one level.  weight: sem_weight id.  learned (weight
// SEM_W_LEARNED): per interface i = 0..n (between elements i-1 and i) the
// pair (s, kt): transition half width scale and shape degree.  Returns "" or
// an error message.
std::string build_dir(const Mesh1D& mesh, int p, int n_o, int weight, Dir1D& out, const double* learned = nullptr);

// Coarse (p = 1) factors: generalised eigenpairs of the assembled 1D pair over
// the unknowns (Dirichlet: nodes 1..n-1; periodic: 0..n-1), and c = S^T 1.
struct Coarse1D {
  int nu = 0;                 // unknowns per direction
  int first = 0;              // global index of the first unknown
  std::vector<double> S, lam, c;
};
std::string build_coarse(const Mesh1D& mesh, Coarse1D& out);

// Variable diffusivity nu(x, y) (Sec. 4.3, Eq. (diffusion)); kind 1:
// 1 + (a-1)(1/2 + 1/2 sin(2 pi x) cos(2 pi y)) (contrast a); kind 2:
// 1 + a sin(2 pi (x - b)) sin(2 pi (y - b)) (amplitude a, shift b).
double nu_value(int kind, double a, double b, double x, double y);

// Element data of B(nu) at order p: G_x = w_j w_i J nu (2/h_x)^2 and
// G_y = w_j w_i J nu (2/h_y)^2 at the element's GLL nodes (row j = y, col i = x),
// and nu_bar, the GLL-quadrature mean of nu over the element (Sec. 4.3).
struct VarData {
  std::vector<double> Gx, Gy;  // (ny * nx) x (p+1)^2
  std::vector<double> nu_bar;  // ny * nx
  std::vector<double> D;       // (p+1)^2 differentiation matrix
};
void build_var(const Mesh1D& mx, const Mesh1D& my, int p, int kind, double a, double b, VarData& out);

// Dense inverse of B(nu) at p = 1 over the Dirichlet unknowns (row-major,
// (nx-1)(ny-1) squared), by a banded Cholesky factorisation; on a periodic
// mesh the dense pseudo-inverse over all nx ny coarse nodes (at most 1024).
std::string coarse_var_inverse(const Mesh1D& mx, const Mesh1D& my, int kind, double a, double b,
                               std::vector<double>& inv);

// Interpolation J[i*(pc+1) + k] = phi_k^{(pc)}(xi_i^{(pf)}).
void interp_matrix(int pf, int pc, std::vector<double>& J);

// Fixed-point even-odd tables of one direction for the integer evaluation of
// the FP64 operator (launch_apply_fx): per element e, L_int = L * 2^t[e] with
// |L_int| < 2^73 (exact unless an element's entries span more than 20 binary
// exponents; then rounded to nearest), E[a][k] = L_int[a][k] + L_int[a][p-k]
// (k < p/2), E[a][p/2] = 2 L_int[a][p/2], O[a][k] = L_int[a][k] -
// L_int[a][p-k], each stored as four ints (l0, l1, l2, 0) with value
// l2 2^50 + l1 2^25 + l0, l0 and l1 in [0, 2^25).  Elements whose tables
// and t are equal share one copy: tab holds k + 1 tables of ((p/2+1)^2 +
// (p/2)^2) entries, the last all zero (t = 0) for missing neighbours; t has
// k + 1 entries; slot (n + 1 entries) gives element e's table, slot[n] the
// zero table (a uniform mesh needs k = 1).  Returns false (tables unusable)
// when an element matrix is not centro-symmetric in these integers,
// L_int[p-a][p-k] == L_int[a][k], which the even-odd form needs.
bool fx_tables(const Dir1D& d, std::vector<int>& tab, std::vector<int>& t, std::vector<int>& slot);

}  // namespace sem
