// Host FP64 set-up (see setup.h).
#include "setup.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <tuple>

namespace sem {

namespace {

// Legendre P_p(x) and P_{p-1}(x) by the three-term recurrence.
void legendre(int p, double x, double& Pp, double& Pm1) {
  double a = 1.0, b = x;  // P_0, P_1
  if (p == 0) { Pp = 1.0; Pm1 = 0.0; return; }
  for (int k = 1; k < p; ++k) {
    double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
    a = b;
    b = c;
  }
  Pp = b;
  Pm1 = a;
}

}  // namespace

void gll(int p, std::vector<double>& xi, std::vector<double>& w) {
  xi.assign(p + 1, 0.0);
  w.assign(p + 1, 0.0);
  xi[0] = -1.0;
  xi[p] = 1.0;
  // interior nodes: roots of P_p'.  Newton on P_p' with P_p'' from the
  // Legendre equation (1-x^2) P'' = 2x P' - p(p+1) P, started at the
  // Chebyshev-Gauss-Lobatto points.
  for (int j = 1; j < p; ++j) {
    double x = -std::cos(M_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double P, Pm;
      legendre(p, x, P, Pm);
      double dP = p * (x * P - Pm) / (x * x - 1.0);
      double d2P = (2.0 * x * dP - p * (p + 1.0) * P) / (1.0 - x * x);
      double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    xi[j] = x;
  }
  for (int j = 0; j <= p / 2; ++j) {  // exact symmetry
    double s = 0.5 * (xi[p - j] - xi[j]);
    xi[j] = -s;
    xi[p - j] = s;
  }
  if (p % 2 == 0) xi[p / 2] = 0.0;
  for (int j = 0; j <= p; ++j) {
    double P, Pm;
    legendre(p, xi[j], P, Pm);
    w[j] = 2.0 / (p * (p + 1.0) * P * P);
  }
}

void deriv_matrix(const std::vector<double>& xi, std::vector<double>& D) {
  const int n = (int)xi.size();
  std::vector<double> c(n, 1.0);  // c_i = prod_{k != i} (xi_i - xi_k)
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k)
      if (k != i) c[i] *= xi[i] - xi[k];
  D.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[i * n + j] = c[i] / (c[j] * (xi[i] - xi[j]));
      diag += 1.0 / (xi[i] - xi[j]);
    }
    D[i * n + i] = diag;
  }
}

void lagrange_eval(const std::vector<double>& xi, const std::vector<double>& x,
                   std::vector<double>& out) {
  const int n = (int)xi.size(), m = (int)x.size();
  out.assign(m * n, 1.0);
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        if (j != k) out[i * n + k] *= (x[i] - xi[j]) / (xi[k] - xi[j]);
}

void element_matrices(int p, double h, std::vector<double>& M, std::vector<double>& L) {
  std::vector<double> xi, w, D;
  gll(p, xi, w);
  deriv_matrix(xi, D);
  const int n = p + 1;
  M.resize(n);
  L.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) M[i] = 0.5 * h * w[i];
  // L_ij = (2/h) sum_q w_q D_qi D_qj
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s += w[q] * D[q * n + i] * D[q * n + j];
      L[i * n + j] = (2.0 / h) * s;
    }
}

bool gen_eig_diag(int n, const std::vector<double>& A, const std::vector<double>& b,
                  std::vector<double>& S, std::vector<double>& lam) {
  // C = B^{-1/2} A B^{-1/2}
  std::vector<double> C(n * n), V(n * n, 0.0), r(n);
  for (int i = 0; i < n; ++i) r[i] = 1.0 / std::sqrt(b[i]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) C[i * n + j] = r[i] * A[i * n + j] * r[j];
  for (int i = 0; i < n; ++i) {
    V[i * n + i] = 1.0;
    for (int j = 0; j < i; ++j) C[i * n + j] = C[j * n + i] = 0.5 * (C[i * n + j] + C[j * n + i]);
  }
  double scale = 0.0;
  for (double v : C) scale = std::max(scale, std::fabs(v));
  bool converged = (n <= 1);
  for (int sweep = 0; sweep < 100 && !converged; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off = std::max(off, std::fabs(C[i * n + j]));
    if (off <= 1e-17 * scale) { converged = true; break; }
    for (int pidx = 0; pidx < n; ++pidx)
      for (int q = pidx + 1; q < n; ++q) {
        double apq = C[pidx * n + q];
        if (std::fabs(apq) <= 1e-300) continue;
        double app = C[pidx * n + pidx], aqq = C[q * n + q];
        // rotation angle that annihilates C[p][q] (classical Jacobi)
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double ckp = C[k * n + pidx], ckq = C[k * n + q];
          C[k * n + pidx] = c * ckp - s * ckq;
          C[k * n + q] = s * ckp + c * ckq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          double cpk = C[pidx * n + k], cqk = C[q * n + k];
          C[pidx * n + k] = c * cpk - s * cqk;
          C[q * n + k] = s * cpk + c * cqk;
        }
        C[pidx * n + q] = C[q * n + pidx] = 0.0;
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + pidx], vkq = V[k * n + q];
          V[k * n + pidx] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  if (!converged) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off = std::max(off, std::fabs(C[i * n + j]));
    converged = off <= 1e-14 * scale;
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int c) { return C[a * n + a] < C[c * n + c]; });
  S.assign(n * n, 0.0);
  lam.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    lam[j] = C[order[j] * n + order[j]];
    for (int i = 0; i < n; ++i) S[i * n + j] = r[i] * V[i * n + order[j]];
  }
  return converged;
}

double shape_phi(int kappa, double x) {
  if (!(std::fabs(x) < 1.0) || kappa == 100) return (x > 0) - (x < 0);
  const double x2 = x * x;
  switch (kappa) {
    case 1: return x;
    case 3: return x * (3.0 - x2) / 2.0;
    case 5: return x * (15.0 + x2 * (-10.0 + 3.0 * x2)) / 8.0;
    case 7: return x * (35.0 + x2 * (-35.0 + x2 * (21.0 - 5.0 * x2))) / 16.0;
    default: return 0.0;
  }
}

std::string build_dir(const Mesh1D& mesh, int p, int n_o, int weight, Dir1D& o) {
  const int n = mesh.n, N = mesh.nodes(p), np1 = p + 1, m = p + 1 + 2 * n_o;
  if (m > N) return "subdomain window larger than the periodic mesh";
  o.n = n; o.p = p; o.n_o = n_o; o.m = m; o.N = N; o.periodic = mesh.periodic;
  std::vector<double> xi, w;
  gll(p, xi, w);
  o.Me.assign(n * np1, 0.0);
  o.Le.assign(n * np1 * np1, 0.0);
  o.Mglob.assign(N, 0.0);
  o.coords.assign(N, 0.0);
  // global stiffness is needed only inside windows: keep a banded copy as a
  // map (i, j) -> value assembled from the element matrices
  std::vector<std::vector<std::pair<int, double>>> Lrow(N);
  auto addL = [&](int i, int j, double v) {
    for (auto& e : Lrow[i]) if (e.first == j) { e.second += v; return; }
    Lrow[i].push_back({j, v});
  };
  for (int e = n - 1; e >= 0; --e) {
    std::vector<double> Me, Le;
    element_matrices(p, mesh.h(e), Me, Le);
    for (int a = 0; a < np1; ++a) {
      o.Me[e * np1 + a] = Me[a];
      for (int b = 0; b < np1; ++b) o.Le[(e * np1 + a) * np1 + b] = Le[a * np1 + b];
    }
    for (int a = 0; a < np1; ++a) {
      int ga = (e * p + a) % (mesh.periodic ? N : N + 1);
      o.Mglob[ga] += Me[a];
      o.coords[ga] = mesh.edges[e] + 0.5 * (1.0 + xi[a]) * mesh.h(e);
      for (int b = 0; b < np1; ++b) {
        int gb = (e * p + b) % (mesh.periodic ? N : N + 1);
        addL(ga, gb, Le[a * np1 + b]);
      }
    }
  }
  if (!mesh.periodic) o.coords[N - 1] = mesh.edges[n];
  auto Lget = [&](int i, int j) {
    for (auto& e : Lrow[i]) if (e.first == j) return e.second;
    return 0.0;
  };
  // window of element e: slot a <-> local k = a - n_o <-> global e*p + k
  auto gidx = [&](int e, int a, bool& valid) {
    int g = e * p + a - n_o;
    if (mesh.periodic) { valid = true; return (g % N + N) % N; }
    valid = (g > 0 && g < n * p);
    return g;
  };
  // counting matrix for the arithmetic mean (Sec. 3.1): windows per node
  std::vector<int> cnt(N, 0);
  for (int e = 0; e < n; ++e)
    for (int a = 0; a < m; ++a) {
      bool v;
      int g = gidx(e, a, v);
      if (v) cnt[g]++;
    }
  const double dO = xi[n_o + 1] + 1.0;  // Eq. (overlap width)
  std::map<std::tuple<int, int, double, double, double>, int> seen;
  o.tab.assign(n, 0);
  o.tables.clear();
  for (int e = 0; e < n; ++e) {
    int L = mesh.neighbour(e, -1), R = mesh.neighbour(e, +1);
    double hl = L >= 0 ? mesh.h(L) : 0.0, hr = R >= 0 ? mesh.h(R) : 0.0, he = mesh.h(e);
    // elements with identical geometry share tables (arith weights depend on
    // counts, which are equal for equal geometry and wall status)
    auto key = std::make_tuple(L >= 0 ? 1 : 0, R >= 0 ? 1 : 0, hl, he, hr);
    if (weight != 101) {
      auto it = seen.find(key);
      if (it != seen.end()) { o.tab[e] = it->second; continue; }
    }
    SubTable t;
    t.S.assign(m * m, 0.0);
    t.lam.assign(m, 1.0);
    t.w.assign(m, 0.0);
    std::vector<int> slots, gl;
    for (int a = 0; a < m; ++a) {
      bool v;
      int g = gidx(e, a, v);
      if (v) { slots.push_back(a); gl.push_back(g); }
    }
    const int mv = (int)slots.size();
    std::vector<double> At(mv * mv), bt(mv), St, lt;
    for (int i = 0; i < mv; ++i) {
      bt[i] = o.Mglob[gl[i]];
      for (int j = 0; j < mv; ++j) At[i * mv + j] = Lget(gl[i], gl[j]);
    }
    if (!gen_eig_diag(mv, At, bt, St, lt)) return "Jacobi eigensolver did not converge";
    for (int i = 0; i < mv; ++i)
      for (int j = 0; j < mv; ++j) t.S[slots[i] * m + j] = St[i * mv + j];
    for (int j = 0; j < mv; ++j) t.lam[j] = lt[j];
    // weights, Eq. (weight function) in the interface form: position s of
    // each slot relative to the left interface of element e
    for (int i = 0; i < mv; ++i) {
      const int a = slots[i], k = a - n_o;
      double s;
      if (k < 0) s = -(1.0 - xi[p + k]) * hl / 2.0;
      else if (k <= p) s = (1.0 + xi[k]) * he / 2.0;
      else s = he + (1.0 + xi[k - p]) * hr / 2.0;
      double wv;
      if (weight == 102) {
        wv = 1.0;
      } else if (weight == 101) {
        wv = 1.0 / cnt[gl[i]];
      } else {
        double tl = 1.0, tr = -1.0;
        if (L >= 0) tl = shape_phi(weight, s / (dO * std::min(hl, he) / 2.0));
        if (R >= 0) tr = shape_phi(weight, (s - he) / (dO * std::min(he, hr) / 2.0));
        // a node exactly on the interface has s == 0 (or s == he) exactly
        if (k == 0 && L >= 0) tl = 0.0;
        if (k == p && R >= 0) tr = 0.0;
        wv = 0.5 * (tl - tr);
      }
      t.w[a] = wv;
    }
    o.tab[e] = (int)o.tables.size();
    seen[key] = o.tab[e];
    o.tables.push_back(std::move(t));
  }
  return "";
}

std::string build_coarse(const Mesh1D& mesh, Coarse1D& o) {
  const int n = mesh.n, N = mesh.nodes(1);
  std::vector<double> Mg(N, 0.0), Lg(N * N, 0.0);
  for (int e = 0; e < n; ++e) {
    std::vector<double> Me, Le;
    element_matrices(1, mesh.h(e), Me, Le);
    for (int a = 0; a < 2; ++a) {
      int ga = (e + a) % (mesh.periodic ? N : N + 1);
      Mg[ga] += Me[a];
      for (int b = 0; b < 2; ++b) {
        int gb = (e + b) % (mesh.periodic ? N : N + 1);
        Lg[ga * N + gb] += Le[a * 2 + b];
      }
    }
  }
  o.first = mesh.periodic ? 0 : 1;
  o.nu = mesh.periodic ? N : N - 2;
  const int nu = o.nu, f = o.first;
  std::vector<double> A(nu * nu), b(nu);
  for (int i = 0; i < nu; ++i) {
    b[i] = Mg[f + i];
    for (int j = 0; j < nu; ++j) A[i * nu + j] = Lg[(f + i) * N + (f + j)];
  }
  if (!gen_eig_diag(nu, A, b, o.S, o.lam)) return "coarse eigensolver did not converge";
  o.c.assign(nu, 0.0);
  for (int j = 0; j < nu; ++j)
    for (int i = 0; i < nu; ++i) o.c[j] += o.S[i * nu + j];
  return "";
}

void interp_matrix(int pf, int pc, std::vector<double>& J) {
  std::vector<double> xf, wf, xc, wc;
  gll(pf, xf, wf);
  gll(pc, xc, wc);
  lagrange_eval(xc, xf, J);
}

}  // namespace sem
