// Host FP64 set-up (see setup.h).
#include "setup.h"

#include <algorithm>
#include <cstdint>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>

namespace sem {

namespace {

// ---- double-double arithmetic ------------------------------------------------
// A value is the unevaluated sum hi + lo with |lo| <= ulp(hi) / 2 (about 106
// significant bits).  Built from the error-free transformations of Knuth
// (two-sum) and Dekker (two-product, here with one fused multiply-add); the
// 1D matrices below are computed in it and rounded once to double, so that
// they are the correctly rounded values of their exact definitions.
struct DD {
  double hi = 0.0, lo = 0.0;
  DD() = default;
  DD(double h) : hi(h) {}  // NOLINT: implicit from double on purpose
  DD(double h, double l) : hi(h), lo(l) {}
};

DD two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return DD(s, (a - (s - bb)) + (b - bb));
}
DD fast_two_sum(double a, double b) {  // |a| >= |b|
  const double s = a + b;
  return DD(s, b - (s - a));
}
DD operator+(const DD& a, const DD& b) {
  DD s = two_sum(a.hi, b.hi);
  const DD t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(s.hi, s.lo + t.lo);
}
DD operator-(const DD& a) { return DD(-a.hi, -a.lo); }
DD operator-(const DD& a, const DD& b) { return a + (-b); }
DD operator*(const DD& a, const DD& b) {
  const double p = a.hi * b.hi;
  const double e = std::fma(a.hi, b.hi, -p);
  const double c = a.hi * b.lo;
  const double d = a.lo * b.hi;
  return fast_two_sum(p, e + (c + d));
}
DD operator/(const DD& a, const DD& b) {  // long division, three partial quotients
  const double q1 = a.hi / b.hi;
  DD r = a - b * DD(q1);
  const double q2 = r.hi / b.hi;
  r = r - b * DD(q2);
  const double q3 = r.hi / b.hi;
  return fast_two_sum(q1, q2) + DD(q3);
}
double fabs_dd(const DD& a) { return std::fabs(a.hi); }

// P_p(x) and P_{p-1}(x) by the three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}.
void legendre_dd(int p, const DD& x, DD& Pp, DD& Pm1) {
  DD a(1.0), b = x;
  if (p == 0) { Pp = DD(1.0); Pm1 = DD(0.0); return; }
  for (int k = 1; k < p; ++k) {
    const DD c = (DD(2.0 * k + 1.0) * x * b - DD((double)k) * a) / DD(k + 1.0);
    a = b;
    b = c;
  }
  Pp = b;
  Pm1 = a;
}

// GLL nodes and weights in double-double: interior nodes are the roots of
// P_p'; Newton on P_p' with P_p' = p (x P_p - P_{p-1}) / (x^2 - 1) and P_p''
// from the Legendre equation (1 - x^2) P'' = 2x P' - p(p+1) P, started at the
// Chebyshev-Gauss-Lobatto points (quadratic convergence; the loop stops once
// a step is below 1e-30).  Weights w_j = 2 / (p (p+1) P_p(xi_j)^2).
void gll_dd(int p, std::vector<DD>& xi, std::vector<DD>& w) {
  xi.assign(p + 1, DD(0.0));
  w.assign(p + 1, DD(0.0));
  xi[0] = DD(-1.0);
  xi[p] = DD(1.0);
  const DD pp1(p * (p + 1.0));
  for (int j = 1; j < p; ++j) {
    DD x(-std::cos(M_PI * j / p));
    for (int it = 0; it < 200; ++it) {
      DD P, Pm;
      legendre_dd(p, x, P, Pm);
      const DD x2m1 = x * x - DD(1.0);
      const DD dP = DD((double)p) * (x * P - Pm) / x2m1;
      const DD d2P = (DD(2.0) * x * dP - pp1 * P) / (-x2m1);
      const DD dx = dP / d2P;
      x = x - dx;
      if (fabs_dd(dx) < 1e-30) break;
    }
    xi[j] = x;
  }
  for (int j = 0; j <= p / 2; ++j) {  // exact symmetry xi_{p-j} = -xi_j
    const DD s = (xi[p - j] - xi[j]) * DD(0.5);
    xi[j] = -s;
    xi[p - j] = s;
  }
  if (p % 2 == 0) xi[p / 2] = DD(0.0);
  for (int j = 0; j <= p; ++j) {
    DD P, Pm;
    legendre_dd(p, xi[j], P, Pm);
    w[j] = DD(2.0) / (pp1 * P * P);
  }
}

// D_ij = phi_j'(xi_i) on the GLL nodes in double-double: off the diagonal the
// barycentric form c_i / (c_j (xi_i - xi_j)), c_i = prod_{k != i} (xi_i - xi_k);
// on it the GLL values -p(p+1)/4, p(p+1)/4 at the end points and 0 inside.
void gll_deriv_dd(int p, const std::vector<DD>& xi, std::vector<DD>& D) {
  const int n = p + 1;
  std::vector<DD> c(n, DD(1.0));
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k)
      if (k != i) c[i] = c[i] * (xi[i] - xi[k]);
  D.assign(n * n, DD(0.0));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (j != i) D[i * n + j] = c[i] / (c[j] * (xi[i] - xi[j]));
  D[0] = DD(-0.25 * p * (p + 1.0));
  D[n * n - 1] = DD(0.25 * p * (p + 1.0));
}

// The correctly rounded 1D set of order p (computed once per order).
struct GllSet {
  std::vector<double> xi, w, D, Lhat;
};

const GllSet& gll_set(int p) {
  static std::map<int, GllSet> cache;  // entries are never erased: references stay valid
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(p);
  if (it != cache.end()) return it->second;
  std::vector<DD> x, w, D;
  gll_dd(p, x, w);
  gll_deriv_dd(p, x, D);
  const int n = p + 1;
  GllSet g;
  g.xi.resize(n);
  g.w.resize(n);
  g.D.resize(n * n);
  g.Lhat.resize(n * n);
  for (int i = 0; i < n; ++i) {
    g.xi[i] = x[i].hi;
    g.w[i] = w[i].hi;
  }
  for (int i = 0; i < n * n; ++i) g.D[i] = D[i].hi;
  // reference stiffness Lhat_ij = sum_q w_q D_qi D_qj (Sec. 2, GLL quadrature)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      DD s(0.0);
      for (int q = 0; q < n; ++q) s = s + w[q] * D[q * n + i] * D[q * n + j];
      g.Lhat[i * n + j] = s.hi;
    }
  return cache.emplace(p, std::move(g)).first->second;
}

}  // namespace

void gll(int p, std::vector<double>& xi, std::vector<double>& w) {
  const GllSet& g = gll_set(p);
  xi = g.xi;
  w = g.w;
}

void gll_deriv(int p, std::vector<double>& D) { D = gll_set(p).D; }

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
  const GllSet& g = gll_set(p);
  const int n = p + 1;
  M.resize(n);
  L.resize(n * n);
  for (int i = 0; i < n; ++i) M[i] = 0.5 * h * g.w[i];
  // L = (2/h) Lhat, Lhat correctly rounded: one rounding of the scaled value
  const double s = 2.0 / h;
  for (int i = 0; i < n * n; ++i) L[i] = s * g.Lhat[i];
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

double shape_phi_blend(double kt, double x) {
  if (!(std::fabs(x) < 1.0)) return (x > 0) - (x < 0);
  const double t = std::min(3.0, std::max(0.0, 0.5 * (kt - 1.0)));
  const int k0 = std::min(2, (int)t);
  const double fr = t - k0;
  return (1.0 - fr) * shape_phi(2 * k0 + 1, x) + fr * shape_phi(2 * k0 + 3, x);
}

std::string build_dir(const Mesh1D& mesh, int p, int n_o, int weight, Dir1D& o, const double* learned) {
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
    valid = !mesh.wall(g, p);
    // a window never reaches across a wall into another stacked problem
    if (valid && mesh.seg > 0 && (g < (e / mesh.seg) * mesh.seg * p || g > (e / mesh.seg + 1) * mesh.seg * p))
      valid = false;
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
  std::map<std::tuple<int, int, double, double, double, double, double, double, double>, int> seen;
  o.tab.assign(n, 0);
  o.tables.clear();
  // widths equal up to rounding (edges e * l / n) count as equal geometry
  std::vector<double> widths;
  auto canon = [&widths](double h) {
    for (double c : widths)
      if (std::fabs(h - c) <= 1e-12 * c) return c;
    widths.push_back(h);
    return h;
  };
  for (int e = 0; e < n; ++e) {
    int L = mesh.neighbour(e, -1), R = mesh.neighbour(e, +1);
    double hl = L >= 0 ? mesh.h(L) : 0.0, hr = R >= 0 ? mesh.h(R) : 0.0, he = mesh.h(e);
    // elements with identical geometry share tables (arith weights depend on
    // counts, which are equal for equal geometry and wall status)
    // learned parameters of the element's left (interface e) and right
    // (interface e + 1) transitions
    double sl = 1.0, kl = 5.0, sr = 1.0, kr = 5.0;
    if (weight == 103 && learned) {
      const int il = e, ir = mesh.periodic ? (e + 1) % n : e + 1;
      sl = learned[2 * il];
      kl = learned[2 * il + 1];
      sr = learned[2 * ir];
      kr = learned[2 * ir + 1];
    }
    auto key = std::make_tuple(L >= 0 ? 1 : 0, R >= 0 ? 1 : 0, L >= 0 ? canon(hl) : 0.0, canon(he),
                               R >= 0 ? canon(hr) : 0.0, sl, kl, sr, kr);
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
      } else if (weight == 103) {
        double tl = 1.0, tr = -1.0;
        if (L >= 0) tl = shape_phi_blend(kl, s / (sl * dO * std::min(hl, he) / 2.0));
        if (R >= 0) tr = shape_phi_blend(kr, (s - he) / (sr * dO * std::min(he, hr) / 2.0));
        if (k == 0 && L >= 0) tl = 0.0;
        if (k == p && R >= 0) tr = 0.0;
        wv = 0.5 * (tl - tr);
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

double nu_value(int kind, double a, double b, double x, double y) {
  if (kind == 1) return 1.0 + (a - 1.0) * (0.5 + 0.5 * std::sin(2.0 * M_PI * x) * std::cos(2.0 * M_PI * y));
  if (kind == 2) return 1.0 + a * std::sin(2.0 * M_PI * (x - b)) * std::sin(2.0 * M_PI * (y - b));
  return 1.0;
}

void build_var(const Mesh1D& mx, const Mesh1D& my, int p, int kind, double a, double b, VarData& o) {
  std::vector<double> xi, w;
  gll(p, xi, w);
  gll_deriv(p, o.D);
  const int np1 = p + 1, nn = np1 * np1;
  o.Gx.assign((size_t)mx.n * my.n * nn, 0.0);
  o.Gy.assign((size_t)mx.n * my.n * nn, 0.0);
  o.nu_bar.assign((size_t)mx.n * my.n, 0.0);
  double wsum = 0.0;
  for (int j = 0; j < np1; ++j)
    for (int i = 0; i < np1; ++i) wsum += w[j] * w[i];
  for (int ey = 0; ey < my.n; ++ey)
    for (int ex = 0; ex < mx.n; ++ex) {
      const double hx = mx.h(ex), hy = my.h(ey), jac = 0.25 * hx * hy;
      const size_t e = (size_t)ey * mx.n + ex;
      double acc = 0.0;
      for (int j = 0; j < np1; ++j)
        for (int i = 0; i < np1; ++i) {
          const double x = mx.edges[ex] + 0.5 * (1.0 + xi[i]) * hx;
          const double y = my.edges[ey] + 0.5 * (1.0 + xi[j]) * hy;
          const double nu = nu_value(kind, a, b, x, y);
          const double q = w[j] * w[i] * jac * nu;
          o.Gx[e * nn + j * np1 + i] = q * (2.0 / hx) * (2.0 / hx);
          o.Gy[e * nn + j * np1 + i] = q * (2.0 / hy) * (2.0 / hy);
          acc += w[j] * w[i] * nu;
        }
      o.nu_bar[e] = acc / wsum;
    }
}

// Periodic mesh: B_0 is singular with the constants as null space, and the
// coarse solution of Alg. 3 is the pseudo-inverse B_0^+ f_0.  Dense: with
// M = B_0 + c 1 1^T (c = trace(B_0) / n^2, symmetric positive definite) and
// the projector P = I - 1 1^T / n onto the range, B_0^+ = P M^{-1} P (for f in
// the range, x = M^{-1} f solves B_0 x = f and is orthogonal to 1).
static std::string coarse_var_pinv_periodic(const Mesh1D& mx, const Mesh1D& my, int kind, double a, double b,
                                            std::vector<double>& inv) {
  const int nx = mx.n, ny = my.n, n = nx * ny;
  VarData v;
  build_var(mx, my, 1, kind, a, b, v);
  std::vector<double> M((size_t)n * n, 0.0);
  const double* D = v.D.data();
  for (int ey = 0; ey < ny; ++ey)
    for (int ex = 0; ex < nx; ++ex) {
      const size_t e = (size_t)ey * nx + ex;
      for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i)
          for (int l = 0; l < 2; ++l)
            for (int k = 0; k < 2; ++k) {
              double kv = 0.0;
              if (j == l)
                for (int q = 0; q < 2; ++q) kv += v.Gx[e * 4 + j * 2 + q] * D[q * 2 + i] * D[q * 2 + k];
              if (i == k)
                for (int q = 0; q < 2; ++q) kv += v.Gy[e * 4 + q * 2 + i] * D[q * 2 + j] * D[q * 2 + l];
              const int r = ((ey + j) % ny) * nx + (ex + i) % nx, c = ((ey + l) % ny) * nx + (ex + k) % nx;
              M[(size_t)r * n + c] += kv;
            }
    }
  double tr = 0.0;
  for (int i = 0; i < n; ++i) tr += M[(size_t)i * n + i];
  const double cst = tr / n / n;
  for (auto& x : M) x += cst;
  // dense Cholesky M = L L^T (lower triangle in place)
  for (int j = 0; j < n; ++j) {
    double d = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= M[(size_t)j * n + k] * M[(size_t)j * n + k];
    if (!(d > 0.0)) return "coarse variable-diffusivity matrix is not positive definite on the range";
    const double ljj = std::sqrt(d);
    M[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double sum = M[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) sum -= M[(size_t)i * n + k] * M[(size_t)j * n + k];
      M[(size_t)i * n + j] = sum / ljj;
    }
  }
  // columns of M^{-1} P: solve M x = e_c - 1/n
  std::vector<double> X((size_t)n * n), y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) y[i] = (i == c ? 1.0 : 0.0) - 1.0 / n;
    for (int i = 0; i < n; ++i) {
      double sum = y[i];
      for (int k = 0; k < i; ++k) sum -= M[(size_t)i * n + k] * y[k];
      y[i] = sum / M[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double sum = y[i];
      for (int k = i + 1; k < n; ++k) sum -= M[(size_t)k * n + i] * y[k];
      y[i] = sum / M[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) X[(size_t)i * n + c] = y[i];
  }
  // P (M^{-1} P): subtract the column means
  inv.assign((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    double mean = 0.0;
    for (int i = 0; i < n; ++i) mean += X[(size_t)i * n + c];
    mean /= n;
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = X[(size_t)i * n + c] - mean;
  }
  return "";
}

std::string coarse_var_inverse(const Mesh1D& mx, const Mesh1D& my, int kind, double a, double b,
                               std::vector<double>& inv) {
  if (mx.periodic != my.periodic) return "mixed periodic and Dirichlet directions are not supported";
  if (mx.periodic) {
    if ((long)mx.n * my.n > 1024) return "periodic variable diffusivity: at most 1024 coarse unknowns (32 x 32 elements)";
    return coarse_var_pinv_periodic(mx, my, kind, a, b, inv);
  }
  const int nux = mx.n - 1, nuy = my.n - 1, n = nux * nuy, bw = nux + 1;  // half bandwidth
  VarData v;
  build_var(mx, my, 1, kind, a, b, v);
  // band storage: Bb[i][d] = B[i][i - d], d = 0..bw (lower band)
  std::vector<double> Bb((size_t)n * (bw + 1), 0.0);
  const double* D = v.D.data();  // 2 x 2
  for (int ey = 0; ey < my.n; ++ey)
    for (int ex = 0; ex < mx.n; ++ex) {
      const size_t e = (size_t)ey * mx.n + ex;
      // element matrix K[(j,i),(l,k)] = sum_q Gx[j][q] D[q][i] D[q][k] d_jl + sum_q Gy[q][i] D[q][j] D[q][l] d_ik
      for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i)
          for (int l = 0; l < 2; ++l)
            for (int k = 0; k < 2; ++k) {
              double kv = 0.0;
              if (j == l)
                for (int q = 0; q < 2; ++q) kv += v.Gx[e * 4 + j * 2 + q] * D[q * 2 + i] * D[q * 2 + k];
              if (i == k)
                for (int q = 0; q < 2; ++q) kv += v.Gy[e * 4 + q * 2 + i] * D[q * 2 + j] * D[q * 2 + l];
              const int gr_y = ey + j, gr_x = ex + i, gc_y = ey + l, gc_x = ex + k;
              if (gr_y < 1 || gr_y > nuy || gr_x < 1 || gr_x > nux) continue;
              if (gc_y < 1 || gc_y > nuy || gc_x < 1 || gc_x > nux) continue;
              const int r = (gr_y - 1) * nux + gr_x - 1, c = (gc_y - 1) * nux + gc_x - 1;
              if (c <= r) Bb[(size_t)r * (bw + 1) + (r - c)] += kv;
            }
    }
  // banded Cholesky B = L L^T, L stored in the same band layout
  for (int i = 0; i < n; ++i) {
    for (int d = std::min(i, bw); d >= 0; --d) {
      const int j = i - d;
      double sum = Bb[(size_t)i * (bw + 1) + d];
      const int k0 = std::max(0, i - bw);
      for (int k = std::max(k0, j - bw); k < j; ++k)
        sum -= Bb[(size_t)i * (bw + 1) + (i - k)] * Bb[(size_t)j * (bw + 1) + (j - k)];
      if (d == 0) {
        if (!(sum > 0.0)) return "coarse variable-diffusivity matrix is not positive definite";
        Bb[(size_t)i * (bw + 1)] = std::sqrt(sum);
      } else {
        Bb[(size_t)i * (bw + 1) + d] = sum / Bb[(size_t)j * (bw + 1)];
      }
    }
  }
  // inverse column by column: L y = e_c, L^T x = y
  inv.assign((size_t)n * n, 0.0);
  std::vector<double> y(n);
  for (int c = 0; c < n; ++c) {
    std::fill(y.begin(), y.end(), 0.0);
    y[c] = 1.0;
    for (int i = c; i < n; ++i) {
      double sum = y[i];
      for (int k = std::max(c, i - bw); k < i; ++k) sum -= Bb[(size_t)i * (bw + 1) + (i - k)] * y[k];
      y[i] = sum / Bb[(size_t)i * (bw + 1)];
    }
    for (int i = n - 1; i >= 0; --i) {
      double sum = y[i];
      for (int k = i + 1; k <= std::min(n - 1, i + bw); ++k) sum -= Bb[(size_t)k * (bw + 1) + (k - i)] * y[k];
      y[i] = sum / Bb[(size_t)i * (bw + 1)];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = y[i];
  }
  return "";
}

bool fx_tables(const Dir1D& d, std::vector<int>& tab, std::vector<int>& t, std::vector<int>& slot) {
  const int p = d.p, np1 = p + 1, H = p / 2;
  const int NE = (H + 1) * (H + 1), NO = H * H;
  const size_t B = (size_t)(NE + NO) * 4;  // ints per table
  std::vector<int> all((size_t)d.n * B, 0), te_of(d.n, 0);
  std::vector<__int128> li(np1 * np1);
  for (int e = 0; e < d.n; ++e) {
    const double* L = d.Le.data() + (size_t)e * np1 * np1;
    double amax = 0.0;
    for (int i = 0; i < np1 * np1; ++i) amax = std::max(amax, std::fabs(L[i]));
    if (!(amax > 0.0) || !std::isfinite(amax)) return false;
    int ex_max = 0;
    std::frexp(amax, &ex_max);  // amax in [2^(ex_max-1), 2^ex_max)
    const int te = 73 - ex_max;  // |L| 2^te < 2^73
    te_of[e] = te;
    for (int i = 0; i < np1 * np1; ++i) {
      int ex = 0;
      const double fr = std::frexp(L[i], &ex);        // L = fr 2^ex, |fr| in [0.5, 1)
      const int64_t m = (int64_t)std::ldexp(fr, 53);  // exact: |m| < 2^53
      const int sh = ex - 53 + te;                    // L 2^te = m 2^sh, sh <= 20
      const __int128 am = m < 0 ? -(__int128)m : (__int128)m;
      __int128 v;
      if (L[i] == 0.0) v = 0;
      else if (sh >= 0) v = am << sh;  // exact
      else if (sh >= -100) v = (am + ((__int128)1 << (-sh - 1))) >> (-sh);  // nearest, ties away from zero
      else v = 0;
      li[i] = m < 0 ? -v : v;
    }
    for (int a = 0; a <= p; ++a)
      for (int k = 0; k <= p; ++k)
        if (li[(p - a) * np1 + (p - k)] != li[a * np1 + k]) return false;
    int* out = all.data() + (size_t)e * B;
    auto put = [&](int idx, __int128 v) {  // v = l2 2^50 + l1 2^25 + l0, l0, l1 in [0, 2^25)
      const __int128 q1 = v >> 25, q2 = v >> 50;  // arithmetic shifts (floor)
      out[4 * idx] = (int)(v - (q1 << 25));
      out[4 * idx + 1] = (int)(q1 - (q2 << 25));
      out[4 * idx + 2] = (int)q2;
    };
    for (int a = 0; a <= H; ++a)
      for (int k = 0; k <= H; ++k)
        put(a * (H + 1) + k, k == H ? 2 * li[a * np1 + H] : li[a * np1 + k] + li[a * np1 + p - k]);
    for (int a = 0; a < H; ++a)
      for (int k = 0; k < H; ++k) put(NE + a * H + k, li[a * np1 + k] - li[a * np1 + p - k]);
  }
  // one copy per distinct (table, t), in order of first use; then the zero table
  tab.clear();
  t.clear();
  slot.assign(d.n + 1, 0);
  std::map<std::pair<int, std::vector<int>>, int> seen;
  for (int e = 0; e < d.n; ++e) {
    auto key = std::make_pair(te_of[e], std::vector<int>(all.begin() + (size_t)e * B, all.begin() + (size_t)(e + 1) * B));
    auto it = seen.find(key);
    if (it == seen.end()) {
      const int k = (int)t.size();
      tab.insert(tab.end(), key.second.begin(), key.second.end());
      t.push_back(te_of[e]);
      it = seen.emplace(std::move(key), k).first;
    }
    slot[e] = it->second;
  }
  slot[d.n] = (int)t.size();
  tab.insert(tab.end(), B, 0);
  t.push_back(0);
  return true;
}

void interp_matrix(int pf, int pc, std::vector<double>& J) {
  std::vector<double> xf, wf, xc, wc;
  gll(pf, xf, wf);
  gll(pc, xc, wc);
  lagrange_eval(xc, xf, J);
}

}  // namespace sem
