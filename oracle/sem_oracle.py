"""Plain FP64 CPU oracle of the hybrid Schwarz/multigrid spectral-element solver
(J. Stiller, "Nonuniformly weighted Schwarz smoothers for spectral element
multigrid", J. Sci. Comput.).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct
restatement of the method that the CUDA library is checked against.  Only the
test-suite, the smoke check of ``__graft_entry__`` and the CPU-baseline legs of
``bench.py`` may import it; the product library never does, and this module
imports nothing from the product package.  Everything is float64 numpy/scipy,
element by element, in the paper's order and notation.

What it follows (paper sections / equations / algorithms):
  * Sec. 2, Eqs. (ansatz), (discrete), (system matrix): GLL Lagrange basis,
    diagonal GLL mass and stiffness per element, assembly with periodic or
    Dirichlet connectivity, A = M_y (x) L_x + L_y (x) M_x applied element by
    element with explicit gather and scatter-add.
  * Sec. 3.1: extended-element subdomains (n_o node layers adopted from each
    neighbour, outer layer excluded), Eq. (overlap width) delta_O = xi_{n_o+1}+1,
    Eq. (subproblem) A_ss = R_s A R_s^T, the fast-diagonalisation inverse of
    Eq. (FDM), Eq. (weight function) and Eq. (shape function) with the shape
    functions of Table (weighting), Alg. 2 (weighted additive Schwarz).
  * Sec. 3.2, Alg. 3: p-multigrid V-cycle, p_l = 2^l, embedded interpolation
    and its transpose, coarse solution by the pseudo-inverse A_0^+.
  * Sec. 3.3, Alg. 4: inexact (flexible) MG-preconditioned CG.
  * Sec. 4: logarithmic convergence rate r_bar and n_10.
  * Sec. 4.3, Eqs. (diffusion), (subproblem:solution): variable diffusivity
    operator B(nu) and the local solve (1/nu_bar_s) A_ss^{-1} r_s.

Readings where the paper is silent or ambiguous (each also listed in the
design notes of the repository):
  R1 mass matrix: GLL-quadrature diagonal (Sec. 4 counts W_op = 2 n_p^3 n_e,
     which is the cost with a diagonal mass).
  R2 w_a is defined by its Sec. 3.1 definition W = R_s C^+ R_s^T, not by the
     shape-function formula with phi_hat = 0.
  R3 phi_kappa is phi_hat on the open interval (-1, 1) and sgn outside it;
     sgn(0) = 0.
  R4 Dirichlet walls: a subdomain side without a neighbour uses the saturated
     value of that side's phi term (+1 left, -1 right).
  R5 stretched meshes: the transition of Eq. (weight function) sits on each
     interface with half width d_I = delta_O * min(h_left, h_right) / 2; this
     equals Eq. (weight function) on uniform meshes.
  R6 Alg. 4 beta line: read as z^T (r - r_old) / delta (Polak-Ribiere, Sec. 3.3
     text); r_old starts at 0 as printed.
  R7 the coarse solution is the pseudo-inverse itself (dense Cholesky of the
     assembled A_0, with the right side projected to zero mean and the
     solution taken orthogonal to the constants when A_0 is singular).
  R8 lower-level corrections u_l (l < L) start from zero in every cycle.
  R9 n_{o,l} = min(rule(p_l), p_l - 1); level 0 is never smoothed.
  R10 nu_bar_s is the GLL-quadrature mean of nu over the embedded element.
  R15 Alg. 1 (multiplicative Schwarz): each local problem is solved on the
     whole extended subdomain, and the update adds the solution on the
     element's own closed node set only (no weights).  Adding it on the whole
     window converges faster than the paper's "mult" columns (r_bar 1.44 /
     1.90 / 1.49 against the printed 1.01 / 1.29 / 1.26 of Table 1);
     this reading reproduces Tables 1 and 3.
  R16 learned weights (not in the paper): per interface line a transition
     half-width scale s in (0, 1] and a shape degree kt in [1, 7], phi the
     convex blend of the two neighbouring odd-degree shape functions.
  R18 variable diffusivity: B(nu) is the weak form with nu sampled at the GLL
     nodes inside the GLL quadrature of each element.
  R19 the 1D GLL set (nodes, weights, D and the reference stiffness
     Lhat = D^T W D of Sec. 2) is taken as the correctly rounded doubles of
     the exact values: computed in 50-digit decimal arithmetic and rounded
     once.  The assembled operator is ill-conditioned enough that the
     discrete solution at 64 x 64 elements, p = 16, moves by ~1e-11 between
     two double-precision evaluations of Lhat in different summation orders;
     the exact values are the one reading two independent FP64 codes can
     share.
"""
from __future__ import annotations

import functools
import math
from decimal import Decimal, localcontext
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
from numpy.polynomial import legendre as npleg

# ---------------------------------------------------------------------------
# 1D spectral basics (Sec. 2)
# ---------------------------------------------------------------------------


_DIGITS = 50  # decimal working precision of the 1D set-up


def _legendre_decimal(p: int, x: Decimal):
    """P_p(x), P_p'(x), P_p''(x) in decimal arithmetic.

    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};  differentiating the identity
    (2k+1) P_k = P'_{k+1} - P'_{k-1} once more gives the derivative recurrences
    P'_{k+1} = P'_{k-1} + (2k+1) P_k and P''_{k+1} = P''_{k-1} + (2k+1) P'_k.
    """
    P0, P1 = Decimal(1), x
    d0, d1 = Decimal(0), Decimal(1)
    s0, s1 = Decimal(0), Decimal(0)
    for k in range(1, p):
        P0, P1 = P1, ((2 * k + 1) * x * P1 - k * P0) / (k + 1)
        d0, d1 = d1, d0 + (2 * k + 1) * P0
        s0, s1 = s1, s0 + (2 * k + 1) * d0
    return P1, d1, s1


@functools.lru_cache(maxsize=None)
def _gll_exact(p: int):
    """GLL nodes, weights and differentiation matrix of order p to 50 digits (Sec. 2).

    Nodes: -1, +1 and the roots of P_p', from numpy's Legendre root finder
    refined by Newton steps on P_p' in decimal arithmetic until a step falls
    below 1e-45.  Weights: w_j = 2 / (p (p+1) P_p(xi_j)^2).  Differentiation
    matrix D_ij = phi_j'(xi_i), in the closed form for GLL nodes:
    P_p(xi_i) / (P_p(xi_j) (xi_i - xi_j)) off the diagonal, -p(p+1)/4 and
    p(p+1)/4 at the two end points, 0 at the interior diagonal entries.
    """
    if p < 1:
        raise ValueError("p >= 1 required")
    with localcontext() as ctx:
        ctx.prec = _DIGITS
        x = [Decimal(-1)]
        if p >= 2:
            c = np.zeros(p + 1)
            c[p] = 1.0
            for x0 in np.sort(np.real(npleg.legroots(npleg.legder(c)))):
                t = Decimal(float(x0))
                for _ in range(100):
                    _, d, s2 = _legendre_decimal(p, t)
                    step = d / s2
                    t -= step
                    if abs(step) < Decimal("1e-45"):
                        break
                x.append(t)
        x.append(Decimal(1))
        for j in range(p // 2 + 1):  # exact symmetry xi_{p-j} = -xi_j
            h = (x[p - j] - x[j]) / 2
            x[j], x[p - j] = -h, h
        if p % 2 == 0:
            x[p // 2] = Decimal(0)
        P = [_legendre_decimal(p, t)[0] for t in x]
        w = [Decimal(2) / (p * (p + 1) * Pj * Pj) for Pj in P]
        n = p + 1
        D = [[Decimal(0)] * n for _ in range(n)]
        for i in range(n):
            for j in range(n):
                if i != j:
                    D[i][j] = P[i] / (P[j] * (x[i] - x[j]))
        D[0][0] = Decimal(-p * (p + 1)) / 4
        D[p][p] = Decimal(p * (p + 1)) / 4
        # reference stiffness Lhat_ij = sum_q w_q D_qi D_qj (GLL quadrature)
        L = [[sum(w[q] * D[q][i] * D[q][j] for q in range(n)) for j in range(n)] for i in range(n)]
        # float(Decimal) is correctly rounded
        xi = np.array([float(t) for t in x])
        wf = np.array([float(t) for t in w])
        Df = np.array([[float(t) for t in row] for row in D])
        Lf = np.array([[float(t) for t in row] for row in L])
    for a in (xi, wf, Df, Lf):
        a.setflags(write=False)
    return xi, wf, Df, Lf


def gll(p: int):
    """GLL nodes xi_0..xi_p and quadrature weights on [-1, 1] (Sec. 2),
    each the correctly rounded double of its exact value."""
    xi, w, _, _ = _gll_exact(p)
    return xi.copy(), w.copy()


def gll_diff(p: int) -> np.ndarray:
    """D[i, j] = phi_j'(xi_i) on the GLL nodes of order p, correctly rounded."""
    return _gll_exact(p)[2].copy()


def lagrange_matrix(xi: np.ndarray, x: np.ndarray) -> np.ndarray:
    """J[i, k] = phi_k(x_i): Lagrange polynomials on nodes xi evaluated at x."""
    n = len(xi)
    J = np.ones((len(x), n))
    for k in range(n):
        for j in range(n):
            if j != k:
                J[:, k] *= (x - xi[j]) / (xi[k] - xi[j])
    return J


def diff_matrix(xi: np.ndarray) -> np.ndarray:
    """D[i, j] = phi_j'(xi_i) for arbitrary distinct nodes, in double
    arithmetic (barycentric form; the GLL set uses gll_diff)."""
    n = len(xi)
    c = np.array([np.prod([xi[i] - xi[k] for k in range(n) if k != i]) for i in range(n)])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = c[i] / (c[j] * (xi[i] - xi[j]))
        D[i, i] = sum(1.0 / (xi[i] - xi[k]) for k in range(n) if k != i)
    return D


def element_matrices(p: int, h: float):
    """1D element mass (diagonal, GLL quadrature) and stiffness on width h (Sec. 2, R1).

    M = (h/2) w and L = (2/h) Lhat with Lhat = D^T W D evaluated exactly and
    rounded once (reading R19), then scaled by one double multiplication.
    """
    _, w, _, Lhat = _gll_exact(p)
    M = 0.5 * h * w
    L = (2.0 / h) * Lhat
    return M, L


# ---------------------------------------------------------------------------
# Meshes and assembly (Sec. 2)
# ---------------------------------------------------------------------------


@dataclass
class Mesh1D:
    """Cartesian 1D mesh: element edges x_0 < ... < x_n and boundary type."""

    edges: np.ndarray
    periodic: bool

    @property
    def n(self) -> int:
        return len(self.edges) - 1

    @property
    def h(self) -> np.ndarray:
        return np.diff(self.edges)

    @staticmethod
    def uniform(n: int, length: float, periodic: bool) -> "Mesh1D":
        return Mesh1D(np.linspace(0.0, length, n + 1), periodic)

    def nodes(self, p: int) -> int:
        """Global node count per direction (Dirichlet: wall nodes included)."""
        return self.n * p if self.periodic else self.n * p + 1

    def gidx(self, p: int) -> np.ndarray:
        """gidx[e, k]: global node of local node k of element e."""
        g = np.arange(self.n)[:, None] * p + np.arange(p + 1)[None, :]
        return g % self.nodes(p) if self.periodic else g

    def unknown(self, p: int) -> np.ndarray:
        """Mask of unknown nodes (Dirichlet wall nodes are not unknowns)."""
        m = np.ones(self.nodes(p), dtype=bool)
        if not self.periodic:
            m[0] = m[-1] = False
        return m

    def coords(self, p: int) -> np.ndarray:
        xi, _ = gll(p)
        x = np.zeros(self.nodes(p))
        g = self.gidx(p)
        for e in reversed(range(self.n)):
            x[g[e]] = self.edges[e] + 0.5 * (1.0 + xi) * self.h[e]
        if not self.periodic:
            x[-1] = self.edges[-1]
        return x

    def neighbour(self, e: int, side: int):
        """Index of the neighbour of element e on side -1/+1, None at a wall."""
        f = e + side
        if 0 <= f < self.n:
            return f
        return f % self.n if self.periodic else None


def assemble_1d(mesh: Mesh1D, p: int):
    """Assembled global 1D mass (diagonal, as a vector) and stiffness (dense)."""
    N = mesh.nodes(p)
    M = np.zeros(N)
    L = np.zeros((N, N))
    g = mesh.gidx(p)
    for e in range(mesh.n):
        Me, Le = element_matrices(p, mesh.h[e])
        M[g[e]] += Me
        L[np.ix_(g[e], g[e])] += Le
    return M, L


def overlap_rule(rule, p_l: int) -> int:
    """n_{o,l} for level order p_l (Sec. 4; capped at p_l - 1, reading R9)."""
    if isinstance(rule, int):
        n = rule
    elif rule == "floor8":
        n = p_l // 8
    elif rule == "ceil8":
        n = -(-p_l // 8)
    elif rule == "ceil2":
        n = -(-p_l // 2)
    else:
        raise ValueError(rule)
    return max(0, min(n, p_l - 1))


def mult_colour_count(mesh: Mesh1D) -> int:
    """Colour classes per direction of the coloured multiplicative order:
    3 on a Dirichlet mesh, the smallest divisor q >= 3 of n on a periodic one
    (so that e and e + q * j share a class also across the wrap)."""
    if not mesh.periodic:
        return 3
    return next(q for q in range(3, mesh.n + 1) if mesh.n % q == 0)


# ---------------------------------------------------------------------------
# Weight functions (Sec. 3.1, Eq. (weight function), Eq. (shape function),
# Table (weighting))
# ---------------------------------------------------------------------------


def phi_hat(kappa, x):
    """Shape functions of Table (weighting)."""
    x = np.asarray(x, dtype=np.float64)
    if kappa == 1:
        return x.copy()
    if kappa == 3:
        return (3 * x - x**3) / 2
    if kappa == 5:
        return (15 * x - 10 * x**3 + 3 * x**5) / 8
    if kappa == 7:
        return (35 * x - 35 * x**3 + 21 * x**5 - 5 * x**7) / 16
    if kappa == "t":
        return np.sign(x)
    raise ValueError(kappa)


def phi(kappa, x):
    """Eq. (shape function): phi_hat on the open interval (-1,1), sgn else (R3)."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(np.abs(x) < 1.0, phi_hat(kappa, np.clip(x, -1, 1)), np.sign(x))


def phi_blend(kt, x):
    """Shape function of continuous degree kt in [1, 7]: convex blend of the two
    neighbouring odd degrees of Table (weighting) (learned weights, R16)."""
    t = min(3.0, max(0.0, 0.5 * (kt - 1.0)))
    k0 = min(2, int(t))
    fr = t - k0
    return (1 - fr) * phi(2 * k0 + 1, x) + fr * phi(2 * k0 + 3, x)


# ---------------------------------------------------------------------------
# One multigrid level: operator, subdomains, FDM factors, weights
# ---------------------------------------------------------------------------


@dataclass
class Sub1D:
    """1D factors of the subdomains of one element row/column (Sec. 3.1)."""

    g: np.ndarray       # global indices of the window nodes that are solved for
    k: np.ndarray       # their element-local indices (-n_o .. p + n_o)
    S: np.ndarray       # generalised eigenvectors, S^T M~ S = I
    lam: np.ndarray     # generalised eigenvalues
    w: np.ndarray       # 1D weights over the window nodes


class Level:
    """Operator and Schwarz data at polynomial order p on a Cartesian mesh."""

    def __init__(self, mx: Mesh1D, my: Mesh1D, p: int, n_o: int, weight=5, nu=None, learned=None):
        self.mx, self.my, self.p, self.n_o, self.weight = mx, my, p, n_o, weight
        # learned weights: (params_x, params_y), each (n+1, 2) arrays of (s, kt)
        # per interface i between elements i-1 and i
        self.learned = learned
        self.NX, self.NY = mx.nodes(p), my.nodes(p)
        self.unknown = my.unknown(p)[:, None] & mx.unknown(p)[None, :]
        self.gx, self.gy = mx.gidx(p), my.gidx(p)
        # element matrices, per element, per direction
        ex = [element_matrices(p, h) for h in mx.h]
        ey = [element_matrices(p, h) for h in my.h]
        self.Mx = np.array([m for m, _ in ex])
        self.Lx = np.array([l for _, l in ex])
        self.My = np.array([m for m, _ in ey])
        self.Ly = np.array([l for _, l in ey])
        self.Mx_glob, self.Lx_glob = assemble_1d(mx, p)
        self.My_glob, self.Ly_glob = assemble_1d(my, p)
        self.nu = None
        if nu is not None:
            self._setup_variable(nu)
        self.sub_x = [self._sub1d(mx, e, self.Mx_glob, self.Lx_glob, 0) for e in range(mx.n)]
        self.sub_y = [self._sub1d(my, e, self.My_glob, self.Ly_glob, 1) for e in range(my.n)]
        if weight == "a":
            self._arith_weights()

    # -- operator ------------------------------------------------------------
    def _setup_variable(self, nu):
        """Variable diffusivity nu(x, y) sampled at the GLL nodes (Sec. 4.3)."""
        xi, w = gll(self.p)
        self.D = gll_diff(self.p)
        self.wq = w
        X = self.mx.coords(self.p)
        Y = self.my.coords(self.p)
        # element-local node coordinates (wall/periodic duplicates are taken
        # from the element's own geometry)
        xe = self.mx.edges[:-1, None] + 0.5 * (1 + xi)[None, :] * self.mx.h[:, None]
        ye = self.my.edges[:-1, None] + 0.5 * (1 + xi)[None, :] * self.my.h[:, None]
        self.nu = nu(xe[None, :, None, :], ye[:, None, :, None])  # (ny, nx, j, i)
        # nu_bar_s: GLL-quadrature mean over the embedded element (R10)
        wq2 = np.outer(w, w)
        self.nu_bar = (self.nu * wq2).sum(axis=(2, 3)) / wq2.sum()
        del X, Y

    def apply(self, u: np.ndarray) -> np.ndarray:
        """A u (Eq. (system matrix)), or B(nu) u (Eq. (diffusion)), element by element."""
        u = np.where(self.unknown, u, 0.0)
        GY = self.gy[:, None, :, None]
        GX = self.gx[None, :, None, :]
        U = u[GY, GX]  # (ny, nx, j, i): gather of the element coefficients
        if self.nu is None:
            # (M_y,e (x) L_x,e + L_y,e (x) M_x,e) u_e
            V = (self.My[:, None, :, None] * (U @ np.swapaxes(self.Lx, 1, 2)[None])
                 + self.Mx[None, :, None, :] * (self.Ly[:, None] @ U))
        else:
            # weak form of -div(nu grad u) with GLL quadrature:
            # sum_q w_q J nu_q (grad phi_a)_q . (grad u)_q
            hx = self.mx.h[None, :, None, None]
            hy = self.my.h[:, None, None, None]
            D = self.D
            ux = (U @ D.T) * (2.0 / hx)            # du/dx at the nodes
            uy = (D @ U) * (2.0 / hy)              # du/dy at the nodes
            wq2 = np.outer(self.wq, self.wq)[None, None]
            jac = 0.25 * hx * hy
            fx = wq2 * jac * self.nu * ux
            fy = wq2 * jac * self.nu * uy
            V = (fx @ D) * (2.0 / hx) + (D.T @ fy) * (2.0 / hy)
        flat = (GY * self.NX + GX)
        flat = np.broadcast_to(flat, V.shape)
        out = np.bincount(flat.ravel(), weights=V.ravel(), minlength=self.NY * self.NX)
        out = out.reshape(self.NY, self.NX)
        return np.where(self.unknown, out, 0.0)

    def mass(self, f_nodal: np.ndarray) -> np.ndarray:
        """b = M_2D f with M_2D = M_y (x) M_x (GLL quadrature of f against phi_i)."""
        b = self.My_glob[:, None] * self.Mx_glob[None, :] * f_nodal
        b = np.where(self.unknown, b, 0.0)
        if self.mx.periodic and self.my.periodic:
            b = b - b.mean()
        return b

    # -- subdomains, FDM factors and weights (Sec. 3.1) ------------------------
    def _positions(self, mesh: Mesh1D, e: int, k: np.ndarray) -> np.ndarray:
        """Window node positions relative to the left interface x_L of element e."""
        xi, _ = gll(self.p)
        p = self.p
        h = mesh.h
        s = np.empty(len(k))
        for t, kk in enumerate(k):
            if kk < 0:
                hl = h[mesh.neighbour(e, -1)]
                s[t] = -(1.0 - xi[p + kk]) * hl / 2
            elif kk <= p:
                s[t] = (1.0 + xi[kk]) * h[e] / 2
            else:
                hr = h[mesh.neighbour(e, +1)]
                s[t] = h[e] + (1.0 + xi[kk - p]) * hr / 2
        return s

    def _weights_1d(self, mesh: Mesh1D, e: int, k: np.ndarray, axis: int = 0) -> np.ndarray:
        """1D weights of Eq. (weight function), readings R3-R5 (learned: R16)."""
        if self.weight == "I":
            return np.ones(len(k))
        if self.weight == "a":
            return np.ones(len(k))  # replaced by C^+ in _arith_weights
        xi, _ = gll(self.p)
        dO = xi[self.n_o + 1] + 1.0  # Eq. (overlap width)
        h = mesh.h
        s = self._positions(mesh, e, k)
        left, right = mesh.neighbour(e, -1), mesh.neighbour(e, +1)
        if self.weight == "learned":
            prm = np.asarray(self.learned[axis])
            il, ir = e, (e + 1) % mesh.n if mesh.periodic else e + 1
            (sl, kl), (sr, kr) = prm[il], prm[ir]
            shape_l = lambda x: phi_blend(kl, x)
            shape_r = lambda x: phi_blend(kr, x)
        else:
            sl = sr = 1.0
            shape_l = shape_r = lambda x: phi(self.weight, x)
        if left is None:
            tl = np.ones(len(k))
        else:
            dl = sl * dO * min(h[left], h[e]) / 2
            tl = shape_l(s / dl)
        if right is None:
            tr = -np.ones(len(k))
        else:
            dr = sr * dO * min(h[e], h[right]) / 2
            tr = shape_r((s - h[e]) / dr)
        return 0.5 * (tl - tr)

    def _sub1d(self, mesh: Mesh1D, e: int, Mg: np.ndarray, Lg: np.ndarray, axis: int = 0) -> Sub1D:
        p, n_o = self.p, self.n_o
        k = np.arange(-n_o, p + n_o + 1)
        g = e * p + k
        N = mesh.nodes(p)
        if mesh.periodic:
            g = g % N
            valid = np.ones(len(k), dtype=bool)
        else:
            valid = (g > 0) & (g < mesh.n * p)
        k, g = k[valid], g[valid]
        if len(np.unique(g)) != len(g):
            raise ValueError("subdomain window wraps onto itself; mesh too small")
        Lt = Lg[np.ix_(g, g)]            # restricted stiffness  R L R^T
        Mt = Mg[g]                       # restricted mass (diagonal)
        lam, S = sla.eigh(Lt, np.diag(Mt))   # L~ s = lambda M~ s,  S^T M~ S = I
        return Sub1D(g=g, k=k, S=S, lam=lam, w=self._weights_1d(mesh, e, k, axis))

    def _arith_weights(self):
        """w_a: W = R_s C^+ R_s^T with C = sum_s R_s^T R_s (Sec. 3.1, R2)."""
        for subs, N in ((self.sub_x, self.NX), (self.sub_y, self.NY)):
            cnt = np.zeros(N)
            for s in subs:
                cnt[s.g] += 1.0
            for s in subs:
                s.w = 1.0 / cnt[s.g]

    def local_solve(self, ex: int, ey: int, rs: np.ndarray) -> np.ndarray:
        """Delta u_s = A_ss^{-1} r_s by fast diagonalisation (Eq. (FDM))."""
        sx, sy = self.sub_x[ex], self.sub_y[ey]
        X = sy.S.T @ rs @ sx.S                        # (S_y^T (x) S_x^T) r_s
        X = X / (sy.lam[:, None] + sx.lam[None, :])   # (I (x) Lam_x + Lam_y (x) I)^{-1}
        du = sy.S @ X @ sx.S.T                        # (S_y (x) S_x)
        if self.nu is not None:
            du = du / self.nu_bar[ey, ex]             # Eq. (subproblem:solution)
        return du

    def schwarz_correction(self, r: np.ndarray) -> np.ndarray:
        """sum_s R_s^T W A_ss^{-1} R_s r (Eq. (correction:global))."""
        du = np.zeros_like(r)
        for ey, sy in enumerate(self.sub_y):
            for ex, sx in enumerate(self.sub_x):
                rs = r[np.ix_(sy.g, sx.g)]                           # R_s r
                dus = self.local_solve(ex, ey, rs)
                du[np.ix_(sy.g, sx.g)] += np.outer(sy.w, sx.w) * dus  # R_s^T W
        return du

    def wschwarz(self, u: np.ndarray, f: np.ndarray, n_it: int) -> np.ndarray:
        """Alg. 2, weighted additive Schwarz, n_it sweeps."""
        for _ in range(n_it):
            r = f - self.apply(u)
            u = u + self.schwarz_correction(r)
        return u

    def mult_order(self, order: str = "lex") -> list:
        """Subdomain sequence of one forward sweep of Alg. 1 as (ex, ey) pairs.

        "lex": the paper's order, s = e = 1..n_el (element rows of x fastest).
        "colour": the same subdomains grouped by colour class
        c = cy * qx + cx, with cx = ex mod qx and cy = ey mod qy, classes in
        increasing c and lexicographic inside a class (mult_colour_count gives
        q).  Two subdomains of one class lie at least q >= 3 elements apart in
        x or in y, also across a periodic wrap (q divides n), so the update of
        one (its element's closed node set, and the residual on the element
        and its neighbours) never reaches the other's window (n_o < p): within
        a class the order does not change the result.
        """
        nx, ny = self.mx.n, self.my.n
        lex = [(ex, ey) for ey in range(ny) for ex in range(nx)]
        if order == "lex":
            return lex
        if order != "colour":
            raise ValueError(order)
        qx, qy = mult_colour_count(self.mx), mult_colour_count(self.my)
        return sorted(lex, key=lambda s: ((s[1] % qy) * qx + s[0] % qx, s[1], s[0]))

    def mschwarz(self, u: np.ndarray, f: np.ndarray, n_it: int, order: str = "lex") -> np.ndarray:
        """Alg. 1, multiplicative Schwarz: the subdomains in sequence, reversed on
        even sweeps, the residual recomputed before each local solve.

        Reading R15: the local problem is solved on the whole extended
        subdomain (Sec. 3.1), and R_s^T of the update line adds the solution
        on the nodes of the element itself, its boundary nodes included
        (element-local indices 0..p), without weights.
        """
        seq = self.mult_order(order)
        for i in range(1, n_it + 1):
            for ex, ey in (seq if i % 2 == 1 else seq[::-1]):
                sx, sy = self.sub_x[ex], self.sub_y[ey]
                r = f - self.apply(u)
                rs = r[np.ix_(sy.g, sx.g)]
                du = self.local_solve(ex, ey, rs)
                own_x = (sx.k >= 0) & (sx.k <= self.p)
                own_y = (sy.k >= 0) & (sy.k <= self.p)
                u = u.copy()
                u[np.ix_(sy.g[own_y], sx.g[own_x])] += du[np.ix_(own_y, own_x)]
        return u

    def dense_operator(self) -> np.ndarray:
        """Dense A over the unknowns, by applying the operator to unit vectors."""
        idx = np.flatnonzero(self.unknown.ravel())
        A = np.zeros((len(idx), len(idx)))
        e = np.zeros(self.NY * self.NX)
        for c, j in enumerate(idx):
            e[j] = 1.0
            A[:, c] = self.apply(e.reshape(self.NY, self.NX)).ravel()[idx]
            e[j] = 0.0
        return A


# ---------------------------------------------------------------------------
# Grid transfer (Sec. 3.2): embedded interpolation and its transpose
# ---------------------------------------------------------------------------


def prolongation_1d(mesh: Mesh1D, p_f: int, p_c: int) -> sp.csr_matrix:
    """Global 1D interpolation P from order p_c to p_f on the same elements."""
    xf, _ = gll(p_f)
    xc, _ = gll(p_c)
    J = lagrange_matrix(xc, xf)   # J[i, k] = phi_k^{(p_c)}(xi_i^{(p_f)})
    P = np.zeros((mesh.nodes(p_f), mesh.nodes(p_c)))
    gf, gc = mesh.gidx(p_f), mesh.gidx(p_c)
    for e in range(mesh.n):
        # interface rows are written by both elements with identical values
        P[np.ix_(gf[e], gc[e])] = J
    return sp.csr_matrix(P)


# ---------------------------------------------------------------------------
# The multigrid hierarchy, V-cycle (Alg. 3) and MGCG (Alg. 4)
# ---------------------------------------------------------------------------


@dataclass
class Hierarchy:
    """Levels p_l = 2^l, l = 0..L, with transfer operators and coarse solver."""

    mx: Mesh1D
    my: Mesh1D
    p: int
    overlap: object = 1
    weight: object = 5
    nu: object = None
    smoother: str = "add"
    mult_order: str = "lex"  # subdomain order of Alg. 1: "lex" or "colour"
    learned: object = None  # (params_x, params_y): arrays [level][interface][2]
    levels: list = field(default_factory=list)

    def __post_init__(self):
        L = int(round(math.log2(self.p)))
        if 2**L != self.p:
            raise ValueError("p must be a power of two (p_l = 2^l)")
        self.L = L
        self.levels = []
        for l in range(L + 1):
            pl = 2**l
            no = overlap_rule(self.overlap, pl) if l > 0 else 0
            if l == 0:
                lev = _CoarseLevel(self.mx, self.my, self.nu)
            else:
                lrn = None if self.learned is None else (self.learned[0][l], self.learned[1][l])
                lev = Level(self.mx, self.my, pl, no, weight=self.weight, nu=self.nu, learned=lrn)
            self.levels.append(lev)
        self.Px = [None] + [prolongation_1d(self.mx, 2**l, 2**(l - 1)) for l in range(1, L + 1)]
        self.Py = [None] + [prolongation_1d(self.my, 2**l, 2**(l - 1)) for l in range(1, L + 1)]

    @property
    def top(self) -> Level:
        return self.levels[-1]

    def prolong(self, l: int, uc: np.ndarray) -> np.ndarray:
        """I_l u_{l-1} = (P_y (x) P_x) u_{l-1}."""
        return np.asarray(self.Px[l] @ np.asarray(self.Py[l] @ uc).T).T

    def restrict(self, l: int, rf: np.ndarray) -> np.ndarray:
        """I_l^T r_l = (P_y^T (x) P_x^T) r_l; coarse wall entries are not unknowns."""
        rc = np.asarray(self.Px[l].T @ np.asarray(self.Py[l].T @ rf).T).T
        return np.where(self.levels[l - 1].unknown, rc, 0.0)

    def smooth(self, l: int, u, f, n):
        lev = self.levels[l]
        if n <= 0:
            return u
        if self.smoother == "mult":
            return lev.mschwarz(u, f, n, self.mult_order)
        return lev.wschwarz(u, f, n)

    def vcycle(self, u: np.ndarray, f: np.ndarray, ns1, ns2) -> np.ndarray:
        """Alg. 3 MultigridCycle(u, f, n_s); ns1/ns2 are per-level step counts."""
        L = self.L
        us = [None] * (L + 1)
        fs = [None] * (L + 1)
        us[L], fs[L] = u, f
        for l in range(L, 0, -1):
            if l < L:
                us[l] = np.zeros_like(fs[l])           # R8
            us[l] = self.smooth(l, us[l], fs[l], ns1[l])   # pre-smoothing
            r = fs[l] - self.levels[l].apply(us[l])
            fs[l - 1] = self.restrict(l, r)           # residual restriction
        us[0] = self.levels[0].solve(fs[0])          # coarse grid solution
        for l in range(1, L + 1):
            us[l] = us[l] + self.prolong(l, us[l - 1])  # correction prolongation
            us[l] = self.smooth(l, us[l], fs[l], ns2[l])  # post-smoothing
        return us[L]

    def steps(self, n1: int, n2: int, variable: bool = False):
        """Per-level smoothing counts; the variable V-cycle doubles them per level."""
        L = self.L
        f = (lambda l: 2 ** (L - l)) if variable else (lambda l: 1)
        return [n1 * f(l) for l in range(L + 1)], [n2 * f(l) for l in range(L + 1)]

    def mg_solve(self, u, f, n1=1, n2=0, reduction=1e-10, max_cycles=200, variable=False):
        """Stand-alone MG(n1, n2) iteration until ||r|| drops by `reduction`."""
        ns1, ns2 = self.steps(n1, n2, variable)
        A = self.top.apply
        hist = [np.linalg.norm(f - A(u))]
        for _ in range(max_cycles):
            u = self.vcycle(u, f, ns1, ns2)
            hist.append(np.linalg.norm(f - A(u)))
            if hist[-1] <= reduction * hist[0]:
                break
        return u, hist

    def mgcg(self, u, f, n1=1, n2=0, tol=1e-10, i_max=200, variable=False,
             precondition=True, r_max=None):
        """Alg. 4 inexact MG-preconditioned CG (reading R6 for the beta line).

        Stops when ||r_i|| <= r_max, r_max = tol * ||r_0|| unless given.
        Returns (u, iterations, residual-norm history).
        """
        ns1, ns2 = self.steps(n1, n2, variable)
        A = self.top.apply
        M = (lambda r: self.vcycle(np.zeros_like(r), r, ns1, ns2)) if precondition else (lambda r: r.copy())
        r_old = np.zeros_like(f)
        r = f - A(u)
        p = M(r)
        delta = np.vdot(p, r)
        hist = [np.linalg.norm(r)]
        if r_max is None:
            r_max = tol * hist[0]
        it = 0
        for i in range(1, i_max + 1):
            it = i
            q = A(p)
            alpha = delta / np.vdot(p, q)
            u = u + alpha * p
            r = r - alpha * q
            hist.append(np.linalg.norm(r))
            if hist[-1] <= r_max:
                break
            z = M(r)
            beta = np.vdot(z, r - r_old) / delta
            p = z + beta * p
            delta = np.vdot(z, r)
            r_old = r.copy()
        return u, it, hist


class _CoarseLevel:
    """Level 0 (p = 1): operator and the coarse solution u_0 = A_0^+ f_0 (R7)."""

    def __init__(self, mx: Mesh1D, my: Mesh1D, nu=None):
        self.lev = Level(mx, my, 1, 0, weight="I", nu=nu)
        self.mx, self.my, self.p = mx, my, 1
        self.unknown = self.lev.unknown
        self.NX, self.NY = self.lev.NX, self.lev.NY
        self.idx = np.flatnonzero(self.unknown.ravel())
        if nu is None:
            # dense A_0 from Eq. (system matrix) over the unknowns
            A = (np.kron(np.diag(self.lev.My_glob), self.lev.Lx_glob)
                 + np.kron(self.lev.Ly_glob, np.diag(self.lev.Mx_glob)))
            A = A[np.ix_(self.idx, self.idx)]
        else:
            A = self.lev.dense_operator()
        self.singular = mx.periodic and my.periodic
        n = len(self.idx)
        if self.singular:
            c = np.trace(A) / n / n
            A = A + c * np.ones((n, n))   # (A + c 1 1^T)^{-1} on 1-perp is A^+
        self.chol = sla.cho_factor(A)

    def apply(self, u):
        return self.lev.apply(u)

    def solve(self, f: np.ndarray) -> np.ndarray:
        b = f.ravel()[self.idx]
        if self.singular:
            b = b - b.mean()   # project the right side onto the range of A_0
        x = sla.cho_solve(self.chol, b)
        if self.singular:
            x = x - x.mean()
        u = np.zeros(self.NY * self.NX)
        u[self.idx] = x
        return u.reshape(self.NY, self.NX)


# ---------------------------------------------------------------------------
# Convergence metrics (Sec. 4)
# ---------------------------------------------------------------------------


def rate(hist) -> float:
    """Average logarithmic convergence rate r_bar = log10(|r0|/|rn|)/n."""
    n = len(hist) - 1
    return math.log10(hist[0] / hist[-1]) / n


def n10(rbar: float) -> int:
    """Cycles to a 1e10 reduction: nearest integer >= 10 / r_bar."""
    return int(math.ceil(10.0 / rbar - 1e-12))


def uniform_hierarchy(nx, ny, p, lx=1.0, ly=1.0, periodic=False, **kw) -> Hierarchy:
    return Hierarchy(Mesh1D.uniform(nx, lx, periodic), Mesh1D.uniform(ny, ly, periodic), p, **kw)
