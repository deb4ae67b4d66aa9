"""Pins of the CPU oracle against closed forms, textbook identities and values
derived by hand from the paper's formulas (no GPU).

Each check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import sem_oracle as O
from tests._golden import rows

# ---------------------------------------------------------------- Sec. 2 basics


def test_gll_closed_form_p4():
    xi, w = O.gll(4)
    s = math.sqrt(3.0 / 7.0)
    np.testing.assert_allclose(xi, [-1, -s, 0, s, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


def _cr_sqrt(num, den):
    """Correctly rounded sqrt(num / den) (60-digit decimal square root)."""
    from decimal import Decimal, localcontext
    with localcontext() as c:
        c.prec = 60
        return float((Decimal(num) / Decimal(den)).sqrt())


def test_gll_closed_forms_are_correctly_rounded():
    """Reading R19: nodes, weights, D and Lhat equal, bit for bit, the
    correctly rounded closed forms (Python's rational division and the
    decimal square root round correctly)."""
    cases = {
        1: ([-1.0, 1.0], [1.0, 1.0]),
        2: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
        3: ([-1.0, -_cr_sqrt(1, 5), _cr_sqrt(1, 5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
        4: ([-1.0, -_cr_sqrt(3, 7), 0.0, _cr_sqrt(3, 7), 1.0], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
    }
    for p, (x, w) in cases.items():
        xi, wq = O.gll(p)
        assert np.array_equal(xi, np.array(x)) and np.array_equal(wq, np.array(w)), p
    # p = 2 on [-1, 1]: phi_j' at the nodes and the exact stiffness (1/6)[7 -8 1; -8 16 -8; 1 -8 7]
    assert np.array_equal(O.gll_diff(2), np.array([[-1.5, 2.0, -0.5], [-0.5, 0.0, 0.5], [0.5, -2.0, 1.5]]))
    _, L2 = O.element_matrices(2, 2.0)
    assert np.array_equal(L2, np.array([[7 / 6, -4 / 3, 1 / 6], [-4 / 3, 8 / 3, -4 / 3], [1 / 6, -4 / 3, 7 / 6]]))
    _, L1 = O.element_matrices(1, 2.0)
    assert np.array_equal(L1, np.array([[0.5, -0.5], [-0.5, 0.5]]))


@pytest.mark.parametrize("p", [3, 5, 8, 13, 16, 24, 32])
def test_reference_stiffness_is_correctly_rounded(p):
    """Lhat (h = 2) keeps the exact identities bit for bit (symmetry,
    centro-symmetry of the GLL nodes) and its rows, whose exact sums vanish
    (constants have zero derivative), sum exactly to at most half an ulp per
    entry: a bound that a correctly rounded matrix meets and a plain double
    evaluation of D^T W D (tens of ulps off at p = 16) does not."""
    import math as m
    _, L = O.element_matrices(p, 2.0)
    assert np.array_equal(L, L.T)
    assert np.array_equal(L, L[::-1, ::-1])
    for row in L:
        assert abs(m.fsum(row)) <= 0.5 * sum(np.spacing(np.abs(row)))
    # the same bound fails for the double-precision evaluation at this size
    if p == 16:
        xi, w = O.gll(p)
        D = O.diff_matrix(xi)
        Ld = D.T @ (w[:, None] * D)
        assert any(abs(m.fsum(r)) > 0.5 * sum(np.spacing(np.abs(r))) for r in Ld)
    # interior diagonal of D is exactly zero, the end points -p(p+1)/4, p(p+1)/4
    D = O.gll_diff(p)
    assert D[0, 0] == -p * (p + 1) / 4 and D[p, p] == p * (p + 1) / 4
    assert np.all(np.diag(D)[1:-1] == 0.0)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 13, 16, 32])
def test_gll_quadrature_exact_to_degree_2p_minus_1(p):
    xi, w = O.gll(p)
    assert abs(w.sum() - 2.0) < 1e-13
    for k in range(0, 2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, xi**k) - exact) < 1e-12, (p, k)
    # P'_p vanishes at the interior nodes
    c = np.zeros(p + 1)
    c[p] = 1
    if p >= 2:
        d = np.polynomial.legendre.legval(xi[1:-1], np.polynomial.legendre.legder(c))
        assert np.abs(d).max() < 1e-10 * p * p


@pytest.mark.parametrize("p", [2, 4, 7, 16])
def test_diff_matrix_differentiates_polynomials(p):
    xi, _ = O.gll(p)
    D = O.diff_matrix(xi)
    for k in range(0, p + 1):
        exact = k * xi ** (k - 1) if k else np.zeros_like(xi)
        assert np.abs(D @ xi**k - exact).max() < 1e-10 * max(1, k) * p


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8])
def test_element_stiffness_equals_exact_integral(p):
    """L = (2/h) D^T W D equals int phi_i' phi_j' dx computed with numpy polynomials."""
    h = 0.37
    M, L = O.element_matrices(p, h)
    xi, w = O.gll(p)
    # Lagrange basis in the monomial basis on [-1, 1], differentiated and
    # integrated exactly (independent of the GLL quadrature)
    V = np.vander(xi, p + 1, increasing=True)
    C = np.linalg.inv(V)  # column j = monomial coefficients of phi_j
    Lex = np.zeros((p + 1, p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            di = np.polynomial.polynomial.polyder(C[:, i])
            dj = np.polynomial.polynomial.polyder(C[:, j])
            prod = np.polynomial.polynomial.polymul(di, dj)
            integ = np.polynomial.polynomial.polyint(prod)
            Lex[i, j] = np.polynomial.polynomial.polyval(1, integ) - np.polynomial.polynomial.polyval(-1, integ)
    np.testing.assert_allclose(L, (2.0 / h) * Lex, atol=1e-9 * np.abs(Lex).max() / h)
    assert np.allclose(L, L.T)
    assert np.abs(L @ np.ones(p + 1)).max() < 1e-12 / h
    assert np.linalg.eigvalsh(L).min() > -1e-12 / h
    assert abs(M.sum() - h) < 1e-14


# ----------------------------------------------- Eq. (system matrix) properties


def _small(periodic, nx=3, ny=2, p=4, lx=1.0, ly=1.0, edges=None):
    mx = O.Mesh1D.uniform(nx, lx, periodic) if edges is None else O.Mesh1D(np.asarray(edges), periodic)
    my = O.Mesh1D.uniform(ny, ly, periodic)
    return O.Level(mx, my, p, 1, weight=5)


@pytest.mark.parametrize("periodic", [False, True])
def test_operator_symmetric_definite(periodic):
    lev = _small(periodic)
    A = lev.dense_operator()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A)
    if periodic:
        assert abs(ev[0]) < 1e-10 * ev[-1] and ev[1] > 1e-6 * ev[-1]
        assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-11 * np.abs(A).max()
    else:
        assert ev[0] > 1e-6 * ev[-1]


@pytest.mark.parametrize("periodic", [False, True])
def test_operator_equals_tensor_form(periodic):
    """Element-by-element apply equals M_y (x) L_x + L_y (x) M_x (Eq. (system matrix))."""
    lev = _small(periodic, edges=[0.0, 0.2, 0.7, 1.0])
    A = lev.dense_operator()
    # kron of the assembled 1D matrices: a different route than the element loop
    Ak = np.kron(np.diag(lev.My_glob), lev.Lx_glob) + np.kron(lev.Ly_glob, np.diag(lev.Mx_glob))
    idx = np.flatnonzero(lev.unknown.ravel())
    np.testing.assert_allclose(A, Ak[np.ix_(idx, idx)], atol=1e-11 * np.abs(A).max())


def test_operator_invariant_under_uniform_scaling():
    a = _small(False, lx=1.0, ly=1.0).dense_operator()
    b = _small(False, lx=2.0, ly=2.0).dense_operator()
    np.testing.assert_allclose(a, b, atol=1e-11 * np.abs(a).max())


def test_spectral_convergence_manufactured_solution():
    """Dense solve of A u = M f on Dirichlet [0,1]^2: error decays exponentially in p."""
    errs = []
    for p in [2, 4, 6, 8, 10, 12]:
        lev = O.Level(O.Mesh1D.uniform(2, 1.0, False), O.Mesh1D.uniform(2, 1.0, False), p, 1)
        X, Y = lev.mx.coords(p), lev.my.coords(p)
        ue = np.sin(np.pi * X[None, :]) * np.sin(np.pi * Y[:, None])
        b = lev.mass(2 * np.pi**2 * ue)
        A = lev.dense_operator()
        idx = np.flatnonzero(lev.unknown.ravel())
        x = np.linalg.solve(A, b.ravel()[idx])
        errs.append(np.abs(x - ue.ravel()[idx]).max())
    assert all(errs[i + 1] < 0.1 * errs[i] for i in range(4))
    assert errs[3] < 1e-9 and errs[5] < 1e-12


# ----------------------------------------------------- Eq. (FDM), subdomains


def _window_dense(lev, ex, ey):
    A = lev.dense_operator()
    idx = np.flatnonzero(lev.unknown.ravel())
    pos = {g: c for c, g in enumerate(idx)}
    sx, sy = lev.sub_x[ex], lev.sub_y[ey]
    rows_ = [pos[gy * lev.NX + gx] for gy in sy.g for gx in sx.g]
    return A[np.ix_(rows_, rows_)]


@pytest.mark.parametrize("periodic,p,n_o,edges", [
    (False, 4, 1, None), (False, 4, 2, None), (True, 4, 1, None), (False, 8, 3, None),
    (False, 4, 2, [0.0, 0.1, 0.5, 0.55, 1.0]), (True, 2, 1, None)])
def test_fdm_equals_dense_subdomain_solve(periodic, p, n_o, edges):
    nx = 4
    mx = O.Mesh1D.uniform(nx, 1.0, periodic) if edges is None else O.Mesh1D(np.asarray(edges), periodic)
    my = O.Mesh1D.uniform(3, 1.3, periodic)
    lev = O.Level(mx, my, p, n_o, weight=5)
    rng = np.random.default_rng(0)
    for ex in range(nx):
        for ey in range(3):
            Ass = _window_dense(lev, ex, ey)
            sx, sy = lev.sub_x[ex], lev.sub_y[ey]
            rs = rng.standard_normal((len(sy.g), len(sx.g)))
            du = lev.local_solve(ex, ey, rs)
            ref = sla.solve(Ass, rs.ravel(), assume_a="pos")
            np.testing.assert_allclose(du.ravel(), ref, rtol=0, atol=1e-11 * np.abs(ref).max())
            # the window: element nodes plus n_o layers, outer layer and walls excluded
            m = p + 1 + 2 * n_o
            assert len(sx.g) <= m and len(sx.g) >= m - n_o - 1


def test_fdm_factor_normalisation():
    lev = O.Level(O.Mesh1D.uniform(4, 1.0, False), O.Mesh1D.uniform(4, 1.0, False), 8, 2)
    for s, Mg, Lg in [(lev.sub_x[0], lev.Mx_glob, lev.Lx_glob), (lev.sub_x[2], lev.Mx_glob, lev.Lx_glob)]:
        Mt = np.diag(Mg[s.g])
        Lt = Lg[np.ix_(s.g, s.g)]
        np.testing.assert_allclose(s.S.T @ Mt @ s.S, np.eye(len(s.g)), atol=1e-12)
        np.testing.assert_allclose(s.S.T @ Lt @ s.S, np.diag(s.lam), atol=1e-9 * s.lam.max())


# --------------------------------------- Eq. (weight function), Table (weighting)


def test_weights_match_hand_derived_values():
    lev_by_kappa = {}
    for row in rows("weights_p4_no1.txt"):
        kappa = row[0] if row[0] == "t" else int(row[0])
        want = np.array([float(v) for v in row[1:]])
        lev = lev_by_kappa.setdefault(kappa, O.Level(O.Mesh1D.uniform(8, 2.0, True),
                                                     O.Mesh1D.uniform(8, 2.0, True), 4, 1, weight=kappa))
        s = lev.sub_x[3]
        assert list(s.k) == list(range(-1, 6))
        np.testing.assert_allclose(s.w, want, atol=1e-14)


@pytest.mark.parametrize("kappa", [1, 3, 5, 7])
def test_shape_function_conditions(kappa):
    """phi_hat(+-1) = +-1, derivatives 1..(kappa-1)/2 vanish at +-1, monotone inside."""
    x = np.linspace(-1, 1, 4 * kappa + 7)
    c = np.polynomial.polynomial.polyfit(x, O.phi_hat(kappa, x), kappa)
    assert abs(np.polynomial.polynomial.polyval(1.0, c) - 1) < 1e-12
    assert abs(np.polynomial.polynomial.polyval(-1.0, c) + 1) < 1e-12
    for k in range(1, (kappa - 1) // 2 + 1):
        d = np.polynomial.polynomial.polyder(c, k)
        assert abs(np.polynomial.polynomial.polyval(1.0, d)) < 1e-9
        assert abs(np.polynomial.polynomial.polyval(-1.0, d)) < 1e-9
    # the next derivative does not vanish (degree is exactly kappa)
    d = np.polynomial.polynomial.polyder(c, (kappa + 1) // 2)
    assert abs(np.polynomial.polynomial.polyval(1.0, d)) > 1e-3
    xx = np.linspace(-0.999, 0.999, 2001)
    assert np.all(np.diff(O.phi_hat(kappa, xx)) > 0)


@pytest.mark.parametrize("kappa", [1, 3, 5, 7, "t", "a"])
@pytest.mark.parametrize("periodic,p,n_o,edges", [
    (True, 2, 1, None), (True, 4, 1, None), (False, 16, 2, None), (True, 32, 4, None),
    (False, 8, 5, None), (False, 8, 2, [0.0, 0.05, 0.3, 0.32, 1.0])])
def test_weights_partition_of_unity(kappa, periodic, p, n_o, edges):
    """sum_s R_s^T W_s R_s 1 = 1 on every unknown (telescoping of Eq. (weight function))."""
    mx = O.Mesh1D.uniform(4, 1.0, periodic) if edges is None else O.Mesh1D(np.asarray(edges), periodic)
    lev = O.Level(mx, O.Mesh1D.uniform(4, 1.0, periodic), p, n_o, weight=kappa)
    tot = np.zeros((lev.NY, lev.NX))
    for sy in lev.sub_y:
        for sx in lev.sub_x:
            tot[np.ix_(sy.g, sx.g)] += np.outer(sy.w, sx.w)
    assert np.abs(tot[lev.unknown] - 1).max() < 1e-13
    for s in lev.sub_x:
        assert s.w.min() >= -1e-15 and s.w.max() <= 1 + 1e-15


def test_weights_symmetric_and_half_at_interfaces():
    lev = O.Level(O.Mesh1D.uniform(6, 1.0, True), O.Mesh1D.uniform(6, 1.0, True), 16, 2, weight=5)
    s = lev.sub_x[2]
    np.testing.assert_allclose(s.w, s.w[::-1], atol=1e-15)
    k = list(s.k)
    assert s.w[k.index(0)] == 0.5 and s.w[k.index(16)] == 0.5
    # values derived from Eq. (weight function) for p = 16, n_o = 2
    np.testing.assert_allclose(s.w[:5], [0.11238, 0.365255, 0.5, 0.634745, 0.88762], atol=6e-6)


def test_arithmetic_mean_equals_shape_free_formula_when_overlap_at_most_one():
    """Sec. 3.1 remark: phi_hat = 0 in Eq. (weight function) gives C^+ when delta_O <= 1."""
    p, n_o = 8, 2
    lev = O.Level(O.Mesh1D.uniform(5, 1.0, True), O.Mesh1D.uniform(5, 1.0, True), p, n_o, weight="a")
    xi, _ = O.gll(p)
    dO = xi[n_o + 1] + 1
    assert dO <= 1
    s = lev.sub_x[1]
    # extended standard coordinate of each window node, from the node index
    pos = np.array([xi[k] if 0 <= k <= p else (xi[p + k] - 2 if k < 0 else xi[k - p] + 2) for k in s.k])
    # ties |x| = 1 are classified by index (|x| within rounding of 1 is outside)
    zero_phi = lambda x: np.where(np.abs(x) < 1 - 1e-12, 0.0, np.sign(x))
    w = 0.5 * (zero_phi((pos + 1) / dO) - zero_phi((pos - 1) / dO))
    np.testing.assert_allclose(s.w, w, atol=1e-15)


def test_identity_weights_give_classical_additive_schwarz():
    lev = O.Level(O.Mesh1D.uniform(3, 1.0, False), O.Mesh1D.uniform(3, 1.0, False), 4, 1, weight="I")
    A = lev.dense_operator()
    idx = np.flatnonzero(lev.unknown.ravel())
    pos = {g: c for c, g in enumerate(idx)}
    B = np.zeros_like(A)
    for ey in range(3):
        for ex in range(3):
            sx, sy = lev.sub_x[ex], lev.sub_y[ey]
            r_ = [pos[gy * lev.NX + gx] for gy in sy.g for gx in sx.g]
            B[np.ix_(r_, r_)] += np.linalg.inv(A[np.ix_(r_, r_)])
    r = np.random.default_rng(3).standard_normal((lev.NY, lev.NX)) * lev.unknown
    np.testing.assert_allclose(lev.schwarz_correction(r).ravel()[idx], B @ r.ravel()[idx], atol=1e-11)


# --------------------------------------------------- Sec. 3.2 grid transfer


@pytest.mark.parametrize("pf", [2, 4, 8, 16, 32])
def test_interpolation_exact_for_coarse_polynomials(pf):
    pc = pf // 2
    xf, _ = O.gll(pf)
    xc, _ = O.gll(pc)
    J = O.lagrange_matrix(xc, xf)
    for k in range(pc + 1):
        assert np.abs(J @ xc**k - xf**k).max() < 1e-12
    # the fine stiffness integrates coarse polynomials exactly: J^T L_f J = L_c
    _, Lf = O.element_matrices(pf, 1.0)
    _, Lc = O.element_matrices(pc, 1.0)
    np.testing.assert_allclose(J.T @ Lf @ J, Lc, atol=1e-10 * np.abs(Lc).max())


@pytest.mark.parametrize("periodic", [False, True])
def test_restriction_is_transpose_of_prolongation(periodic):
    H = O.uniform_hierarchy(3, 4, 8, periodic=periodic, overlap=1)
    rng = np.random.default_rng(1)
    for l in range(1, H.L + 1):
        uc = rng.standard_normal((H.levels[l - 1].NY, H.levels[l - 1].NX)) * H.levels[l - 1].unknown
        rf = rng.standard_normal((H.levels[l].NY, H.levels[l].NX)) * H.levels[l].unknown
        a = np.vdot(H.prolong(l, uc), rf)
        b = np.vdot(uc, H.restrict(l, rf))
        assert abs(a - b) < 1e-12 * (abs(a) + 1)


def test_prolongation_reproduces_piecewise_polynomial():
    H = O.uniform_hierarchy(3, 2, 8, periodic=False, overlap=1)
    for l in range(1, H.L + 1):
        pc, pf = 2 ** (l - 1), 2**l
        fc = lambda x, y: x * (1 - x) * y * (1 - y) * (1 + x) ** max(0, pc - 2)
        cx, cy = H.levels[l - 1].mx.coords(pc), H.levels[l - 1].my.coords(pc)
        fxs, fys = H.levels[l].mx.coords(pf), H.levels[l].my.coords(pf)
        if pc >= 2:
            uc = fc(cx[None, :], cy[:, None]) * H.levels[l - 1].unknown
            uf = H.prolong(l, uc)
            np.testing.assert_allclose(uf, fc(fxs[None, :], fys[:, None]) * H.levels[l].unknown, atol=1e-13)


# ----------------------------------------------------- coarse solve, MGCG


@pytest.mark.parametrize("periodic", [False, True])
def test_coarse_solve_is_pseudo_inverse(periodic):
    H = O.uniform_hierarchy(6, 5, 2, periodic=periodic)
    c = H.levels[0]
    f = np.random.default_rng(2).standard_normal((c.NY, c.NX)) * c.unknown
    u = c.solve(f)
    A = c.lev.dense_operator()
    idx = c.idx
    ref = np.linalg.pinv(A, rcond=1e-10, hermitian=True) @ f.ravel()[idx]
    np.testing.assert_allclose(u.ravel()[idx], ref, atol=1e-11 * np.abs(ref).max())


def test_mgcg_with_identity_preconditioner_is_plain_cg():
    """Alg. 4 with MultigridCycle replaced by the identity reproduces textbook CG."""
    H = O.uniform_hierarchy(3, 3, 4, periodic=False)
    lev = H.top
    A = lev.dense_operator()
    idx = np.flatnonzero(lev.unknown.ravel())
    f = np.random.default_rng(4).standard_normal((lev.NY, lev.NX)) * lev.unknown
    x = np.zeros(len(idx))
    b = f.ravel()[idx]
    r = b.copy()
    pp = r.copy()
    rr = r @ r
    hist = [np.sqrt(rr)]
    for _ in range(12):
        q = A @ pp
        a = rr / (pp @ q)
        x = x + a * pp
        r = r - a * q
        rr_new = r @ r
        hist.append(np.sqrt(rr_new))
        pp = r + (rr_new / rr) * pp
        rr = rr_new
    u, it, h2 = O.Hierarchy.mgcg(H, np.zeros_like(f), f, tol=0.0, i_max=12, precondition=False)
    np.testing.assert_allclose(h2, hist, rtol=1e-8)
    np.testing.assert_allclose(u.ravel()[idx], x, atol=1e-10 * np.abs(x).max())


def test_mgcg_solution_equals_dense_solve():
    H = O.uniform_hierarchy(4, 4, 4, periodic=False, overlap=1, weight=5)
    lev = H.top
    X, Y = lev.mx.coords(4), lev.my.coords(4)
    b = lev.mass(2 * np.pi**2 * np.sin(np.pi * X[None, :]) * np.sin(np.pi * Y[:, None]))
    u, it, hist = H.mgcg(np.zeros_like(b), b, tol=1e-12)
    A = lev.dense_operator()
    idx = np.flatnonzero(lev.unknown.ravel())
    ref = np.linalg.solve(A, b.ravel()[idx])
    assert np.abs(u.ravel()[idx] - ref).max() < 1e-10 * np.abs(ref).max()
    assert hist[-1] <= 1e-12 * hist[0] and it <= 14
