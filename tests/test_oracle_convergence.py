"""The oracle reproduces the convergence rates printed in the paper's Tables 1,
3 and 4 (Sec. 4): the strongest end-to-end pin of the whole method (operator,
subdomains, FDM, weights, V-cycle, transfer, coarse solve and MGCG)."""
import math

import numpy as np
import pytest

import sem_inputs as SI
from oracle import sem_oracle as O
from tests._golden import rows


def _close(got, want):
    return abs(got - want) <= 0.05 * want + 0.02


def _n10_close(got, want):
    # n_10 = ceil(10 / r_bar) magnifies small differences of slow rates
    return abs(got - want) <= max(1, 0.05 * want)


def _periodic_case(p, weight, overlap, n=8, AR=1, seed=1):
    H = O.Hierarchy(O.Mesh1D.uniform(n, 2.0 * AR, True), O.Mesh1D.uniform(n, 2.0, True), p,
                    overlap=overlap, weight=weight)
    lev = H.top
    X, Y = lev.mx.coords(p), lev.my.coords(p)
    f = lev.mass(2 * np.pi**2 * np.sin(np.pi * X[None, :]) * np.sin(np.pi * Y[:, None]))
    u0 = SI.uniform_nodal(seed, f.shape, 0.0, 1.0)   # random initial guess in [0, 1]
    return H, u0, f


_T1 = rows("table1_rates.txt")
_T1_CASES = []
for r in _T1:
    p = int(r[0])
    for col, kappa in zip(r[1:7], ["a", 1, 3, 5, 7, "t"]):
        _T1_CASES.append((p, kappa, float(col)))


@pytest.mark.parametrize("p,kappa,want", [c for c in _T1_CASES if c[0] <= 16])
def test_table1_rates(p, kappa, want):
    H, u0, f = _periodic_case(p, kappa, 1)
    _, hist = H.mg_solve(u0, f)
    rb = O.rate(hist)
    assert _close(rb, want), (p, kappa, rb, want)
    assert _n10_close(O.n10(rb), math.ceil(10 / want))


@pytest.mark.slow
@pytest.mark.parametrize("p,kappa,want", [c for c in _T1_CASES if c[0] == 32])
def test_table1_rates_p32(p, kappa, want):
    H, u0, f = _periodic_case(p, kappa, 1)
    _, hist = H.mg_solve(u0, f)
    assert _close(O.rate(hist), want)


@pytest.mark.parametrize("row", rows("table3_problem_size.txt"), ids=lambda r: "p%s_n%s" % (r[0], r[1]))
def test_table3_rates(row):
    p, n, want, n10 = int(row[0]), int(row[1]), float(row[2]), int(row[3])
    if p * n > 256:
        pytest.skip("large case; covered by the slow marker run")
    H, u0, f = _periodic_case(p, 5, "ceil8", n=n)
    _, hist = H.mg_solve(u0, f)
    rb = O.rate(hist)
    assert _close(rb, want), (rb, want)
    assert _n10_close(O.n10(rb), n10)


@pytest.mark.parametrize("row", rows("table4_aspect_ratio.txt"), ids=lambda r: "p%s_AR%s" % (r[0], r[1]))
def test_table4_mg_and_mgcg(row):
    p, AR = int(row[0]), int(row[1])
    if p >= 16 and AR > 1 or p * AR > 32:
        pytest.skip("long case")
    H, u0, f = _periodic_case(p, 5, "ceil8", n=16, AR=AR)
    _, hist = H.mg_solve(u0, f, max_cycles=150)
    rb = O.rate(hist)
    assert _close(rb, float(row[2])), ("MG", rb, row)
    assert _n10_close(O.n10(rb), int(row[3]))
    _, it, hist = H.mgcg(u0, f, tol=1e-10, i_max=150)
    rb = O.rate(hist)
    assert _close(rb, float(row[4])), ("MGCG", rb, row)
    # the printed n_10 of (p=8, AR=2, MGCG) is 8 while its own r_bar = 1.03
    # gives ceil(10/1.03) = 10 by the definition of Sec. 4: the definition wins
    assert _n10_close(O.n10(rb), math.ceil(10 / float(row[4])))


def test_dirichlet_unit_square_p4_converges_like_the_periodic_case():
    """4x4 Dirichlet unit square, p = 4, n_o = 1, w_5: MG(1,0) and MGCG reach 1e-10
    at a rate in the range of the periodic results of Tables 1 and 4."""
    H = O.uniform_hierarchy(4, 4, 4, periodic=False, overlap=1, weight=5)
    lev = H.top
    X, Y = lev.mx.coords(4), lev.my.coords(4)
    ue = np.sin(np.pi * X[None, :]) * np.sin(np.pi * Y[:, None])
    f = lev.mass(2 * np.pi**2 * ue)
    _, hist = H.mg_solve(np.zeros_like(f), f)
    assert 0.8 <= O.rate(hist) <= 1.6
    u, it, hist = H.mgcg(np.zeros_like(f), f, tol=1e-10)
    assert hist[-1] <= 1e-10 * hist[0] and 5 <= it <= 12
    # discretisation error of p = 4 on 4x4 elements
    assert np.abs(u - ue).max() < 1e-4
