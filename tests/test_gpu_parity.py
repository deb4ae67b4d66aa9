"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every test feeds the same seeded inputs to both sides and compares element by
element.  FP64 bars: operator and one Schwarz sweep to 1e-13 relative, V-cycle
to 1e-12, MGCG solution to 1e-12 relative with identical iteration counts.
Mixed-precision bars: true residual <= 1e-10 ||b|| and solution error <= 1e-9
relative to the FP64 oracle solution.
"""
import numpy as np
import pytest

import sem_inputs as SI
from oracle import sem_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1512_02390_gb300")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load_library()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _pair(nx=4, ny=4, p=4, periodic=False, overlap=1, weight=5, edges=None, lx=1.0, ly=1.0, **kw):
    """(library solver, oracle hierarchy) for the same configuration."""
    S = P.Solver(nx=nx, ny=ny, p=p, periodic=periodic, overlap=overlap, weight=weight, x_edges=edges,
                 lx=lx, ly=ly, **kw)
    mx = O.Mesh1D.uniform(nx, lx, periodic) if edges is None else O.Mesh1D(np.asarray(edges), periodic)
    H = O.Hierarchy(mx, O.Mesh1D.uniform(ny, ly, periodic), p, overlap=overlap, weight=weight)
    return S, H


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _tol(H):
    """FP64 bar for results that pass through the FDM: four length-m
    contractions per output plus a residual summed in another order; their
    rounding is bounded by eps * m^3 (m = window size of the finest level)."""
    m = H.top.p + 1 + 2 * H.top.n_o
    return max(1e-12, np.finfo(np.float64).eps * m**3)


CASES = [
    dict(nx=4, ny=4, p=4),                                  # the 4x4, p = 4 Dirichlet unit square
    dict(nx=5, ny=3, p=4, overlap=2),                       # ragged tiles (5 is not a multiple of 8)
    dict(nx=3, ny=2, p=2),                                  # smallest order, two elements
    dict(nx=4, ny=6, p=8, periodic=True, overlap=3),        # periodic wrap
    dict(nx=6, ny=5, p=16, overlap=2, weight="a"),          # arithmetic mean, several tiles
    dict(nx=3, ny=3, p=32, overlap="ceil8", weight=7),      # highest order, ceil(p/8) overlap
    dict(nx=4, ny=3, p=8, overlap=1, weight="t", edges=[0.0, 0.1, 0.5, 0.55, 1.0]),  # stretched x
]


def _ids(c):
    return "_".join("%s%s" % (k, v if not isinstance(v, list) else "str") for k, v in c.items())


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_apply_matches_oracle(case):
    S, H = _pair(**case)
    lev = H.top
    u = SI.uniform_nodal(11, (lev.NY, lev.NX)) * lev.unknown
    Au = torch.empty(lev.NY * lev.NX, dtype=torch.float64, device="cuda")
    S.apply(_dev(u).reshape(-1), Au)
    got = _host(Au).reshape(lev.NY, lev.NX)
    want = lev.apply(u)
    assert _rel(got, want) < 1e-13


@pytest.mark.parametrize("case", CASES[:4], ids=_ids)
def test_mass_and_coords_match_oracle(case):
    S, H = _pair(**case)
    lev = H.top
    x, y = S.coords()
    np.testing.assert_allclose(x, lev.mx.coords(lev.p), atol=1e-14)
    np.testing.assert_allclose(y, lev.my.coords(lev.p), atol=1e-14)
    fn = SI.uniform_nodal(3, (lev.NY, lev.NX))
    b = torch.empty(lev.NY * lev.NX, dtype=torch.float64, device="cuda")
    S.mass(_dev(fn).reshape(-1), b)
    assert _rel(_host(b).reshape(lev.NY, lev.NX), lev.mass(fn)) < 1e-13


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_schwarz_sweep_matches_oracle(case):
    """Alg. 2, two sweeps from a random u: gather, FDM, weights, scatter-add."""
    S, H = _pair(**case)
    lev = H.top
    u0 = SI.uniform_nodal(5, (lev.NY, lev.NX)) * lev.unknown
    f = lev.mass(SI.uniform_nodal(6, (lev.NY, lev.NX)))
    ud = _dev(u0).reshape(-1)
    S.smooth(ud, _dev(f).reshape(-1), 2)
    want = lev.wschwarz(u0, f, 2)
    assert _rel(_host(ud).reshape(lev.NY, lev.NX), want) < _tol(H)


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_vcycle_matches_oracle(case):
    """Alg. 3 MG(1,0) from a random u."""
    S, H = _pair(**case)
    lev = H.top
    u0 = SI.uniform_nodal(7, (lev.NY, lev.NX)) * lev.unknown
    f = lev.mass(SI.uniform_nodal(8, (lev.NY, lev.NX)))
    ud = _dev(u0).reshape(-1)
    S.vcycle(ud, _dev(f).reshape(-1))
    ns1, ns2 = H.steps(1, 0)
    want = H.vcycle(u0, f, ns1, ns2)
    got = _host(ud).reshape(lev.NY, lev.NX)
    if H.mx.periodic:  # periodic solutions are defined up to a constant
        got, want = got - got.mean(), want - want.mean()
    assert _rel(got, want) < _tol(H)


@pytest.mark.parametrize("prec,u_in", [("fp32", 2.0**-24), ("tf32", 2.0**-11), ("bf16", 2.0**-8)])
@pytest.mark.parametrize("case", [dict(nx=5, ny=4, p=16, overlap=2), dict(nx=4, ny=4, p=8, periodic=True, overlap=1),
                                  dict(nx=3, ny=3, p=32, overlap=4), dict(nx=6, ny=3, p=4, overlap=1)], ids=_ids)
def test_reduced_precision_sweep_matches_oracle(case, prec, u_in):
    """One Schwarz correction from u = 0 in FP32 SIMT or on the tensor cores
    (TF32 / BF16 operands, FP32 accumulation).  Four contractions each round
    their operands once (unit roundoff u_in); with orthonormal-like S the
    error stays within 64 u_in of max|correction|."""
    S, H = _pair(precision=prec, **case)
    lev = H.top
    f = lev.mass(SI.uniform_nodal(12, (lev.NY, lev.NX)))
    ud = torch.zeros(lev.NY * lev.NX, dtype=torch.float64, device="cuda")
    S.smooth(ud, _dev(f).reshape(-1), 1)
    want = lev.wschwarz(np.zeros_like(f), f, 1)
    err = _rel(_host(ud).reshape(lev.NY, lev.NX), want)
    assert err < 64 * u_in, err


def test_vcycle_with_post_smoothing_and_variable_cycle():
    S, H = _pair(nx=4, ny=4, p=8, overlap=2, ns1=1, ns2=1, variable_cycle=True)
    lev = H.top
    u0 = SI.uniform_nodal(9, (lev.NY, lev.NX)) * lev.unknown
    f = lev.mass(SI.uniform_nodal(10, (lev.NY, lev.NX)))
    ud = _dev(u0).reshape(-1)
    S.vcycle(ud, _dev(f).reshape(-1))
    ns1, ns2 = H.steps(1, 1, variable=True)
    assert _rel(_host(ud).reshape(lev.NY, lev.NX), H.vcycle(u0, f, ns1, ns2)) < 1e-12


def _manufactured(lev):
    X, Y = lev.mx.coords(lev.p), lev.my.coords(lev.p)
    return 2 * np.pi**2 * np.sin(np.pi * X[None, :]) * np.sin(np.pi * Y[:, None])


def test_pcg_unit_square_p4_matches_oracle():
    """4x4 Dirichlet unit square, p = 4, n_o = 1, w_5, RHS of u = sin(pi x) sin(pi y)."""
    S, H = _pair(nx=4, ny=4, p=4)
    lev = H.top
    f = lev.mass(_manufactured(lev))
    want, it_o, hist_o = H.mgcg(np.zeros_like(f), f, tol=1e-10)
    ud = torch.zeros(lev.NY * lev.NX, dtype=torch.float64, device="cuda")
    res, hist = S.pcg_solve(ud, _dev(f).reshape(-1), history_len=64)
    assert res.status == P.SEM_OK
    assert res.iterations == it_o
    np.testing.assert_allclose(hist, hist_o, rtol=1e-9)
    assert _rel(_host(ud).reshape(lev.NY, lev.NX), want) < 1e-12


@pytest.mark.parametrize("case", [dict(nx=8, ny=8, p=16, overlap=2), dict(nx=6, ny=4, p=8, periodic=True, overlap=1),
                                  dict(nx=5, ny=7, p=32, overlap=3)], ids=_ids)
def test_pcg_matches_oracle(case):
    S, H = _pair(**case)
    lev = H.top
    f = lev.mass(SI.uniform_nodal(1, (lev.NY, lev.NX)))
    want, it_o, _ = H.mgcg(np.zeros_like(f), f, tol=1e-10)
    fd = _dev(f).reshape(-1)
    ud = torch.zeros(lev.NY * lev.NX, dtype=torch.float64, device="cuda")
    res, h1 = S.pcg_solve(ud, fd, history_len=200)  # first solve: launch by launch
    assert res.status == P.SEM_OK and res.iterations == it_o
    got = _host(ud).reshape(lev.NY, lev.NX)
    # second solve replays the captured graph (WHILE node): bitwise identical
    ud2 = torch.zeros_like(ud)
    res2, h2 = S.pcg_solve(ud2, fd, history_len=200)
    assert res2.iterations == res.iterations and res2.status == res.status
    assert np.array_equal(h1, h2) and np.array_equal(_host(ud2).reshape(lev.NY, lev.NX), got)
    if H.mx.periodic:
        got, want = got - got.mean(), want - want.mean()
    assert _rel(got, want) < 1e-12


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_mixed_precision_reaches_fp64_accuracy(prec):
    """Mixed V-cycle inside the FP64 MGCG: true residual <= 1e-10 ||b||, error <= 1e-9."""
    S, H = _pair(nx=8, ny=8, p=16, overlap=2, precision=prec)
    lev = H.top
    f = lev.mass(SI.uniform_nodal(2, (lev.NY, lev.NX)))
    want, it_o, _ = H.mgcg(np.zeros_like(f), f, tol=1e-12)
    ud = torch.zeros(lev.NY * lev.NX, dtype=torch.float64, device="cuda")
    res, _ = S.pcg_solve(ud, _dev(f).reshape(-1))
    assert res.status == P.SEM_OK
    got = _host(ud).reshape(lev.NY, lev.NX)
    true_res = np.linalg.norm(f - lev.apply(got))
    assert true_res <= 1e-10 * np.linalg.norm(f) * 1.5
    assert _rel(got, want) < 1e-9


def test_zero_rhs_returns_immediately():
    S, H = _pair()
    n = H.top.NY * H.top.NX
    for _ in range(2):  # launch by launch, then the captured graph
        ud = torch.zeros(n, dtype=torch.float64, device="cuda")
        res, _ = S.pcg_solve(ud, torch.zeros(n, dtype=torch.float64, device="cuda"))
        assert res.status == P.SEM_OK and res.iterations == 0
        assert float(ud.abs().max()) == 0.0


def test_nan_rhs_reports_breakdown_and_device_stays_usable():
    S, H = _pair()
    lev = H.top
    n = lev.NY * lev.NX
    f = np.ones((lev.NY, lev.NX))
    f[2, 2] = np.nan
    for _ in range(2):
        ud = torch.zeros(n, dtype=torch.float64, device="cuda")
        res, _ = S.pcg_solve(ud, _dev(f).reshape(-1))
        assert res.status == P.SEM_BREAKDOWN
    # the context still works
    Au = torch.empty(n, dtype=torch.float64, device="cuda")
    S.apply(torch.ones(n, dtype=torch.float64, device="cuda"), Au)
    assert np.isfinite(_host(Au)).all()


def test_iteration_limit_reports_not_converged():
    S, H = _pair(i_max=2)
    lev = H.top
    f = lev.mass(_manufactured(lev))
    for _ in range(2):
        ud = torch.zeros(lev.NY * lev.NX, dtype=torch.float64, device="cuda")
        res, _ = S.pcg_solve(ud, _dev(f).reshape(-1))
        assert res.status == P.SEM_NOT_CONVERGED and res.iterations == 2


def test_mg_solve_rate_matches_oracle():
    """Stand-alone MG(1,0) on the periodic 8x8 [0,2]^2 case of Table 1 (p = 8, w_5)."""
    S, H = _pair(nx=8, ny=8, p=8, periodic=True, lx=2.0, ly=2.0, overlap=1)
    lev = H.top
    X, Y = lev.mx.coords(8), lev.my.coords(8)
    f = lev.mass(2 * np.pi**2 * np.sin(np.pi * X[None, :]) * np.sin(np.pi * Y[:, None]))
    u0 = SI.uniform_nodal(1, f.shape, 0.0, 1.0)
    _, hist_o = H.mg_solve(u0.copy(), f)
    ud = _dev(u0).reshape(-1)
    res, hist = S.mg_solve(ud, _dev(f).reshape(-1), history_len=64)
    assert res.iterations == len(hist_o) - 1
    # rounding of the residual itself is ~eps * ||A|| ||u||, so compare on the
    # scale of the initial residual
    np.testing.assert_allclose(hist, hist_o, rtol=1e-8, atol=1e-13 * hist_o[0])
    assert abs(res.rbar - 1.29) < 0.05  # Table 1, p = 8, w_5


@pytest.mark.parametrize("case", [dict(nx=4, ny=4, p=4), dict(nx=4, ny=6, p=8, periodic=True, overlap=3),
                                  dict(nx=12, ny=10, p=4, overlap=1), dict(nx=9, ny=9, p=8, periodic=True, overlap=1),
                                  dict(nx=65, ny=20, p=2, overlap=1), dict(nx=66, ny=12, p=2, overlap=1)], ids=_ids)
@pytest.mark.parametrize("eo", [0, 1])
def test_fp32_vcycle_matches_oracle(case, eo):
    """Alg. 3 in the FP32 V-cycle (SIMT sweeps; the clustered FP32 coarse solve
    where the coarse grid has at most 64 x 64 unknowns, the four-launch
    product beyond; level residuals in the plain or the even-odd form): the
    correction u_new - u_old agrees with the FP64 oracle's to FP32 accuracy
    (1e-5 of its maximum)."""
    S, H = _pair(precision="fp32", **case)
    for l in range(1, S.levels + 1):
        S.set_tune(l, 0, 1, 0, eo)
    lev = H.top
    u0 = SI.uniform_nodal(7, (lev.NY, lev.NX)) * lev.unknown
    f = lev.mass(SI.uniform_nodal(8, (lev.NY, lev.NX)))
    ud = _dev(u0).reshape(-1)
    S.vcycle(ud, _dev(f).reshape(-1))
    ns1, ns2 = H.steps(1, 0)
    want = H.vcycle(u0, f, ns1, ns2) - u0
    got = _host(ud).reshape(lev.NY, lev.NX) - u0
    if H.mx.periodic:
        got, want = got - got.mean(), want - want.mean()
    assert _rel(got, want) < 1e-5
