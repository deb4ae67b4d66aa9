"""Parity of the variable-diffusivity path (Sec. 4.3) on the GPU with the
oracle: B(nu) residuals, the 1/nu_bar_s local solves, the dense coarse
inverse of B_0(nu), stretched meshes (Dirichlet walls)."""
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
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda().reshape(-1)


def _host(t, shape):
    torch.cuda.synchronize()
    return t.cpu().numpy().reshape(shape)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _pair(nx, ny, p, nu, overlap=1, edges=None, **kw):
    if nu[0] == "contrast":
        fn = SI.nu_contrast(nu[1])
    else:
        fn = SI.nu_paper(nu[1], nu[2])
    S = P.Solver(nx=nx, ny=ny, p=p, overlap=overlap, weight=5, x_edges=edges, nu=nu, **kw)
    mx = O.Mesh1D.uniform(nx, 1.0, False) if edges is None else O.Mesh1D(np.asarray(edges), False)
    H = O.Hierarchy(mx, O.Mesh1D.uniform(ny, 1.0, False), p, overlap=overlap, weight=5, nu=fn)
    return S, H


CASES = [
    dict(nx=4, ny=3, p=8, nu=("contrast", 10.0)),
    dict(nx=5, ny=4, p=4, nu=("paper", 0.9, 0.2), overlap=2),
    dict(nx=6, ny=4, p=8, nu=("contrast", 100.0), edges=list(SI.geometric_edges(6, 0.02))),
    dict(nx=3, ny=3, p=16, nu=("contrast", 10.0), overlap=2),
]


def _ids(c):
    return "p%d_%s%s" % (c["p"], c["nu"][0], "_str" if "edges" in c else "")


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_variable_operator_matches_oracle(case):
    S, H = _pair(**case)
    lev = H.top
    u = SI.uniform_nodal(31, (lev.NY, lev.NX)) * lev.unknown
    out = torch.empty(lev.NY * lev.NX, dtype=torch.float64, device="cuda")
    S.apply(_dev(u), out)
    assert _rel(_host(out, u.shape), lev.apply(u)) < 1e-13


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_variable_sweep_and_vcycle_match_oracle(case):
    S, H = _pair(**case)
    lev = H.top
    u0 = SI.uniform_nodal(32, (lev.NY, lev.NX)) * lev.unknown
    f = lev.mass(SI.uniform_nodal(33, (lev.NY, lev.NX)))
    m = lev.p + 1 + 2 * lev.n_o
    tol = max(1e-12, np.finfo(np.float64).eps * m**3)
    ud = _dev(u0)
    S.smooth(ud, _dev(f), 1)
    assert _rel(_host(ud, u0.shape), lev.wschwarz(u0, f, 1)) < tol
    ud = _dev(u0)
    S.vcycle(ud, _dev(f))
    ns1, ns2 = H.steps(1, 0)
    assert _rel(_host(ud, u0.shape), H.vcycle(u0, f, ns1, ns2)) < tol


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_variable_pcg_matches_oracle(prec):
    S, H = _pair(nx=6, ny=5, p=8, nu=("contrast", 100.0), edges=list(SI.geometric_edges(6, 0.01)), precision=prec)
    lev = H.top
    f = lev.mass(SI.uniform_nodal(34, (lev.NY, lev.NX)))
    want, it_o, _ = H.mgcg(np.zeros_like(f), f, tol=1e-10, i_max=300)
    ud = torch.zeros(lev.NY * lev.NX, dtype=torch.float64, device="cuda")
    res, _ = S.pcg_solve(ud, _dev(f))
    assert res.status == P.SEM_OK
    got = _host(ud, f.shape)
    if prec == "fp64":
        assert res.iterations == it_o
        assert _rel(got, want) < 1e-12
    else:
        assert np.linalg.norm(f - lev.apply(got)) <= 1.1e-10 * np.linalg.norm(f)
        assert _rel(got, want) < 1e-9
