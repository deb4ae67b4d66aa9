"""Parity of the three-dimensional extension (sem3_* entry points) with the
3D FP64 oracle, element by element on the same seeded inputs.  FP64 bars: the
operator and the mass to 1e-13, Schwarz sweeps and V-cycles to eps m^3, the
MGCG solution to 1e-12 with identical iteration counts.  FP32 V-cycle: the
correction to 1e-5 of its maximum; MGCG reaches the true residual
1e-10 ||b|| and 1e-9 of the FP64 oracle solution."""
import numpy as np
import pytest

import sem_inputs as SI
from oracle import sem3d_oracle as O3
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
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).cuda()


def _host(t, shape):
    torch.cuda.synchronize()
    return t.cpu().numpy().reshape(shape)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _demean(a):
    return a - a.mean()


def _pair(nx=3, ny=3, nz=3, p=4, periodic=False, overlap=1, weight=5, lx=1.0, ly=1.0, lz=1.0, **kw):
    S = P.Solver3(nx=nx, ny=ny, nz=nz, p=p, periodic=periodic, overlap=overlap, weight=weight, lx=lx, ly=ly, lz=lz,
                  **kw)
    H = O3.Hierarchy3(O.Mesh1D.uniform(nx, lx, periodic), O.Mesh1D.uniform(ny, ly, periodic),
                      O.Mesh1D.uniform(nz, lz, periodic), p, overlap=overlap, weight=weight)
    return S, H


def _tol(H):
    m = H.top.p + 1 + 2 * H.top.n_o
    return max(1e-12, np.finfo(np.float64).eps * m**3)


CASES = [
    dict(nx=3, ny=3, nz=3, p=4),                                     # Dirichlet cube
    dict(nx=4, ny=3, nz=2, p=4, overlap=2, lx=2.0),                  # ragged, anisotropic elements
    dict(nx=2, ny=2, nz=3, p=2),                                     # smallest order
    dict(nx=3, ny=4, nz=3, p=8, periodic=True),                      # periodic wrap
    dict(nx=2, ny=3, nz=2, p=16, overlap=2),                         # m = 21
    dict(nx=3, ny=3, nz=3, p=8, overlap=1, weight="a"),              # arithmetic mean
]


def _ids(c):
    return "_".join("%s%s" % (k, v) for k, v in c.items())


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_3d_operator_and_mass_match_oracle(case):
    S, H = _pair(**case)
    lev = H.top
    x, y, z = S.coords()
    np.testing.assert_allclose(x, lev.dx.mesh.coords(lev.p), atol=1e-14)
    np.testing.assert_allclose(z, lev.dz.mesh.coords(lev.p), atol=1e-14)
    u = SI.uniform_nodal(11, lev.shape) * lev.unknown
    out = torch.empty(u.size, dtype=torch.float64, device="cuda")
    S.apply(_dev(u), out)
    assert _rel(_host(out, u.shape), lev.apply(u)) < 1e-13
    fn = SI.uniform_nodal(12, lev.shape)
    S.mass(_dev(fn), out)
    assert _rel(_host(out, u.shape), lev.mass(fn)) < 1e-13


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_3d_schwarz_sweeps_match_oracle(case):
    """Alg. 2 in 3D, two sweeps from a random u: gather of the m^3 window,
    fast diagonalisation with three contractions per side, weights, scatter."""
    S, H = _pair(**case)
    lev = H.top
    u0 = SI.uniform_nodal(5, lev.shape) * lev.unknown
    f = lev.mass(SI.uniform_nodal(6, lev.shape))
    ud = _dev(u0)
    S.smooth(ud, _dev(f), 2)
    assert _rel(_host(ud, u0.shape), lev.wschwarz(u0, f, 2)) < _tol(H)


@pytest.mark.parametrize("case", CASES, ids=_ids)
@pytest.mark.parametrize("ns", [(1, 0), (1, 1)])
def test_3d_vcycle_matches_oracle(case, ns):
    S, H = _pair(ns1=ns[0], ns2=ns[1], **case)
    lev = H.top
    u0 = SI.uniform_nodal(7, lev.shape) * lev.unknown
    f = lev.mass(SI.uniform_nodal(8, lev.shape))
    ud = _dev(u0)
    S.vcycle(ud, _dev(f))
    got, want = _host(ud, u0.shape), H.vcycle(u0, f, *ns)
    if case.get("periodic"):
        got, want = _demean(got), _demean(want)
    assert _rel(got, want) < _tol(H)


@pytest.mark.parametrize("case", [dict(nx=4, ny=4, nz=4, p=8, overlap=1), dict(nx=3, ny=4, nz=3, p=8, periodic=True),
                                  dict(nx=3, ny=3, nz=2, p=16, overlap=2), dict(nx=8, ny=8, nz=8, p=4, overlap=1)],
                         ids=_ids)
def test_3d_pcg_matches_oracle(case):
    """Alg. 4 in 3D: identical iterations, the oracle's residual history and
    the solution within 1e-12."""
    S, H = _pair(**case)
    lev = H.top
    f = lev.mass(SI.uniform_nodal(1, lev.shape))
    want, it_o, hist_o = H.mgcg(np.zeros_like(f), f, tol=1e-10)
    ud = torch.zeros(f.size, dtype=torch.float64, device="cuda")
    res, hist = S.pcg_solve(ud, _dev(f), history_len=200)
    assert res.status == P.SEM_OK and res.iterations == it_o
    np.testing.assert_allclose(hist, hist_o, rtol=1e-8, atol=1e-13 * hist_o[0])
    got = _host(ud, f.shape)
    if case.get("periodic"):
        got, want = _demean(got), _demean(want)
    assert _rel(got, want) < 1e-12


@pytest.mark.parametrize("case", [dict(nx=4, ny=4, nz=4, p=8, overlap=1), dict(nx=3, ny=4, nz=3, p=8, periodic=True)],
                         ids=_ids)
def test_3d_fp32_vcycle_inside_fp64_mgcg(case):
    S, H = _pair(precision="fp32", **case)
    lev = H.top
    u0 = SI.uniform_nodal(7, lev.shape) * lev.unknown
    f = lev.mass(SI.uniform_nodal(8, lev.shape))
    ud = _dev(u0)
    S.vcycle(ud, _dev(f))
    got, want = _host(ud, u0.shape) - u0, H.vcycle(u0, f) - u0
    if case.get("periodic"):
        got, want = _demean(got), _demean(want)
    assert _rel(got, want) < 1e-5
    sol, _, _ = H.mgcg(np.zeros_like(f), f, tol=1e-12)
    ud = torch.zeros(f.size, dtype=torch.float64, device="cuda")
    res, _ = S.pcg_solve(ud, _dev(f))
    assert res.status == P.SEM_OK
    got = _host(ud, f.shape)
    assert np.linalg.norm(f - lev.apply(got)) <= 1.1e-10 * np.linalg.norm(f)
    if case.get("periodic"):
        got, sol = _demean(got), _demean(sol)
    assert _rel(got, sol) < 1e-9


def test_3d_rejects_unsupported_configurations():
    for kw in (dict(p=32), dict(precision="tf32"), dict(p=16, overlap=6)):
        with pytest.raises(P.SemError) as ei:
            P.Solver3(**kw)
        assert ei.value.status == P.SEM_BAD_ARG
