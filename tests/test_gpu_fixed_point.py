"""The FP64 operator of Eq. (system matrix) evaluated exactly in integer
arithmetic (fixed-point operands, exact 64-bit sums, one final rounding)
against the oracle's FP64 operator and the library's FP64-pipe evaluation.

Error model.  The FP64 evaluation of (A u)_i errs by about eps (|A| |u|)_i.
The fixed-point one rounds each staged value to about eps of its tile's
largest |u|, holds each element matrix exactly (75-bit fixed point), then sums
exactly, so it errs by at most about eps (|A| 1)_i max|u| plus its one final
rounding.
The bar below, 16 eps ((|A| |u|)_i + (|A| 1)_i max|u|), holds both with room;
|A| is bounded by M_y (x) |L_x| + |L_y| (x) M_x from the oracle's assembled 1D
matrices.  Inputs: uniform random, and random with magnitudes spread over 30
decades (a tile then holds values far below its scale), on uniform, ragged,
periodic and stretched meshes at every order the operator takes."""
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


EPS = np.finfo(np.float64).eps

CASES = [
    dict(nx=4, ny=4, p=4),
    dict(nx=5, ny=3, p=4, overlap=2),                         # ragged tiles (4 elements per tile)
    dict(nx=3, ny=5, p=4, periodic=True),                     # periodic tiles wider than the mesh
    dict(nx=6, ny=3, p=4, periodic=True, overlap=2),
    dict(nx=4, ny=6, p=8, periodic=True, overlap=3),
    dict(nx=7, ny=5, p=16, overlap=2),                        # ragged tiles (2 elements per tile)
    dict(nx=3, ny=3, p=32),
    dict(nx=3, ny=4, p=32, periodic=True),
    dict(nx=4, ny=3, p=8, edges=[0.0, 0.1, 0.5, 0.55, 1.0]),  # stretched x
    dict(nx=5, ny=4, p=8, edges=[0.0, 0.25, 0.5, 0.625, 0.75, 1.0]),  # two element widths, interleaved (shared tables)
    dict(nx=5, ny=3, p=32, edges=[0.0, 0.25, 0.375, 0.5, 0.75, 1.0], periodic=True),
    dict(nx=6, ny=4, p=16, edges=list(SI.geometric_edges(6, 1.0 / 48))),
]


def _ids(c):
    return "_".join("%s%s" % (k, v if not isinstance(v, list) else "str") for k, v in c.items())


def _pair(nx, ny, p, periodic=False, overlap=1, edges=None, **kw):
    S = P.Solver(nx=nx, ny=ny, p=p, periodic=periodic, overlap=overlap, weight=5, x_edges=edges, **kw)
    mx = O.Mesh1D.uniform(nx, 1.0, periodic) if edges is None else O.Mesh1D(np.asarray(edges), periodic)
    H = O.Hierarchy(mx, O.Mesh1D.uniform(ny, 1.0, periodic), p, overlap=overlap, weight=5)
    return S, H.top


def _apply(S, u):
    ud = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float64).reshape(-1)).cuda()
    out = torch.empty_like(ud)
    S.apply(ud, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(u.shape)


def _abs_bound(lev, a):
    """(M_y (x) |L_x| + |L_y| (x) M_x) a for a >= 0, on the unknowns."""
    b = lev.My_glob[:, None] * (a @ np.abs(lev.Lx_glob).T) + lev.Mx_glob[None, :] * (np.abs(lev.Ly_glob) @ a)
    return np.where(lev.unknown, b, 0.0)


def _inputs(lev, kind):
    u = SI.uniform_nodal(17, (lev.NY, lev.NX))
    if kind == "spread":
        u = u * 10.0 ** (-30.0 * SI.uniform_nodal(18, (lev.NY, lev.NX)) ** 2)
    return np.where(lev.unknown, u, 0.0)


@pytest.mark.parametrize("kind", ["uniform", "spread"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_fixed_point_operator_within_fp64_bound(case, kind):
    S, lev = _pair(**case)
    assert S.fixed_point_operator() == (True, True)
    u = _inputs(lev, kind)
    want = lev.apply(u)
    bar = 16 * EPS * (_abs_bound(lev, np.abs(u)) + _abs_bound(lev, np.ones_like(u)) * np.abs(u).max())
    got = _apply(S, u)
    assert np.all(np.abs(got - want) <= bar)
    S.set_fixed_point_operator(False)  # the FP64-pipe evaluation meets the same bar
    got64 = _apply(S, u)
    assert np.all(np.abs(got64 - want) <= bar)
    S.set_fixed_point_operator(True)
    assert np.array_equal(_apply(S, u), got)  # deterministic
    S.close()


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_solves_with_fixed_point_operator_match_oracle(prec):
    """MGCG (Alg. 4) with the integer operator: FP64 mode reaches the oracle's
    solution to 1e-12 in the same number of iterations; the TF32 V-cycle meets
    the mixed bars (true residual 1.1e-10 ||b||, error 1e-9)."""
    S, lev = _pair(nx=12, ny=10, p=16, overlap=2, precision=prec, tol=1e-10, i_max=100)
    H = O.uniform_hierarchy(12, 10, 16, periodic=False, overlap=2, weight=5)
    b = lev.mass(SI.uniform_nodal(5, (lev.NY, lev.NX)))
    want, it_o, _ = H.mgcg(np.zeros_like(b), b, tol=1e-10)
    bd = torch.from_numpy(np.ascontiguousarray(b).reshape(-1)).cuda()
    for _ in range(2):  # host loop, then the captured graph
        u = torch.zeros_like(bd)
        r, _ = S.pcg_solve(u, bd)
        assert r.status == P.SEM_OK
        got = u.cpu().numpy().reshape(b.shape)
        rel = np.abs(got - want).max() / np.abs(want).max()
        if prec == "fp64":
            assert r.iterations == it_o
            assert rel <= 1e-12, rel
        else:
            assert np.linalg.norm(b - lev.apply(got)) <= 1.1e-10 * np.linalg.norm(b)
            assert rel <= 1e-9, rel
    S.close()


def test_non_finite_input_gives_nan_in_its_tile_only():
    S, lev = _pair(nx=8, ny=8, p=16, overlap=2)
    u = _inputs(lev, "uniform")
    u[5, 7] = np.inf
    got = _apply(S, u)
    assert np.isnan(got[5, 7])
    # tiles of 2 x 2 elements (32 x 32 nodes): the far corner tile is untouched
    assert np.all(np.isfinite(got[64:, 64:]))
    S.close()


def test_availability():
    S = P.Solver(nx=4, ny=4, p=2, overlap=1)
    assert S.fixed_point_operator() == (False, False)
    with pytest.raises(P.SemError):
        S.set_fixed_point_operator(True)
    S.close()
    S = P.Solver(nx=4, ny=4, p=8, overlap=1, nu=("contrast", 10.0))
    assert S.fixed_point_operator() == (False, False)
    S.close()
