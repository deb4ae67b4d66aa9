"""Parity at the full sizes of the high-order and learned-weight workloads,
in the launch configuration the bench times (autotuned shapes; the solve is
replayed from its graph on the second call).

High order: 32 x 32 elements, p = 32 (1,050,625 nodes), n_o = 3. The FP64
MGCG of Alg. 4 must match the oracle's solve with identical iterations and a
relative solution error <= 1e-12. With the BF16 V-cycle the true residual of
the oracle's operator must be <= 1e-10 ||b||, and the solution within 1e-9 of
the oracle's.

Learned weights: 64 x 64 elements, p = 16, n_o = 2, x geometric 1:32, nu of
contrast 100.
- The B(nu) operator of Eq. (diffusion) is checked element by element.
- One Schwarz correction of Alg. 2 is checked with learned-family weights
  (R16), using seeded (s, kt) parameters given to both sides, in TF32 against
  the oracle's.
- The MGCG solve with the weights the trained network predicts reaches a true
  residual of the oracle's operator <= 1e-10 ||b||, and a solution within 1e-9
  of the plain FP64 method's (whose own true residual is checked the same way).
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
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).cuda()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


# ---- high order: 32 x 32, p = 32 -----------------------------------------------

C3 = dict(nx=32, ny=32, p=32, overlap=3, weight=5, tol=1e-10, i_max=100)


@pytest.fixture(scope="module")
def c3():
    H = O.uniform_hierarchy(32, 32, 32, periodic=False, overlap=3, weight=5)
    lev = H.top
    b = lev.mass(SI.uniform_nodal(1, (lev.NY, lev.NX), -1.0, 1.0))  # the bench's right side
    u, it, _ = H.mgcg(np.zeros_like(b), b, tol=1e-10)
    return H, b, u, it


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_high_order_mgcg_full_size(c3, prec):
    H, b, u_ref, it_ref = c3
    lev = H.top
    S = P.Solver(precision=prec, **C3)
    S.autotune()
    bd = _dev(b)
    for _ in range(2):  # launch by launch, then the captured graph
        ud = torch.zeros_like(bd)
        res, _ = S.pcg_solve(ud, bd)
        assert res.status == P.SEM_OK
        got = ud.cpu().numpy().reshape(b.shape)
        assert np.linalg.norm(b - lev.apply(got)) <= 1.1e-10 * np.linalg.norm(b)
        err = _rel(got, u_ref)
        if prec == "fp64":
            assert res.iterations == it_ref
            assert err <= 1e-12, err
        else:
            assert abs(res.iterations - it_ref) <= 2
            assert err <= 1e-9, err


# ---- learned weights: 64 x 64, p = 16, stretched 1:32, contrast 100 ------------

N4, P4, NO4, CONTRAST = 64, 16, 2, 100.0


def _c4_kw(**extra):
    return dict(nx=N4, ny=N4, p=P4, overlap=NO4, x_edges=SI.geometric_edges(N4, 1.0 / N4 / 32),
                nu=("contrast", CONTRAST), tol=1e-10, i_max=400, **extra)


def _c4_level(**kw):
    mx = O.Mesh1D(np.asarray(SI.geometric_edges(N4, 1.0 / N4 / 32)), False)
    return O.Level(mx, O.Mesh1D.uniform(N4, 1.0, False), P4, NO4, nu=SI.nu_contrast(CONTRAST), **kw)


def _seeded_learned():
    """(s, kt) per level and interface line: s in [0.25, 1], kt in [1, 7]."""
    L = int(np.log2(P4))
    out = []
    for seed in (41, 42):
        s = SI.uniform_nodal(seed, (L + 1, N4 + 1), 0.25, 1.0)
        kt = SI.uniform_nodal(seed + 10, (L + 1, N4 + 1), 1.0, 7.0)
        out.append(np.stack([s, kt], axis=-1))
    return out


def test_variable_operator_full_size():
    lev = _c4_level(weight=5)
    S = P.Solver(precision="fp64", weight=5, **_c4_kw())
    u = SI.uniform_nodal(5, (lev.NY, lev.NX)) * lev.unknown
    out = torch.empty(u.size, dtype=torch.float64, device="cuda")
    S.apply(_dev(u), out)
    want = lev.apply(u)
    assert _rel(out.cpu().numpy().reshape(want.shape), want) <= 1e-13


def test_learned_weight_correction_full_size():
    px, py = _seeded_learned()
    L = px.shape[0] - 1
    lev = _c4_level(weight="learned", learned=(px[L], py[L]))
    S = P.Solver(precision="tf32", weight="learned", learned_x=px.ravel(), learned_y=py.ravel(), **_c4_kw())
    b = lev.mass(SI.uniform_nodal(21, (lev.NY, lev.NX)))
    want = lev.wschwarz(np.zeros_like(b), b, 1)
    ud = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    S.smooth(ud, _dev(b), 1)
    assert _rel(ud.cpu().numpy().reshape(want.shape), want) <= 64 * 2.0**-11


def test_learned_solve_full_size():
    from paper_1512_02390_gb300 import learned as LW
    params, _ = LW.load_model()
    px, py = LW.predict(params, **_c4_kw())
    lev = _c4_level(weight=5)
    b = lev.mass(SI.uniform_nodal(1, (lev.NY, lev.NX), -1.0, 1.0))
    bd = _dev(b)
    S64 = P.Solver(precision="fp64", weight=5, **_c4_kw())
    u64 = torch.zeros_like(bd)
    r64, _ = S64.pcg_solve(u64, bd)
    assert r64.status == P.SEM_OK
    ref = u64.cpu().numpy().reshape(b.shape)
    assert np.linalg.norm(b - lev.apply(ref)) <= 1.1e-10 * np.linalg.norm(b)
    S = P.Solver(precision="tf32", weight="learned", learned_x=px.ravel(), learned_y=py.ravel(), **_c4_kw())
    S.autotune()
    for _ in range(2):
        ud = torch.zeros_like(bd)
        res, _ = S.pcg_solve(ud, bd)
        assert res.status == P.SEM_OK
        got = ud.cpu().numpy().reshape(b.shape)
        assert np.linalg.norm(b - lev.apply(got)) <= 1.1e-10 * np.linalg.norm(b)
        assert _rel(got, ref) <= 1e-9


@pytest.fixture(scope="module")
def c4_fp64_oracle():
    """The oracle's FP64 MGCG solve of the learned-weight workload with w_5."""
    H = O.Hierarchy(O.Mesh1D(np.asarray(SI.geometric_edges(N4, 1.0 / N4 / 32)), False),
                    O.Mesh1D.uniform(N4, 1.0, False), P4, overlap=NO4, weight=5, nu=SI.nu_contrast(CONTRAST))
    lev = H.top
    b = lev.mass(SI.uniform_nodal(1, (lev.NY, lev.NX), -1.0, 1.0))
    u, it, _ = H.mgcg(np.zeros_like(b), b, tol=1e-10, i_max=400)
    return lev, b, u, it


def test_fp64_variable_mgcg_full_size_matches_oracle(c4_fp64_oracle):
    """The plain FP64 method on the learned-weight workload (B(nu) operator,
    1/nu_bar local solves, dense coarse inverse): identical iterations and the
    solution within 1e-12 of the oracle's."""
    lev, b, want, it_o = c4_fp64_oracle
    S = P.Solver(precision="fp64", weight=5, **_c4_kw())
    S.autotune()
    bd = _dev(b)
    for _ in range(2):  # launch by launch, then the captured graph
        ud = torch.zeros_like(bd)
        res, _ = S.pcg_solve(ud, bd)
        assert res.status == P.SEM_OK and res.iterations == it_o
        got = ud.cpu().numpy().reshape(b.shape)
        assert _rel(got, want) <= 1e-12


def test_learned_handle_from_network_through_the_c_abi():
    """The weight network evaluated inside the library: sem_create with the
    network's parameters (features, forward kernel and (s, kt) tables in C),
    and sem_mlp_load on a w_5 handle, solve bitwise like weights predicted in
    Python and passed as learned_x / learned_y."""
    from paper_1512_02390_gb300 import learned as LW
    params, _ = LW.load_model()
    px, py = LW.predict(params, **_c4_kw())
    lev = _c4_level(weight=5)
    bd = _dev(lev.mass(SI.uniform_nodal(1, (lev.NY, lev.NX), -1.0, 1.0)))
    handles = [P.Solver(precision="tf32", weight="learned", learned_x=px.ravel(), learned_y=py.ravel(), **_c4_kw()),
               P.Solver(precision="tf32", weight="learned", mlp_params=params, **_c4_kw()),
               P.Solver(precision="tf32", weight=5, **_c4_kw())]
    handles[2].mlp_load(params)
    out = []
    for S in handles:
        ud = torch.zeros_like(bd)
        res, hist = S.pcg_solve(ud, bd, history_len=400)
        assert res.status == P.SEM_OK
        out.append((res.iterations, hist, ud.cpu().numpy()))
    for it, hist, u in out[1:]:
        assert it == out[0][0]
        assert np.array_equal(hist, out[0][1]) and np.array_equal(u, out[0][2])
