"""Parity at the full size of the throughput workload (64 x 64 elements,
p = 16, n_o = 2: 1,046,529 unknowns) in the launch configuration the bench
times (autotuned launch shapes, the solve replayed from its graph): the FP64
operator of Eq. (system matrix) element by element, one FP64 and one TF32
(tcgen05) Schwarz correction of Alg. 2, and the MGCG solve of Alg. 4 in FP64
(identical iterations, 1e-12) and with the TF32 V-cycle (true residual of the
oracle's own operator <= 1e-10 ||b||, solution within 1e-9 of the oracle's)."""
import numpy as np
import pytest

import sem_inputs as SI
from oracle import sem_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1512_02390_gb300")

KW = dict(nx=64, ny=64, p=16, overlap=2, weight=5, tol=1e-10, i_max=100)


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load_library()


@pytest.fixture(scope="module")
def oracle():
    H = O.uniform_hierarchy(64, 64, 16, periodic=False, overlap=2, weight=5)
    lev = H.top
    b = lev.mass(SI.uniform_nodal(1, (lev.NY, lev.NX), -1.0, 1.0))  # the bench's right side
    u, it, hist = H.mgcg(np.zeros_like(b), b, tol=1e-10)
    return H, b, u, it


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).cuda()


def test_operator_full_size(oracle):
    H, b, _, _ = oracle
    lev = H.top
    u = SI.uniform_nodal(5, (lev.NY, lev.NX)) * lev.unknown
    S = P.Solver(precision="fp64", **KW)
    out = torch.empty(u.size, dtype=torch.float64, device="cuda")
    S.apply(_dev(u), out)
    want = lev.apply(u)
    got = out.cpu().numpy().reshape(want.shape)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("prec,bar", [("fp64", 3e-12), ("tf32", 64 * 2.0**-11)])
def test_schwarz_correction_full_size(oracle, prec, bar):
    H, b, _, _ = oracle
    lev = H.top
    S = P.Solver(precision=prec, **KW)
    if prec == "tf32":
        assert S.get_tune(S.levels)["tc"] == 1  # the tcgen05 sweep on the finest level
    ud = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    S.smooth(ud, _dev(b), 1)
    want = lev.wschwarz(np.zeros_like(b), b, 1)
    got = ud.cpu().numpy().reshape(want.shape)
    assert np.abs(got - want).max() <= bar * np.abs(want).max()


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_mgcg_full_size(oracle, prec):
    H, b, u_ref, it_ref = oracle
    lev = H.top
    S = P.Solver(precision=prec, **KW)
    S.autotune()
    bd = _dev(b)
    for _ in range(2):  # launch by launch, then the captured graph
        ud = torch.zeros_like(bd)
        res, _ = S.pcg_solve(ud, bd)
        assert res.status == P.SEM_OK
        got = ud.cpu().numpy().reshape(b.shape)
        true_res = np.linalg.norm(b - lev.apply(got))
        assert true_res <= 1.1e-10 * np.linalg.norm(b)  # the recursive residual met 1e-10 ||r_0||
        err = np.abs(got - u_ref).max() / np.abs(u_ref).max()
        if prec == "fp64":
            assert res.iterations == it_ref
            assert err <= 1e-12
        else:
            assert abs(res.iterations - it_ref) <= 1
            assert err <= 1e-9
