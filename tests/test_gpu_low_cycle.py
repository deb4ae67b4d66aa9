"""The persistent low-level cycle (levels p_l <= 8 and the coarse solve in one
cooperative kernel) against the per-level launches and against the FP64
oracle's V-cycle (Alg. 3), and inside MGCG (Alg. 4): the V-cycle corrections
agree to the rounding of the reduced-precision sweeps; the solve reaches 1e-10
and the FP64 solution; the graph replays the first solve bitwise."""
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


CASES = [dict(nx=16, ny=16, p=16, overlap=2, precision="tf32"),
         dict(nx=12, ny=10, p=8, overlap=1, precision="bf16"),
         dict(nx=8, ny=8, p=4, overlap=1, precision="tf32", periodic=True),
         dict(nx=20, ny=12, p=32, overlap=2, precision="tf32"),
         dict(nx=10, ny=6, p=16, overlap=3, precision="bf16")]


def _ids(c):
    return "_".join("%s%s" % (k, v) for k, v in c.items())


def _vcycle(S, u0, f):
    ud = torch.from_numpy(np.ascontiguousarray(u0).reshape(-1)).cuda()
    S.vcycle(ud, torch.from_numpy(np.ascontiguousarray(f).reshape(-1)).cuda())
    torch.cuda.synchronize()
    return ud.cpu().numpy().reshape(u0.shape) - u0


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_low_cycle_matches_launches_and_oracle(case):
    S = P.Solver(**case)
    assert S.low_cycle() == (True, False)
    S.set_low_cycle(True)
    assert S.low_cycle() == (True, True)
    periodic = case.get("periodic", False)
    H = O.Hierarchy(O.Mesh1D.uniform(case["nx"], 1.0, periodic), O.Mesh1D.uniform(case["ny"], 1.0, periodic),
                    case["p"], overlap=case["overlap"], weight=5)
    lev = H.top
    u0 = SI.uniform_nodal(7, (lev.NY, lev.NX)) * lev.unknown
    f = lev.mass(SI.uniform_nodal(8, (lev.NY, lev.NX)))
    got_on = _vcycle(S, u0, f)
    S.set_low_cycle(False)
    got_off = _vcycle(S, u0, f)
    ns1, ns2 = H.steps(1, 0)
    want = H.vcycle(u0, f, ns1, ns2) - u0
    if periodic:
        got_on, got_off, want = got_on - got_on.mean(), got_off - got_off.mean(), want - want.mean()
    scale = np.abs(want).max()
    u_in = 2.0**-11 if case["precision"] == "tf32" else 2.0**-8
    # off: the low levels default to the tcgen05 sweep, which rounds its
    # reduced-precision products in another order than the mma.sync one
    assert np.abs(got_on - got_off).max() <= 16 * u_in * scale
    assert np.abs(got_on - want).max() <= 64 * u_in * scale


@pytest.mark.parametrize("case", CASES[:3], ids=_ids)
def test_low_cycle_inside_mgcg(case):
    S = P.Solver(**case)
    S.set_low_cycle(True)
    S64 = P.Solver(**dict(case, precision="fp64"))
    fn = torch.from_numpy(SI.uniform_nodal(9, S.shape).ravel()).cuda()
    b = torch.empty_like(fn)
    S64.mass(fn, b)
    u64 = torch.zeros_like(b)
    S64.pcg_solve(u64, b)
    sols = []
    for _ in range(2):  # launch by launch, then the captured graph
        u = torch.zeros_like(b)
        r, _ = S.pcg_solve(u, b)
        assert r.status == P.SEM_OK and r.res <= 1e-10 * r.res0
        sols.append(u.cpu().numpy())
    assert np.array_equal(sols[0], sols[1])
    a, c = sols[0], u64.cpu().numpy()
    if case.get("periodic"):
        a, c = a - a.mean(), c - c.mean()
    assert np.abs(a - c).max() <= 1e-9 * np.abs(c).max()


def test_low_cycle_not_offered_where_it_does_not_apply():
    for kw in (dict(precision="fp64"), dict(precision="fp32"), dict(precision="tf32", nu=("contrast", 10.0)),
               dict(precision="tf32", ns2=1)):
        S = P.Solver(nx=8, ny=8, p=8, overlap=1, **kw)
        assert S.low_cycle() == (False, False), kw
        with pytest.raises(P.SemError):
            S.set_low_cycle(True)
