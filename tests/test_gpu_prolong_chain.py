"""The up-leg of the V-cycle (Alg. 3 without post-smoothing) in one launch
against the level-by-level prolongations: the same solve with the fused launch
on and off must give the same iterations, the same residual history and the
same solution, bit for bit (every node is interpolated with the same
arithmetic in the same order; a node shared by two tiles is interpolated
through the exact 0 / 1 end rows of J).  Covers every finest order the
launch takes (p = 4, 8, 16, 32), FP64, FP32 and TF32 V-cycles, periodic wrap,
stretched meshes, variable diffusivity, partial tiles and the fused MGCG dot
products.  Solutions against the oracle are checked by the parity tests,
which run with the launch on (the default)."""
import numpy as np
import pytest

import sem_inputs as SI

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1512_02390_gb300")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load_library()


CASES = [
    dict(nx=16, ny=16, p=16, overlap=2, precision="tf32"),
    dict(nx=12, ny=10, p=16, overlap=2, precision="fp64"),
    dict(nx=7, ny=9, p=16, overlap=1, precision="fp32"),                     # partial tiles (TE = 2)
    dict(nx=6, ny=5, p=32, overlap=2, precision="tf32"),                     # L = 5, TE = 1
    dict(nx=5, ny=6, p=32, overlap=1, precision="fp64", periodic=True),
    dict(nx=10, ny=12, p=8, overlap=1, precision="tf32", periodic=True),
    dict(nx=9, ny=7, p=4, overlap=1, precision="fp64"),                      # TE = 4, partial tiles
    dict(nx=12, ny=12, p=16, overlap=2, precision="tf32", stretch=True),
    dict(nx=10, ny=10, p=8, overlap=1, precision="fp64", nu=("contrast", 10.0)),
    dict(nx=8, ny=8, p=16, overlap=2, precision="bf16", variable_cycle=True),
]


def _ids(c):
    return "_".join("%s%s" % (k, v if not isinstance(v, tuple) else v[1]) for k, v in c.items())


def _solver(case):
    c = dict(case)
    if c.pop("stretch", False):
        c["x_edges"] = list(SI.geometric_edges(c["nx"], 1.0 / c["nx"] / 8))
    return P.Solver(weight=5, tol=1e-10, i_max=100, **c)


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_fused_up_leg_is_bitwise_the_level_by_level_path(case):
    S = _solver(case)
    assert S.fused_prolongation() == (True, True)
    f = torch.from_numpy(SI.uniform_nodal(3, S.shape).ravel()).cuda()
    b = torch.empty_like(f)
    S.mass(f, b)
    runs = {}
    for on in (True, False):
        S.set_fused_prolongation(on)
        assert S.fused_prolongation() == (True, on)
        out = []
        for _ in range(2):  # host loop, then the captured graph
            u = torch.zeros_like(b)
            res, hist = S.pcg_solve(u, b, history_len=101)
            assert res.status == P.SEM_OK
            out.append((res.iterations, np.array(hist[:res.iterations + 1]), u.cpu().numpy()))
        v = torch.zeros_like(b)
        S.vcycle(v, b)
        out.append(v.cpu().numpy())
        runs[on] = out
    for k in range(2):
        it_on, h_on, u_on = runs[True][k]
        it_off, h_off, u_off = runs[False][k]
        assert it_on == it_off
        assert np.array_equal(h_on, h_off)
        assert np.array_equal(u_on, u_off)
    assert np.array_equal(runs[True][2], runs[False][2])
    S.close()


def test_fused_up_leg_unavailable_with_post_smoothing():
    S = P.Solver(nx=8, ny=8, p=16, overlap=2, ns1=1, ns2=1, precision="tf32")
    assert S.fused_prolongation() == (False, False)
    with pytest.raises(P.SemError):
        S.set_fused_prolongation(True)
    S.set_fused_prolongation(False)
    S.close()


def test_fused_up_leg_needs_two_levels():
    S = P.Solver(nx=8, ny=8, p=2, overlap=1, precision="fp64")
    assert S.fused_prolongation() == (False, False)
    S.close()
