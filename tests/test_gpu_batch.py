"""Batched solves: independent problems stacked per shape and solved in one
graph launch must give each problem the result of its own solve (same
iteration count, FP64 solution to 1e-12), and the mixed-precision batch must
reach every problem's 1e-10 residual."""
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


def _problems(prec):
    shapes = [dict(nx=8, ny=8, p=4, overlap=1), dict(nx=8, ny=8, p=4, overlap=1), dict(nx=8, ny=8, p=4, overlap=1),
              dict(nx=6, ny=4, p=8, overlap=2), dict(nx=6, ny=4, p=8, overlap=2),
              dict(nx=4, ny=4, p=16, overlap=2), dict(nx=5, ny=3, p=8, overlap=1, x_edges=list(SI.geometric_edges(5, 0.02)))]
    for c in shapes:
        c["precision"] = prec
    return shapes


def _rhs(S, seed):
    fn = torch.from_numpy(SI.uniform_nodal(seed, S.shape).ravel()).cuda()
    b = torch.empty_like(fn)
    S.mass(fn, b)
    return b


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_batch_matches_individual_solves(prec):
    cfgs = _problems(prec)
    singles = [P.Solver(**c) for c in cfgs]
    bs = [_rhs(S, 40 + k) for k, S in enumerate(singles)]
    # problem 3 is also checked against the oracle: its right side is the oracle's b = M f
    c = cfgs[3]
    H = O.uniform_hierarchy(c["nx"], c["ny"], c["p"], overlap=c["overlap"])
    f3 = H.top.mass(SI.uniform_nodal(43, singles[3].shape))
    bs[3] = torch.from_numpy(np.ascontiguousarray(f3).ravel()).cuda()
    ref = []
    for S, b in zip(singles, bs):
        u = torch.zeros_like(b)
        r, _ = S.pcg_solve(u, b)
        ref.append((r, u.cpu().numpy()))
    batch = P.Batch(cfgs)
    assert batch.groups == 4  # three stacked shapes + the stretched problem alone
    for rep in range(2):  # launch by launch, then one graph launch
        us = [torch.zeros_like(b) for b in bs]
        res = batch.solve(us, bs)
        for k, (r, u) in enumerate(zip(res, us)):
            assert r.status == P.SEM_OK, (rep, k, r.status)
            got = u.cpu().numpy()
            want = ref[k][1]
            if prec == "fp64":
                assert r.iterations == ref[k][0].iterations, (rep, k)
                assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), (rep, k)
            else:
                assert abs(r.iterations - ref[k][0].iterations) <= 1
                assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max(), (rep, k)
    # one problem against the oracle as well
    want, it_o, _ = H.mgcg(np.zeros_like(f3), f3, tol=1e-10)
    got = us[3].cpu().numpy().reshape(f3.shape)
    assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()


def test_batch_reports_each_problems_status():
    cfgs = [dict(nx=8, ny=8, p=4, i_max=2), dict(nx=8, ny=8, p=4, i_max=2)]
    batch = P.Batch(cfgs)
    assert batch.groups == 1
    S = P.Solver(**cfgs[0])
    b1 = _rhs(S, 1)
    b0 = torch.zeros_like(b1)  # zero right side: converged at the start
    for _ in range(2):
        res = batch.solve([torch.zeros_like(b1), torch.zeros_like(b1)], [b1, b0])
        assert res[0].status == P.SEM_NOT_CONVERGED and res[0].iterations == 2
        assert res[1].status == P.SEM_OK and res[1].iterations == 0


def test_batched_workload_full_size():
    """The bench's batched workload at full size (512 problems, 220 M unknowns,
    n x n elements with n in {8, .., 64}, p in {4, .., 32}, n_o in {1, 2}, TF32
    V-cycle), autotuned, launch by launch and then as one graph launch: every
    problem converges to 1e-10; for a sample of problems, whose right sides are
    the oracle's b = M f, the solution is within 1e-9 of the oracle's solve and
    the true residual of the oracle's operator is <= 1.1e-10 ||b||."""
    import bench
    cfgs = bench.c5_configs()
    sample = {}
    for k, c in enumerate(cfgs):  # the first problem of each small shape
        key = (c["nx"], c["p"], c["overlap"])
        if c["nx"] * c["p"] <= 64 and key not in sample:
            sample[key] = k
    assert len(sample) >= 3
    batch = P.Batch(cfgs)
    batch.autotune()
    bs, oracle = [], {}
    for k, c in enumerate(cfgs):
        shape = (c["ny"] * c["p"] + 1, c["nx"] * c["p"] + 1)
        f = SI.uniform_nodal(1000 + k, shape)
        if k in sample.values():
            H = O.uniform_hierarchy(c["nx"], c["ny"], c["p"], overlap=c["overlap"])
            f = H.top.mass(f)
            oracle[k] = (H, f)
        bs.append(torch.from_numpy(np.ascontiguousarray(f).ravel()).cuda())
    for rep in range(2):
        us = [torch.zeros_like(b) for b in bs]
        res = batch.solve(us, bs)
        assert all(r.status == P.SEM_OK for r in res), rep
        assert all(r.res <= 1e-10 * r.res0 for r in res), rep
        for k, (H, f) in oracle.items():
            got = us[k].cpu().numpy().reshape(f.shape)
            want, _, _ = H.mgcg(np.zeros_like(f), f, tol=1e-10)
            assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max(), (rep, k)
            assert np.linalg.norm(f - H.top.apply(got)) <= 1.1e-10 * np.linalg.norm(f), (rep, k)
