"""Launch-shape tuning changes how the V-cycle is launched, never what it
computes: with the scatter fused into the level residual and any number of
subdomains per warp in the tensor-core sweep, MGCG must take the same
iterations and return the bitwise-identical solution, on the first solve
(launch by launch) and on the replayed graph; the autotuner's JSON-lines cache
must round-trip."""
import json

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


def _rhs(S, seed):
    fn = torch.from_numpy(SI.uniform_nodal(seed, S.shape).ravel()).cuda()
    b = torch.empty_like(fn)
    S.mass(fn, b)
    return b


def _solves(S, b, n=2):
    out = []
    for _ in range(n):
        u = torch.zeros_like(b)
        r, _ = S.pcg_solve(u, b)
        out.append((r.iterations, r.status, u.cpu().numpy()))
    return out


CASES = [dict(nx=16, ny=16, p=16, overlap=2, precision="tf32"),
         dict(nx=16, ny=16, p=8, overlap=1, precision="fp32"),
         dict(nx=12, ny=8, p=8, overlap=2, precision="fp64"),
         dict(nx=8, ny=8, p=4, overlap=1, precision="bf16", periodic=True)]


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: "p%d_no%d_%s" % (c["p"], c["overlap"], c["precision"]))
def test_tuned_shapes_give_identical_solves(cfg):
    S = P.Solver(**cfg)
    b = _rhs(S, 71)
    ref = _solves(S, b)
    assert ref[0][1] == P.SEM_OK
    assert np.array_equal(ref[0][2], ref[1][2])
    for fuse, spw in [(1, 1), (1, 2), (0, 4)]:
        for l in range(1, S.levels + 1):
            S.set_tune(l, fuse, spw)
        got = _solves(S, b)
        for it, st, u in got:
            assert (it, st) == ref[0][:2], (fuse, spw)
            assert np.array_equal(u, ref[0][2]), (fuse, spw, np.max(np.abs(u - ref[0][2])))


def test_autotune_cache_roundtrip(tmp_path):
    cfg = dict(nx=16, ny=16, p=16, overlap=2, precision="tf32")
    path = str(tmp_path / "tune.jsonl")
    S = P.Solver(**cfg)
    b = _rhs(S, 72)
    ref = _solves(S, b)
    tuned = S.autotune(path)
    assert set(tuned) == set(range(1, S.levels + 1))
    for fuse, spw, us in tuned.values():
        assert fuse in (0, 1) and spw in (1, 2, 4) and us > 0
    lines = [json.loads(l) for l in open(path).read().splitlines()]
    assert len(lines) == S.levels
    assert len({d["key"] for d in lines}) == S.levels
    got = _solves(S, b)
    for it, st, u in got:
        assert (it, st) == ref[0][:2]
        assert np.array_equal(u, ref[0][2])
    # a second handle of the same shape reads the cache instead of timing
    S2 = P.Solver(**cfg)
    again = S2.autotune(path)
    for l in tuned:
        assert again[l][:2] == tuned[l][:2]
        assert abs(again[l][2] - round(tuned[l][2], 3)) < 1e-9
    assert len(open(path).read().splitlines()) == S.levels


def test_set_tune_rejects_bad_values():
    S = P.Solver(nx=8, ny=8, p=8, overlap=1)
    with pytest.raises(P.SemError):
        S.set_tune(0, 0, 1)
    with pytest.raises(P.SemError):
        S.set_tune(S.levels + 1, 0, 1)
    with pytest.raises(P.SemError):
        S.set_tune(1, 2, 1)
    with pytest.raises(P.SemError):
        S.set_tune(1, 0, 0)


def test_batch_autotune_keeps_results(tmp_path):
    cfgs = [dict(nx=8, ny=8, p=8, overlap=1, precision="tf32") for _ in range(3)]
    cfgs += [dict(nx=8, ny=8, p=4, overlap=1, precision="tf32")]
    singles = [P.Solver(**c) for c in cfgs]
    bs = [_rhs(S, 80 + k) for k, S in enumerate(singles)]
    batch = P.Batch(cfgs)
    first = []
    for rep in range(2):
        us = [torch.zeros_like(b) for b in bs]
        res = batch.solve(us, bs)
        first.append(([r.iterations for r in res], [u.cpu().numpy() for u in us]))
    batch.autotune(str(tmp_path / "tune.jsonl"))
    for rep in range(2):  # the first replays a newly captured graph
        us = [torch.zeros_like(b) for b in bs]
        res = batch.solve(us, bs)
        assert [r.status for r in res] == [P.SEM_OK] * len(cfgs)
        assert [r.iterations for r in res] == first[1][0]
        for k, u in enumerate(us):
            assert np.array_equal(u.cpu().numpy(), first[1][1][k]), k
