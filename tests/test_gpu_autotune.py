"""Launch-shape tuning changes how the V-cycle is launched, not what it
computes: with the scatter fused into the level residual and any number of
subdomains per warp in the mma.sync sweep, MGCG must take the same iterations
and return the bitwise-identical solution, on the first solve (launch by
launch) and on the replayed graph.  The tcgen05 sweep rounds its products in
another order: the same solve to 1e-8 and +-1 iteration.  The autotuner's
JSON-lines cache must round-trip."""
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
    avail = [l for l in range(1, S.levels + 1) if S.get_tune(l)["tc_available"]]
    for tc in (0, 1):
        if tc and not avail:
            continue
        for l in range(1, S.levels + 1):
            S.set_tune(l, 0, 1, tc if l in avail else 0)
        ref = _solves(S, b)
        assert ref[0][1] == P.SEM_OK
        assert np.array_equal(ref[0][2], ref[1][2])
        for fuse, spw in [(1, 1), (1, 2), (0, 4)]:
            for l in range(1, S.levels + 1):
                S.set_tune(l, fuse, spw, tc if l in avail else 0)
            for it, st, u in _solves(S, b):
                assert (it, st) == ref[0][:2], (tc, fuse, spw)
                assert np.array_equal(u, ref[0][2]), (tc, fuse, spw, np.max(np.abs(u - ref[0][2])))
        if tc == 0:
            ref0 = ref
    if avail:  # tcgen05 and mma.sync sweeps round in another order: same solve to the tolerance
        it0, it1 = ref0[0][0], ref[0][0]
        assert abs(it0 - it1) <= 1
        u1, u0 = ref[0][2], ref0[0][2]
        if cfg.get("periodic"):  # solutions are unique up to a constant
            u1, u0 = u1 - u1.mean(), u0 - u0.mean()
        assert np.abs(u1 - u0).max() <= 1e-8 * np.abs(u0).max()


def test_autotune_cache_roundtrip(tmp_path):
    cfg = dict(nx=16, ny=16, p=16, overlap=2, precision="tf32")
    path = str(tmp_path / "tune.jsonl")
    S = P.Solver(**cfg)
    b = _rhs(S, 72)
    tuned = S.autotune(path)
    assert set(tuned) == set(range(1, S.levels + 1))
    for t in tuned.values():
        assert t["fuse"] in (0, 1) and t["spw"] in (1, 2, 4) and t["tc"] in (0, 1) and t["us"] > 0
        assert t["tc"] <= t["tc_available"]
    lines = [json.loads(l) for l in open(path).read().splitlines()]
    low = [d for d in lines if "|low-cycle|" in d["key"]]
    assert len(low) == (1 if S.low_cycle()[0] else 0)
    assert len(lines) == S.levels + len(low)
    assert len({d["key"] for d in lines}) == len(lines)
    ref = _solves(S, b)
    for it, st, u in ref:
        assert st == P.SEM_OK
        assert np.array_equal(u, ref[0][2])
    # a second handle of the same shape reads the cache instead of timing, and
    # solves bitwise the same with the same launch shapes
    S2 = P.Solver(**cfg)
    again = S2.autotune(path)
    for l in tuned:
        for k in ("fuse", "spw", "tc", "eo"):
            assert again[l][k] == tuned[l][k]
        assert abs(again[l]["us"] - round(tuned[l]["us"], 3)) < 1e-9
    assert len(open(path).read().splitlines()) == len(lines)
    assert S2.low_cycle() == S.low_cycle()
    for it, st, u in _solves(S2, b):
        assert (it, st) == ref[0][:2]
        assert np.array_equal(u, ref[0][2])


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
    with pytest.raises(P.SemError):  # FP64: no tensor-core sweep
        S.set_tune(1, 0, 1, tc=1)


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
    got = []
    for rep in range(2):  # the first replays a newly captured graph
        us = [torch.zeros_like(b) for b in bs]
        res = batch.solve(us, bs)
        assert [r.status for r in res] == [P.SEM_OK] * len(cfgs)
        got.append(([r.iterations for r in res], [u.cpu().numpy() for u in us]))
        for k, u in enumerate(got[-1][1]):
            want = first[1][1][k]
            assert abs(got[-1][0][k] - first[1][0][k]) <= 1, k
            assert np.abs(u - want).max() <= 1e-8 * np.abs(want).max(), k
    assert got[0][0] == got[1][0]
    for a, b in zip(got[0][1], got[1][1]):
        assert np.array_equal(a, b)
