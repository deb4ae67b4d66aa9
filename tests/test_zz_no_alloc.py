"""The allocation-free Schwarz correction (sem_schwarz_correction_noalloc).

It serves callers that cannot call cudaMalloc — code inside a framework that
owns the device memory through its own pool, code with a fixed memory budget,
latency-critical loops where an allocation would synchronise the device — by
keeping its scratch in a static device array.  This test calls it through the
C ABI and checks it against the regular entry point sem_smooth (one sweep from
u = 0 is exactly one correction of r = f) on two calls in a row, and checks that
a problem larger than the static scratch is rejected.  It lives in its own file,
collected last, and needs nothing from the other tests.
"""
import numpy as np
import pytest

import sem_inputs as SI

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1512_02390_gb300")


def _tables(cfg, level):
    """Upload the x-direction tables that sem_inspect_level reports."""
    t = P.sem_inspect_level(cfg, level)
    keep = [torch.from_numpy(np.ascontiguousarray(t["tab"])).cuda(),
            torch.from_numpy(np.ascontiguousarray(t["S"])).cuda(),
            torch.from_numpy(np.ascontiguousarray(t["lam"])).cuda(),
            torch.from_numpy(np.ascontiguousarray(t["w"])).cuda()]
    d = P.sem_sweep_tables(n=cfg.nx, p=t["p"], n_o=t["n_o"], periodic=cfg.periodic, tab=keep[0].data_ptr(),
                           S=keep[1].data_ptr(), lam=keep[2].data_ptr(), w=keep[3].data_ptr())
    return d, keep, t


def _tables_xy(nx, ny, periodic, level=4):
    """x tables of an nx x ny mesh, and its y tables as the x tables of the
    ny x nx mesh on the same unit square (same element widths and walls)."""
    kw = dict(p=16, periodic=periodic, overlap=2, weight=5)
    dx, kx, t = _tables(P.make_config(nx=nx, ny=ny, **kw), level)
    dy, ky, _ = _tables(P.make_config(nx=ny, ny=nx, **kw), level)
    return dx, dy, kx + ky, t


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("nx,ny", [(8, 8), (8, 4)])
def test_noalloc_correction_matches_regular_entry_point(periodic, nx, ny):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S = P.Solver(nx=nx, ny=ny, p=16, periodic=periodic, overlap=2, weight=5)
    dx, dy, keep, t = _tables_xy(nx, ny, periodic)
    m = t["p"] + 1 + 2 * t["n_o"]
    # FP64 bar of the sweep tests: eps * m^3 (four length-m contractions)
    tol = max(1e-12, np.finfo(np.float64).eps * m**3)
    for seed in (21, 22):  # two calls in a row, different right sides
        r = torch.from_numpy(SI.uniform_nodal(seed, S.shape).ravel()).cuda()
        u_ref = torch.zeros_like(r)
        S.smooth(u_ref, r, 1)  # from u = 0 the residual is r itself
        u = torch.zeros_like(r)
        P.sem_schwarz_correction_noalloc(dx, dy, r, u)
        torch.cuda.synchronize()
        a, b = u.cpu().numpy(), u_ref.cpu().numpy()
        assert np.abs(a - b).max() <= tol * np.abs(b).max()
    del keep


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = P.make_config(nx=8, ny=8, p=16, overlap=2)
    d, keep, _ = _tables(cfg, 4)
    big = P.sem_sweep_tables(n=128, p=16, n_o=2, periodic=0, tab=d.tab, S=d.S, lam=d.lam, w=d.w)
    # never touched: the call is rejected before any device work
    r = torch.zeros((128 * 16 + 1) ** 2, dtype=torch.float64, device="cuda")
    with pytest.raises(P.SemError) as ei:
        P.sem_schwarz_correction_noalloc(big, big, r, r)
    assert ei.value.status == P.SEM_BAD_ARG
    assert "static limit" in str(ei.value)
    del keep


def test_noalloc_rejects_windows_beyond_shared_memory_then_runs():
    """p = 32, n_o = 26 (m = 85) fits the static scratch on 2 x 2 elements but
    its FP64 local solve does not fit one block's shared memory: a bad
    argument, and a valid call right after it still succeeds."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = P.make_config(nx=8, ny=8, p=16, overlap=2)
    d, keep, _ = _tables(cfg, 4)
    wide = P.sem_sweep_tables(n=2, p=32, n_o=26, periodic=0, tab=d.tab, S=d.S, lam=d.lam, w=d.w)
    r = torch.zeros((2 * 32 + 1) ** 2, dtype=torch.float64, device="cuda")
    with pytest.raises(P.SemError) as ei:
        P.sem_schwarz_correction_noalloc(wide, wide, r, r)
    assert ei.value.status == P.SEM_BAD_ARG
    assert "shared memory" in str(ei.value)
    S = P.Solver(nx=8, ny=8, p=16, overlap=2, weight=5)
    rr = torch.from_numpy(SI.uniform_nodal(23, S.shape).ravel()).cuda()
    u_ref = torch.zeros_like(rr)
    S.smooth(u_ref, rr, 1)
    u = torch.zeros_like(rr)
    P.sem_schwarz_correction_noalloc(d, d, rr, u)
    torch.cuda.synchronize()
    a, b = u.cpu().numpy(), u_ref.cpu().numpy()
    assert np.abs(a - b).max() <= max(1e-12, np.finfo(np.float64).eps * 21**3) * np.abs(b).max()
    del keep
