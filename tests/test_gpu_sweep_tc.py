"""The reduced-precision Schwarz sweep on the tcgen05 tensor cores (stacks of
floor(128 / m) subdomains per MMA) against the FP64 oracle: one weighted
additive correction from u = 0 (Alg. 2, Eq. (correction:global)) on meshes
large enough that the stacks are built (several tiles of stacks, partial last
stacks, wall-adjacent table classes, periodic wrap, a stretched direction,
variable diffusivity).  Bar: 64 u_in of max|correction| (four contractions,
each rounding its operands once), the same bar as the mma.sync kernel, which
is checked on the same inputs."""
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


U_IN = {"tf32": 2.0**-11, "bf16": 2.0**-8}

CASES = [
    dict(nx=32, ny=30, p=2, overlap=1),                     # m = 5, 25 per stack
    dict(nx=24, ny=20, p=4, overlap=1),                     # m = 7, 18 per stack, wall classes
    dict(nx=20, ny=18, p=4, overlap=2, periodic=True),      # m = 9
    dict(nx=16, ny=16, p=4, overlap=3),                     # m = 11
    dict(nx=14, ny=12, p=8, overlap=3),                     # m = 15
    dict(nx=12, ny=14, p=8, overlap=4),                     # m = 17, 7 per stack
    dict(nx=16, ny=12, p=8, overlap=2, periodic=True),      # m = 13, one table class
    dict(nx=12, ny=10, p=16, overlap=2),                    # m = 21, the bench's window
    dict(nx=12, ny=9, p=16, overlap=1),                     # m = 19
    dict(nx=10, ny=8, p=16, overlap=3, periodic=True),      # m = 23, periodic wrap of every window
    dict(nx=12, ny=12, p=16, overlap=2, stretch=True),      # m = 21, a table per column (tables change mid-range)
    dict(nx=12, ny=10, p=16, overlap=1, nu=("contrast", 10.0)),  # m = 19, 1 / nu_bar per subdomain
    dict(nx=7, ny=6, p=32, overlap=2),                      # m = 37, three per stack, 48-column accumulator
    dict(nx=6, ny=7, p=32, overlap=1, periodic=True),       # m = 35, periodic wrap
    dict(nx=5, ny=6, p=32, overlap=3),                      # m = 39, two gather passes per window row
    dict(nx=24, ny=24, p=8, overlap=1, stretch=True),       # x geometric: a table per column
    dict(nx=16, ny=16, p=8, overlap=1, nu=("contrast", 10.0)),  # 1 / nu_bar per subdomain
]


def _ids(c):
    return "_".join("%s%s" % (k, v if not isinstance(v, tuple) else v[1]) for k, v in c.items())


def _pair(case, prec):
    c = dict(case)
    edges = None
    if c.pop("stretch", False):
        edges = SI.geometric_edges(c["nx"], 1.0 / c["nx"] / 8)
    nu = c.pop("nu", None)
    S = P.Solver(precision=prec, x_edges=None if edges is None else list(edges), nu=nu, **c)
    periodic = c.get("periodic", False)
    mx = O.Mesh1D.uniform(c["nx"], 1.0, periodic) if edges is None else O.Mesh1D(np.asarray(edges), periodic)
    H = O.Hierarchy(mx, O.Mesh1D.uniform(c["ny"], 1.0, periodic), c["p"], overlap=c["overlap"], weight=5,
                    nu=None if nu is None else SI.nu_contrast(nu[1]))
    return S, H


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_tcgen05_sweep_matches_oracle(case, prec):
    S, H = _pair(case, prec)
    top = S.levels
    assert S.get_tune(top)["tc_available"] == 1, "stacks not built for this case"
    lev = H.top
    f = lev.mass(SI.uniform_nodal(21, (lev.NY, lev.NX)))
    want = lev.wschwarz(np.zeros_like(f), f, 1)
    fd = torch.from_numpy(np.ascontiguousarray(f).reshape(-1)).cuda()
    scale = np.abs(want).max()
    for tc in (1, 0):  # tcgen05 stacks, then mma.sync on the same inputs
        S.set_tune(top, 0, 1, tc)
        ud = torch.zeros_like(fd)
        S.smooth(ud, fd, 1)
        torch.cuda.synchronize()
        got = ud.cpu().numpy().reshape(lev.NY, lev.NX)
        err = np.abs(got - want).max() / scale
        assert err < 64 * U_IN[prec], (tc, err)


@pytest.fixture(scope="module")
def mgcg_oracle():
    """The oracle's FP64 MGCG solve of the 16 x 16, p = 16, n_o = 2 problem."""
    H = O.uniform_hierarchy(16, 16, 16, periodic=False, overlap=2, weight=5)
    lev = H.top
    b = lev.mass(SI.uniform_nodal(5, (lev.NY, lev.NX)))
    u, it, _ = H.mgcg(np.zeros_like(b), b, tol=1e-12)
    return lev, b, u


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tcgen05_mgcg_reaches_fp64_accuracy(prec, mgcg_oracle):
    """MGCG with the tcgen05 sweep on every level that has stacks: the true
    residual of the oracle's operator reaches 1e-10 ||b|| and the solution
    agrees with the oracle's FP64 solve to 1e-9."""
    lev, b, want = mgcg_oracle
    S = P.Solver(precision=prec, nx=16, ny=16, p=16, overlap=2)
    assert any(S.get_tune(l)["tc"] for l in range(1, S.levels + 1))
    bd = torch.from_numpy(np.ascontiguousarray(b).reshape(-1)).cuda()
    for _ in range(2):  # host loop, then the captured graph
        u = torch.zeros_like(bd)
        r, _ = S.pcg_solve(u, bd)
        assert r.status == P.SEM_OK
        assert r.res <= 1e-10 * r.res0
        got = u.cpu().numpy().reshape(b.shape)
        assert np.linalg.norm(b - lev.apply(got)) <= 1.1e-10 * np.linalg.norm(b)
        rel = np.abs(got - want).max() / np.abs(want).max()
        assert rel < 1e-9, rel
