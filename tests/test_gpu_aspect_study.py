"""The solver-parameter study of Sec. 4.2 (Fig. 3) on the GPU: MGCG variants
at p = 16 on 16 x 16 periodic elements of aspect ratio AR = 1..16, compared
with what the text states about the figure (tests/golden/fig3_text_values.txt)
and with Table 4's MGCG(1,0) column.

Operator applications per decade: omega_1 = (1 / r_bar) W_cyc / W_op with the
cost model of Sec. 4, W_cyc / W_op = [4 (1 + 2 n_o / n_p)^3 c_s n_s + 2 c_s +
c_cg] / 2, n_s = pre- plus post-smoothing steps, c_s = 4/3 (2 for the
variable V-cycle), c_cg = 2.  The multiplicative smoother runs in the
coloured order (a departure from Alg. 1's lexicographic order that converges
faster), so its omega_1 is held to at most the printed value.
"""
import numpy as np
import pytest

import sem_inputs as SI
from tests._golden import rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1512_02390_gb300")

ARS = (1, 2, 4, 8, 16)
VARIANTS = {
    "add_w5_10": dict(smoother="add", weight=5, overlap="ceil8", ns=(1, 0)),
    "add_w5_11": dict(smoother="add", weight=5, overlap="ceil8", ns=(1, 1)),
    "mult_11": dict(smoother="mult", weight=5, overlap="ceil8", ns=(1, 1)),
    "add_w5_11_var": dict(smoother="add", weight=5, overlap="ceil8", ns=(1, 1), variable=True),
    "mult_no0_22": dict(smoother="mult", weight=5, overlap=0, ns=(2, 2)),
    "add_wa_no1_11": dict(smoother="add", weight="a", overlap=1, ns=(1, 1)),
}


def omega1(rbar, n_o, p, ns, variable):
    cs = 2.0 if variable else 4.0 / 3.0
    return (4 * (1 + 2 * n_o / (p + 1)) ** 3 * cs * ns + 2 * cs + 2.0) / 2.0 / rbar


@pytest.fixture(scope="module")
def study():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = {}
    for AR in ARS:
        for name, v in VARIANTS.items():
            S = P.Solver(nx=16, ny=16, p=16, periodic=True, lx=2.0 * AR, ly=2.0, overlap=v["overlap"],
                         weight=v["weight"], smoother=v["smoother"], ns1=v["ns"][0], ns2=v["ns"][1],
                         variable_cycle=v.get("variable", False), tol=1e-10, i_max=400)
            x, y = S.coords()
            f = 2 * np.pi**2 * np.sin(np.pi * x[None, :]) * np.sin(np.pi * y[:, None])
            b = torch.empty(f.size, dtype=torch.float64, device="cuda")
            S.mass(torch.from_numpy(f.ravel()).cuda(), b)
            u = torch.from_numpy(SI.uniform_nodal(1, S.shape, 0.0, 1.0).ravel()).cuda()
            res, _ = S.pcg_solve(u, b)
            assert res.status == P.SEM_OK, (name, AR)
            no = {"ceil8": 2}.get(v["overlap"], v["overlap"])
            out[name, AR] = (res.rbar, omega1(res.rbar, no, 16, sum(v["ns"]), v.get("variable", False)))
    return out


def _text():
    return {r[0]: float(r[1]) for r in rows("fig3_text_values.txt")}


def test_mgcg10_matches_table4(study):
    want = {int(r[1]): float(r[4]) for r in rows("table4_aspect_ratio.txt") if int(r[0]) == 16}
    for AR in (1, 2, 4, 8):
        rb = study["add_w5_10", AR][0]
        assert abs(rb - want[AR]) <= 0.05 * want[AR] + 0.02, (AR, rb, want[AR])


def test_post_smoothing_raises_rate_by_1p5_to_2(study):
    t = _text()
    for AR in ARS:
        k = study["add_w5_11", AR][0] / study["add_w5_10", AR][0]
        assert t["post_smoothing_rbar_factor_min"] - 0.05 <= k <= t["post_smoothing_rbar_factor_max"] + 0.05, (AR, k)


def test_operator_applications_at_aspect_ratio_16(study):
    """About 34 operator applications per decade for the additive w_5
    MGCG(1,1) at AR = 16, against 26 for the multiplicative one, which needs
    the fewest of the figure's MGCG(1,1) and (2,2) variants at every AR."""
    t = _text()
    om_add, om_mult = study["add_w5_11", 16][1], study["mult_11", 16][1]
    assert abs(om_add - t["omega1_mgcg11_add_w5_AR16"]) <= 0.15 * t["omega1_mgcg11_add_w5_AR16"], om_add
    assert om_mult <= 1.05 * t["omega1_mgcg11_mult_AR16"], om_mult
    for AR in ARS:  # among the variants of the figure (two or more smoothing steps)
        best = min(study[k, AR][1] for k in VARIANTS if k != "add_w5_10")
        assert study["mult_11", AR][1] == best, AR


def test_variable_cycle_costs_more_than_it_gains(study):
    for AR in ARS:
        assert study["add_w5_11_var", AR][1] > study["add_w5_11", AR][1], AR


def test_zero_overlap_mgcg22_like_mgcg10(study):
    """Multiplicative MGCG(2,2) with n_o = 0 converges at a rate similar to the
    additive MGCG(1,0) with level-dependent overlap."""
    for AR in ARS:
        k = study["mult_no0_22", AR][0] / study["add_w5_10", AR][0]
        assert 0.7 <= k <= 1.6, (AR, k)


def test_arithmetic_two_steps_against_quintic_one_step(study):
    """w_a with n_o = 1 and two smoothing steps reaches about two thirds of
    the rate of w_5 with one step at AR = 1 and overtakes it at larger AR."""
    k1 = study["add_wa_no1_11", 1][0] / study["add_w5_10", 1][0]
    assert 0.55 <= k1 <= 0.8, k1
    for AR in (4, 8, 16):
        assert study["add_wa_no1_11", AR][0] > study["add_w5_10", AR][0], AR
