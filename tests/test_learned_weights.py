"""Learned-weight parameterisation (per interface line: width scale s and
continuous shape degree kt): properties that hold for any parameter values,
checked on the oracle and on the library's host set-up (no GPU)."""
import numpy as np
import pytest

import sem_inputs as SI
from oracle import sem_oracle as O


def _params(n, levels, seed):
    u = SI.uniform_nodal(seed, (levels, n + 1, 2), 0.0, 1.0)
    prm = np.empty_like(u)
    prm[..., 0] = 0.25 + 0.75 * u[..., 0]
    prm[..., 1] = 1.0 + 6.0 * u[..., 1]
    return prm


@pytest.mark.parametrize("kt", [1.0, 3.0, 5.0, 7.0])
def test_blend_at_odd_degrees_is_the_table_shape_function(kt):
    x = np.linspace(-1.3, 1.3, 101)
    np.testing.assert_allclose(O.phi_blend(kt, x), O.phi(int(kt), x), atol=1e-15)


@pytest.mark.parametrize("kt", [1.0, 2.2, 4.5, 6.9])
def test_blend_is_odd_monotone_and_saturates(kt):
    x = np.linspace(-0.999, 0.999, 999)
    y = O.phi_blend(kt, x)
    np.testing.assert_allclose(y, -O.phi_blend(kt, -x), atol=1e-15)
    assert np.all(np.diff(y) > 0)
    assert O.phi_blend(kt, 1.0) == 1.0 and O.phi_blend(kt, -1.0) == -1.0


@pytest.mark.parametrize("periodic,edges", [(False, None), (True, None), (False, "stretched")])
def test_learned_weights_partition_of_unity(periodic, edges):
    n, p, n_o = 6, 8, 2
    mx = O.Mesh1D.uniform(n, 1.0, periodic) if edges is None else O.Mesh1D(SI.geometric_edges(n, 0.02), periodic)
    prm = _params(n, 1, 5)[0]
    lev = O.Level(mx, O.Mesh1D.uniform(n, 1.0, periodic), p, n_o, weight="learned",
                  learned=(prm, _params(n, 1, 6)[0]))
    tot = np.zeros((lev.NY, lev.NX))
    for sy in lev.sub_y:
        for sx in lev.sub_x:
            tot[np.ix_(sy.g, sx.g)] += np.outer(sy.w, sx.w)
    assert np.abs(tot[lev.unknown] - 1).max() < 1e-13


def test_learned_with_unit_scale_and_degree_five_is_quintic():
    n, p = 5, 8
    prm = np.tile([1.0, 5.0], (n + 1, 1))
    mx = O.Mesh1D(SI.geometric_edges(n, 0.05), False)
    a = O.Level(mx, O.Mesh1D.uniform(n, 1.0, False), p, 2, weight="learned", learned=(prm, prm))
    b = O.Level(mx, O.Mesh1D.uniform(n, 1.0, False), p, 2, weight=5)
    for sa, sb in zip(a.sub_x, b.sub_x):
        np.testing.assert_allclose(sa.w, sb.w, atol=1e-15)


def test_library_learned_tables_match_oracle():
    P = pytest.importorskip("paper_1512_02390_gb300")
    try:
        P.load_library()
    except RuntimeError as e:
        pytest.skip(str(e))
    n, p = 6, 16
    L = 4
    px, py = _params(n, L + 1, 7), _params(n, L + 1, 8)
    edges = SI.geometric_edges(n, 0.01)
    cfg = P.make_config(nx=n, ny=n, p=p, overlap=2, weight="learned", x_edges=edges,
                        learned_x=px.ravel(), learned_y=py.ravel())
    for level in range(1, L + 1):
        t = P.sem_inspect_level(cfg, level)
        pl = 2**level
        lev = O.Level(O.Mesh1D(edges, False), O.Mesh1D.uniform(n, 1.0, False), pl, t["n_o"], weight="learned",
                      learned=(px[level], py[level]))
        for e in range(n):
            s = lev.sub_x[e]
            w = np.zeros(t["m"])
            w[s.k + t["n_o"]] = s.w
            np.testing.assert_allclose(t["w"][t["tab"][e]], w, atol=1e-13)
