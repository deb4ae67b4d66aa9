"""The FP64 MLP oracle's backpropagation against central finite differences
of its own forward pass (pins the oracle; no GPU)."""
import numpy as np

import sem_inputs as SI
from oracle import mlp_oracle as M


def _data(seed, n=37):
    prm = SI.uniform_nodal(seed, (M.N_PARAMS,), -0.5, 0.5)
    X = SI.uniform_nodal(seed + 1, (n, 4), -1.0, 1.0)
    T = SI.uniform_nodal(seed + 2, (n, 2), -2.0, 2.0)
    return prm, X, T


def test_backprop_equals_finite_differences():
    prm, X, T = _data(3)
    loss, g = M.loss_grad(prm, X, T)
    idx = np.linspace(0, M.N_PARAMS - 1, 97).astype(int)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(prm)
        e[i] = h
        fd = (M.loss_grad(prm + e, X, T)[0] - M.loss_grad(prm - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (abs(g[i]) + 1e-3), (i, fd, g[i])


def test_forward_layer_structure():
    prm, X, _ = _data(5, n=3)
    W1, b1, W2, b2, W3, b3 = M.unpack(prm)
    o, _ = M.forward(prm, X)
    x = X[1]
    h1 = np.maximum(W1 @ x + b1, 0)
    h2 = np.maximum(W2 @ h1 + b2, 0)
    np.testing.assert_allclose(o[1], W3 @ h2 + b3, rtol=1e-14)
    assert M.N_PARAMS == 4610
