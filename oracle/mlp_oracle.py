"""Plain FP64 numpy model of the learned-weight MLP (4 -> 64 -> 64 -> 2,
ReLU hidden layers, linear output), its mean-squared loss and its gradient by
textbook backpropagation.

TEST INFRASTRUCTURE ONLY: the GPU library's forward, backward and training
kernels are checked against this module (and against finite differences of
its forward); only tests/ and the CPU legs of bench.py use it.

Parameter vector layout (4610 values): W1 (64 x 4), b1 (64), W2 (64 x 64),
b2 (64), W3 (2 x 64), b3 (2), each row-major.  Loss over N samples:
L = (1 / (2N)) sum_n sum_j (o_nj - t_nj)^2.
"""
import numpy as np

N_IN, N_HID, N_OUT = 4, 64, 2
N_PARAMS = N_HID * N_IN + N_HID + N_HID * N_HID + N_HID + N_OUT * N_HID + N_OUT


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    out = []
    for shape in [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_OUT, N_HID), (N_OUT,)]:
        k = int(np.prod(shape))
        out.append(p[o:o + k].reshape(shape))
        o += k
    return out


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    return h2 @ W3.T + b3, (z1, h1, z2, h2)


def loss_grad(params, X, T):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    o, (z1, h1, z2, h2) = forward(params, X)
    d = (o - T) / n
    loss = 0.5 * np.sum((o - T) ** 2) / n
    gW3 = d.T @ h2
    gb3 = d.sum(0)
    dh2 = (d @ W3) * (z2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def to_weight_params(o):
    """Network outputs -> (s, kt): s = 0.25 + 0.75 sigmoid(o0), kt = 1 + 6 sigmoid(o1)."""
    sg = 1.0 / (1.0 + np.exp(-np.asarray(o, dtype=np.float64)))
    return np.stack([0.25 + 0.75 * sg[..., 0], 1.0 + 6.0 * sg[..., 1]], axis=-1)
