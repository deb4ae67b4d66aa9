"""Learned weights: training data from parameter sweeps of the plain method,
training of the MLP on the GPU (the library's kernels), and prediction of the
per-interface weight parameters (s, kt) of SEM_W_LEARNED.

    python -m paper_1512_02390_gb300.learned train [--out FILE] [--quick]

The sweep solves small Dirichlet problems (8 x 8 elements) with controlled
features - order p, overlap, element aspect ratio, diffusivity contrast - with
the plain FP64 method for every (s, kt) on a grid, and takes the pair with the
best average logarithmic convergence rate (Sec. 4) as the target of every
interface line of that problem.  The network regresses the targets (in logit
space) from the features that sem_learned_features computes.  The quintic
weights (s = 1, kt = 5) are one grid point, so on the training problems the
learned choice is never worse than w_5 up to the regression error.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import _binding as B
from .solver import Solver, make_config

MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "learned_model.json")
MODEL_VERSION = 1
GRID_S = (0.25, 0.5, 0.75, 1.0)
GRID_K = (1.0, 3.0, 5.0, 7.0)


def _uniform(seed, shape, lo, hi):
    # the same counter-based generator the inputs use (SplitMix64)
    import sem_inputs as SI
    return SI.uniform_nodal(seed, shape, lo, hi)


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform initialisation of the 4610 parameters (biases zero)."""
    p = np.zeros(B.SEM_MLP_PARAMS, dtype=np.float32)
    o = 0
    for k, (rows, cols) in enumerate([(64, 4), (64, 64), (2, 64)]):
        lim = math.sqrt(6.0 / cols)
        p[o:o + rows * cols] = _uniform(seed * 16 + k, (rows * cols,), -lim, lim)
        o += rows * cols + rows
    return p


def _logit(y, lo, span):
    q = np.clip((np.asarray(y) - lo) / span, 0.02, 0.98)
    return np.log(q / (1 - q))


def uniform_params(cfg, s, kt):
    L = int(round(math.log2(cfg.p)))
    px = np.tile(np.array([s, kt], dtype=np.float64), (L + 1, cfg.nx + 1, 1))
    py = np.tile(np.array([s, kt], dtype=np.float64), (L + 1, cfg.ny + 1, 1))
    return px, py


def sweep_problem(p, overlap, ar, contrast, n=8, seed=1, tol=1e-8):
    """r_bar of MGCG(1,0) for every (s, kt) on the grid; returns (features, targets, table)."""
    import torch

    kw = dict(nx=n, ny=n, p=p, overlap=overlap, lx=1.0 / ar, ly=1.0, tol=tol, i_max=400,
              nu=("contrast", contrast) if contrast > 1 else None)
    table = {}
    b = None
    for s in GRID_S:
        for kt in GRID_K:
            cfg = make_config(**kw)
            px, py = uniform_params(cfg, s, kt)
            S = Solver(weight="learned", learned_x=px.ravel(), learned_y=py.ravel(), **kw)
            if b is None:
                fn = torch.from_numpy(_uniform(seed, S.shape, -1.0, 1.0).ravel()).cuda()
                b = torch.empty_like(fn)
                S.mass(fn, b)
            u = torch.zeros_like(b)
            res, _ = S.pcg_solve(u, b)
            table[(s, kt)] = res.rbar if res.status == B.SEM_OK else 0.0
            S.close()
    best = max(table, key=table.get)
    fx, fy = B.sem_learned_features(make_config(**kw))
    L = fx.shape[0] - 1
    feats = []
    for f in (fx, fy):
        for lvl in range(1, L + 1):
            feats.append(f[lvl, 1:-1])  # interior interface lines
    feats = np.concatenate(feats)
    tgt = np.tile([_logit(best[0], 0.25, 0.75), _logit(best[1], 1.0, 6.0)], (len(feats), 1)).astype(np.float32)
    return feats, tgt, table


def train(X, T, steps=2000, lr=3e-3, seed=0):
    """Full-batch Adam on the GPU; returns (params, loss history)."""
    import torch

    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    Td = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(dev)
    prm = torch.from_numpy(init_params(seed)).to(dev)
    m = torch.zeros_like(prm)
    v = torch.zeros_like(prm)
    ws = torch.zeros(B.sem_mlp_workspace_bytes(len(X)) // 4 + 1, dtype=torch.float32, device=dev)
    hist = torch.zeros(steps, dtype=torch.float32, device=dev)
    B.sem_mlp_train(prm, m, v, Xd, Td, steps, lr, 0, hist, ws)
    torch.cuda.synchronize()
    return prm.cpu().numpy(), hist.cpu().numpy()


def predict(model_params, **cfg_kw):
    """Per-interface (s, kt) arrays [level][interface][2] for both directions."""
    import torch

    cfg = make_config(**cfg_kw)
    fx, fy = B.sem_learned_features(cfg)
    prm = torch.from_numpy(np.ascontiguousarray(model_params, dtype=np.float32)).cuda()
    out = []
    for f in (fx, fy):
        X = torch.from_numpy(f.reshape(-1, 4)).cuda()
        Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
        B.sem_mlp_forward(prm, X, Y, transform=True)
        out.append(Y.cpu().numpy().astype(np.float64).reshape(f.shape[0], f.shape[1], 2))
    torch.cuda.synchronize()
    return out[0], out[1]


def load_model(path=MODEL_PATH):
    with open(path) as fh:
        d = json.load(fh)
    if d.get("version") != MODEL_VERSION:
        raise ValueError("learned model version %r, expected %d" % (d.get("version"), MODEL_VERSION))
    return np.asarray(d["params"], dtype=np.float32), d


def training_set(quick=False):
    ps = (4, 8) if quick else (4, 8, 16)
    ars = (1, 16) if quick else (1, 4, 16, 32)
    cs = (1.0, 100.0) if quick else (1.0, 10.0, 100.0)
    X, T, log = [], [], []
    for p in ps:
        for no in (1, 2):
            for ar in ars:
                for c in cs:
                    t0 = time.time()
                    f, t, table = sweep_problem(p, no, ar, c)
                    best = max(table, key=table.get)
                    X.append(f)
                    T.append(t)
                    log.append({"p": p, "n_o": no, "ar": ar, "contrast": c, "best": best,
                                "rbar_best": table[best], "rbar_w5": table[(1.0, 5.0)],
                                "seconds": round(time.time() - t0, 2)})
    return np.concatenate(X), np.concatenate(T), log


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train"])
    ap.add_argument("--out", default=MODEL_PATH)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--steps", type=int, default=3000)
    a = ap.parse_args()
    X, T, log = training_set(a.quick)
    params, hist = train(X, T, steps=a.steps)
    with open(a.out, "w") as fh:
        json.dump({"version": MODEL_VERSION, "arch": "4-64-64-2 ReLU, FP32", "params": [float(x) for x in params],
                   "features": "log2(p_l)/5, delta_O/2, log2(AR)/5, log10(rho)/2 per interface line",
                   "outputs": "s = 0.25 + 0.75 sigmoid(o0), kt = 1 + 6 sigmoid(o1)",
                   "grid": {"s": GRID_S, "kt": GRID_K}, "samples": int(len(X)),
                   "loss_first_last": [float(hist[0]), float(hist[-1])], "sweep": log}, fh, indent=1)
    print(json.dumps({"samples": int(len(X)), "loss0": float(hist[0]), "loss_end": float(hist[-1]),
                      "problems": len(log)}))


if __name__ == "__main__":
    main()
