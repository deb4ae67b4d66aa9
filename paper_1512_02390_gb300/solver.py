"""Convenience wrapper around one sem_handle (argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding as B

_WEIGHTS = {1: B.SEM_W_LINEAR, 3: B.SEM_W_CUBIC, 5: B.SEM_W_QUINTIC, 7: B.SEM_W_SEPTIC,
            "t": B.SEM_W_TOPHAT, "a": B.SEM_W_ARITH, "I": B.SEM_W_IDENTITY, "learned": B.SEM_W_LEARNED}
_OVERLAP = {"floor8": B.SEM_OVERLAP_FLOOR8, "ceil8": B.SEM_OVERLAP_CEIL8, "ceil2": B.SEM_OVERLAP_CEIL2}
_PREC = {"fp64": B.SEM_PREC_FP64, "fp32": B.SEM_PREC_FP32, "tf32": B.SEM_PREC_TF32, "bf16": B.SEM_PREC_BF16}


def make_config(nx=4, ny=4, p=4, periodic=False, lx=1.0, ly=1.0, overlap=1, weight=5, ns1=1, ns2=0,
                variable_cycle=False, precision="fp64", tol=1e-10, i_max=200, x_edges=None, y_edges=None,
                nu=None, learned_x=None, learned_y=None, smoother="add", mlp_params=None):
    """nu: None (Poisson), ("contrast", c) or ("paper", amplitude, shift).
    smoother: "add" (Alg. 2) or "mult" (Alg. 1).  mlp_params: the weight
    network's parameters, used by sem_create when weight="learned" and no
    learned_x / learned_y are given."""
    cfg = B.sem_default_config()
    cfg.nx, cfg.ny, cfg.p, cfg.periodic = nx, ny, p, int(bool(periodic))
    cfg.lx, cfg.ly = lx, ly
    if isinstance(overlap, str):
        cfg.overlap_rule, cfg.overlap = _OVERLAP[overlap], 0
    else:
        cfg.overlap_rule, cfg.overlap = B.SEM_OVERLAP_FIXED, int(overlap)
    cfg.weight = _WEIGHTS[weight]
    cfg.ns1, cfg.ns2, cfg.variable_cycle = ns1, ns2, int(bool(variable_cycle))
    cfg.precision = _PREC[precision]
    cfg.tol, cfg.i_max = tol, i_max
    cfg.smoother = {"add": B.SEM_SMOOTH_ADDITIVE, "mult": B.SEM_SMOOTH_MULT}[smoother]
    if nu is not None:
        if nu[0] == "contrast":
            cfg.nu_kind, cfg.nu_a, cfg.nu_b = 1, float(nu[1]), 0.0
        elif nu[0] == "paper":
            cfg.nu_kind, cfg.nu_a, cfg.nu_b = 2, float(nu[1]), float(nu[2])
        else:
            raise ValueError(nu)
    keep = []
    for name, e in (("x_edges", x_edges), ("y_edges", y_edges), ("learned_x", learned_x), ("learned_y", learned_y)):
        if e is not None:
            arr = np.ascontiguousarray(e, dtype=np.float64)
            keep.append(arr)
            setattr(cfg, name, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if mlp_params is not None:
        arr = np.ascontiguousarray(mlp_params, dtype=np.float32)
        if arr.size != B.SEM_MLP_PARAMS:
            raise ValueError("expected %d network parameters" % B.SEM_MLP_PARAMS)
        keep.append(arr)
        cfg.mlp_params = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    cfg._keep = keep  # keep edge arrays alive while the config is in use
    return cfg


class Solver:
    """One solver handle on the current CUDA device."""

    def __init__(self, **kw):
        self.cfg = make_config(**kw)
        self.h = B.sem_create(self.cfg)
        self.n_unknowns, self.nx_nodes, self.ny_nodes = B.sem_sizes(self.h)
        self.shape = (self.ny_nodes, self.nx_nodes)
        self.levels = int(self.cfg.p).bit_length() - 1  # L = log2(p)

    def close(self):
        if self.h is not None:
            B.sem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coords(self):
        return B.sem_coords(self.h)

    def mass(self, f_nodal, b, stream=None):
        B.sem_mass(self.h, f_nodal, b, stream)

    def apply(self, u, Au, stream=None):
        B.sem_apply(self.h, u, Au, stream)

    def smooth(self, u, f, n_it=1, stream=None):
        B.sem_smooth(self.h, u, f, n_it, stream)

    def vcycle(self, u, f, stream=None):
        B.sem_vcycle(self.h, u, f, stream)

    def mg_solve(self, u, f, history_len=0, stream=None):
        return B.sem_mg_solve(self.h, u, f, history_len, stream)

    def pcg_solve(self, u, f, history_len=0, stream=None):
        return B.sem_pcg_solve(self.h, u, f, history_len, stream)

    def profile(self, enable=True):
        B.sem_profile(self.h, enable)

    def profile_read(self):
        return B.sem_profile_read(self.h)

    def profile_read_level(self, level):
        return B.sem_profile_read_level(self.h, level)

    def autotune(self, cache_path=None, stream=None):
        """Pick the launch shapes of every level by timing (results unchanged)."""
        B.sem_autotune(self.h, cache_path, stream)
        return {l: B.sem_get_tune(self.h, l) for l in range(1, self.levels + 1)}

    def set_tune(self, level, fuse, spw=1, tc=0, eo=-1):
        B.sem_set_tune(self.h, level, fuse, spw, tc, eo)

    def get_tune(self, level):
        return B.sem_get_tune(self.h, level)

    def mlp_load(self, params):
        """Learned weights from the network parameters (sem_mlp_load)."""
        B.sem_mlp_load(self.h, params)

    def set_low_cycle(self, enable):
        B.sem_set_low_cycle(self.h, enable)

    def low_cycle(self):
        """(available, enabled) of the persistent low-level cycle."""
        return B.sem_get_low_cycle(self.h)

    def set_fused_prolongation(self, enable):
        B.sem_set_fused_prolongation(self.h, enable)

    def fused_prolongation(self):
        """(available, enabled) of the one-launch up-leg of the V-cycle."""
        return B.sem_get_fused_prolongation(self.h)

    def set_fixed_point_operator(self, enable):
        B.sem_set_fixed_point_operator(self.h, enable)

    def fixed_point_operator(self):
        """(available, enabled) of the FP64 operator in exact integer arithmetic."""
        return B.sem_get_fixed_point_operator(self.h)

    def set_tune_from(self, other):
        """Copy the launch shapes of a handle with the same levels."""
        for l in range(1, self.levels + 1):
            t = other.get_tune(l)
            tc = t["tc"] if self.get_tune(l)["tc_available"] else 0
            B.sem_set_tune(self.h, l, t["fuse"], t["spw"], tc, t["eo"])


def batch_workload(count=512, seed=7, precision="tf32", tol=1e-10, i_max=200):
    """The seeded batched workload: problem k has n x n elements (n in
    {8, 16, 32, 64}), order p in {4, 8, 16, 32} and overlap n_o in {1, 2},
    drawn uniformly and independently with SplitMix64 (seed 7), Dirichlet
    walls, w_5."""
    import sem_inputs as SI
    d = (SI.uniform01(seed, 3 * count).reshape(count, 3) * np.array([4, 4, 2])).astype(int)
    return [dict(nx=8 << int(a), ny=8 << int(a), p=4 << int(b), overlap=1 + int(c), weight=5, precision=precision,
                 tol=tol, i_max=i_max) for a, b, c in d]


class Batch:
    """Many independent problems solved together (sem_batch_*)."""

    def __init__(self, configs):
        self.configs = [make_config(**c) for c in configs]
        self.h = B.sem_batch_create(self.configs)
        self.groups, self.unknowns = B.sem_batch_info(self.h)

    def close(self):
        if self.h is not None:
            B.sem_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, us, fs, stream=None):
        return B.sem_batch_solve(self.h, us, fs, stream)

    def launches(self):
        return B.sem_batch_launches(self.h)

    def autotune(self, cache_path=None, stream=None):
        B.sem_batch_autotune(self.h, cache_path, stream)


class Solver3:
    """One handle of the three-dimensional extension on the current CUDA device."""

    def __init__(self, nx=4, ny=4, nz=4, p=4, periodic=False, lx=1.0, ly=1.0, lz=1.0, overlap=1, weight=5, ns1=1,
                 ns2=0, precision="fp64", tol=1e-10, i_max=200):
        cfg = B.sem3_default_config()
        cfg.nx, cfg.ny, cfg.nz, cfg.p, cfg.periodic = nx, ny, nz, p, int(bool(periodic))
        cfg.lx, cfg.ly, cfg.lz = lx, ly, lz
        if isinstance(overlap, str):
            cfg.overlap_rule, cfg.overlap = _OVERLAP[overlap], 0
        else:
            cfg.overlap_rule, cfg.overlap = B.SEM_OVERLAP_FIXED, int(overlap)
        cfg.weight = _WEIGHTS[weight]
        cfg.ns1, cfg.ns2 = ns1, ns2
        cfg.precision = _PREC[precision]
        cfg.tol, cfg.i_max = tol, i_max
        self.cfg = cfg
        self.h = B.sem3_create(cfg)
        self.n_unknowns, nxn, nyn, nzn = B.sem3_sizes(self.h)
        self.shape = (nzn, nyn, nxn)

    def close(self):
        if self.h is not None:
            B.sem3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coords(self):
        return B.sem3_coords(self.h)

    def mass(self, f_nodal, b, stream=None):
        B.sem3_mass(self.h, f_nodal, b, stream)

    def apply(self, u, Au, stream=None):
        B.sem3_apply(self.h, u, Au, stream)

    def smooth(self, u, f, n_it=1, stream=None):
        B.sem3_smooth(self.h, u, f, n_it, stream)

    def vcycle(self, u, f, stream=None):
        B.sem3_vcycle(self.h, u, f, stream)

    def pcg_solve(self, u, f, history_len=0, stream=None):
        return B.sem3_pcg_solve(self.h, u, f, history_len, stream)


def main(argv=None):
    """Solve one seeded random-RHS problem (b = M f, f ~ U[-1, 1] at the GLL
    nodes, u0 = 0) a few times and print one JSON line per solve:

        python -m paper_1512_02390_gb300.solver --nx 64 --ny 64 --p 16 --overlap 2 --precision tf32

    --trace runs every solve launch by launch with CUDA-event tracing (no
    graph replay; what a kernel profiler can attribute), --tune autotunes the
    launch shapes first, --set-tune L:FUSE:SPW:TC fixes level L's shapes."""
    import argparse
    import json

    import torch

    import sem_inputs as SI

    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=64)
    ap.add_argument("--ny", type=int, default=64)
    ap.add_argument("--p", type=int, default=16)
    ap.add_argument("--overlap", type=int, default=2)
    ap.add_argument("--precision", default="tf32", choices=sorted(_PREC))
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--solves", type=int, default=3)
    ap.add_argument("--trace", action="store_true")
    ap.add_argument("--tune", action="store_true")
    ap.add_argument("--tune-cache", default=None,
                    help="with --tune: read the launch shapes from this JSON-lines cache, timing and "
                         "appending only the missing ones")
    ap.add_argument("--set-tune", action="append", default=[])
    ap.add_argument("--batch", type=int, default=0,
                    help="solve the first N problems of the seeded batched workload instead (one batch "
                         "solve per --solves; the first runs launch by launch, later ones replay the graph)")
    a = ap.parse_args(argv)
    if a.batch:
        cfgs = batch_workload(a.batch, precision=a.precision, tol=a.tol)
        shapes = {}
        for c in cfgs:
            key = (c["nx"], c["p"], c["overlap"])
            shapes[key] = shapes.get(key, 0) + 1
        print(json.dumps({"groups": [{"n": k[0], "p": k[1], "n_o": k[2], "problems": v,
                                      "nodes": v * (k[0] * k[1] + 1) ** 2} for k, v in sorted(shapes.items())]}))
        Bt = Batch(cfgs)
        if a.tune:
            Bt.autotune(a.tune_cache)
        us, fs = [], []
        for k, c in enumerate(cfgs):
            n = c["nx"] * c["p"] + 1
            fs.append(torch.from_numpy(SI.uniform_nodal(1000 + k, (n, n)).ravel()).cuda())
            us.append(torch.zeros_like(fs[-1]))
        for k in range(a.solves):
            for u in us:
                u.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            res = Bt.solve(us, fs)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            print(json.dumps({"batch_solve": k, "problems": len(cfgs), "groups": Bt.groups, "unknowns": Bt.unknowns,
                              "converged": sum(1 for r in res if r.status == 0), "ms": round(ms, 3),
                              "dof_per_s": Bt.unknowns / (ms * 1e-3)}))
        Bt.close()
        return
    S = Solver(nx=a.nx, ny=a.ny, p=a.p, overlap=a.overlap, precision=a.precision, tol=a.tol, i_max=500)
    if a.tune:
        S.autotune(a.tune_cache)
    for spec in a.set_tune:
        lvl, fuse, spw, tc = (int(x) for x in spec.split(":"))
        S.set_tune(lvl, fuse, spw, tc)
    fn = torch.from_numpy(SI.uniform_nodal(a.seed, S.shape).ravel()).cuda()
    b = torch.empty_like(fn)
    S.mass(fn, b)
    S.profile(a.trace)
    for k in range(a.solves):
        u = torch.zeros_like(b)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res, _ = S.pcg_solve(u, b)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        print(json.dumps({"solve": k, "iterations": res.iterations, "status": B.status_name(res.status),
                          "rel_res": res.res / res.res0 if res.res0 else 0.0, "ms": round(ms, 4),
                          "dof_per_s": S.n_unknowns / (ms * 1e-3)}))
    if a.trace:
        print(json.dumps({"class_ms_total": {k: round(v[0], 4) for k, v in S.profile_read().items()}}))
    S.close()


if __name__ == "__main__":
    main()
