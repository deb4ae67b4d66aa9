"""ctypes binding of include/sem_schwarz.h: argument marshalling only.

Every function here has the name of the C entry point it forwards to.  Vector
arguments are CUDA float64 torch tensors (or raw device addresses as int);
``stream`` is a torch.cuda.Stream, a raw cudaStream_t as int, or None for the
current torch stream.  There is no CPU fallback: if the compiled library is
missing the first call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsemschwarz.so")

# sem_status
SEM_OK, SEM_NOT_CONVERGED, SEM_BREAKDOWN, SEM_TIMEOUT, SEM_BAD_ARG, SEM_CUDA_ERROR, SEM_OOM = range(7)
# sem_weight
SEM_W_LINEAR, SEM_W_CUBIC, SEM_W_QUINTIC, SEM_W_SEPTIC = 1, 3, 5, 7
SEM_W_TOPHAT, SEM_W_ARITH, SEM_W_IDENTITY, SEM_W_LEARNED = 100, 101, 102, 103
# sem_overlap_rule
SEM_OVERLAP_FIXED, SEM_OVERLAP_FLOOR8, SEM_OVERLAP_CEIL8, SEM_OVERLAP_CEIL2 = range(4)
# sem_precision
SEM_PREC_FP64, SEM_PREC_FP32, SEM_PREC_TF32, SEM_PREC_BF16 = range(4)
# sem_smoother
SEM_SMOOTH_ADDITIVE, SEM_SMOOTH_MULT = range(2)

EXPORTS = [
    "sem_default_config", "sem_create", "sem_destroy", "sem_sizes", "sem_coords", "sem_mass",
    "sem_apply", "sem_smooth", "sem_vcycle", "sem_mg_solve", "sem_pcg_solve",
    "sem_inspect_level", "sem_gll_tables", "sem_profile", "sem_profile_read", "sem_profile_read_level", "sem_schwarz_correction_noalloc",
    "sem_learned_features", "sem_mlp_load", "sem_mlp_forward", "sem_mlp_workspace_bytes", "sem_mlp_loss_grad", "sem_mlp_train",
    "sem_batch_create", "sem_batch_destroy", "sem_batch_info", "sem_batch_solve", "sem_batch_launches",
    "sem_autotune", "sem_get_tune", "sem_set_tune", "sem_batch_autotune", "sem_set_low_cycle", "sem_get_low_cycle",
    "sem_set_fused_prolongation", "sem_get_fused_prolongation", "sem_set_fixed_point_operator",
    "sem_get_fixed_point_operator",
    "sem_status_string", "sem_last_error",
    "sem3_default_config", "sem3_create", "sem3_destroy", "sem3_sizes", "sem3_coords", "sem3_mass", "sem3_apply",
    "sem3_smooth", "sem3_vcycle", "sem3_pcg_solve",
]
SEM_MLP_PARAMS = 4610
# sem_kernel_class
KERNEL_CLASSES = ["apply_fp64", "apply_mg", "sweep", "scatter", "restrict", "prolong", "coarse", "vector",
                  "low_cycle"]


class sem_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("p", ctypes.c_int32), ("periodic", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("x_edges", ctypes.POINTER(ctypes.c_double)), ("y_edges", ctypes.POINTER(ctypes.c_double)),
        ("overlap_rule", ctypes.c_int32), ("overlap", ctypes.c_int32), ("weight", ctypes.c_int32),
        ("ns1", ctypes.c_int32), ("ns2", ctypes.c_int32), ("variable_cycle", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("tol", ctypes.c_double), ("i_max", ctypes.c_int32),
        ("nu_kind", ctypes.c_int32), ("nu_a", ctypes.c_double), ("nu_b", ctypes.c_double),
        ("learned_x", ctypes.POINTER(ctypes.c_double)), ("learned_y", ctypes.POINTER(ctypes.c_double)),
        ("smoother", ctypes.c_int32), ("mlp_params", ctypes.POINTER(ctypes.c_float)),
    ]


class sem3_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("p", ctypes.c_int32),
        ("periodic", ctypes.c_int32), ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("overlap_rule", ctypes.c_int32), ("overlap", ctypes.c_int32), ("weight", ctypes.c_int32),
        ("ns1", ctypes.c_int32), ("ns2", ctypes.c_int32), ("precision", ctypes.c_int32), ("tol", ctypes.c_double),
        ("i_max", ctypes.c_int32),
    ]


class sem_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("status", ctypes.c_int32), ("res0", ctypes.c_double),
                ("res", ctypes.c_double), ("rbar", ctypes.c_double)]


class sem_level_info(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("n_o", ctypes.c_int32), ("m", ctypes.c_int32),
                ("n_tables_x", ctypes.c_int32), ("nx_nodes", ctypes.c_int32)]


class sem_level_tune(ctypes.Structure):
    _fields_ = [("fuse", ctypes.c_int32), ("spw", ctypes.c_int32), ("tc", ctypes.c_int32),
                ("tc_available", ctypes.c_int32), ("eo", ctypes.c_int32), ("us", ctypes.c_double)]


class sem_sweep_tables(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("p", ctypes.c_int32), ("n_o", ctypes.c_int32), ("periodic", ctypes.c_int32),
                ("tab", ctypes.c_void_p), ("S", ctypes.c_void_p), ("lam", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class SemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (status_name(status), msg))
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: build it with `python -m paper_1512_02390_gb300.build` "
                           "(or __graft_entry__.build()); there is no CPU fallback" % path)
    lib = ctypes.CDLL(path)
    vp, i32, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)
    sig = {
        "sem_default_config": (None, [ctypes.POINTER(sem_config)]),
        "sem_create": (i32, [ctypes.POINTER(sem_config), ctypes.POINTER(vp)]),
        "sem_destroy": (None, [vp]),
        "sem_sizes": (i32, [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_int64)]),
        "sem_coords": (i32, [vp, dp, dp]),
        "sem_mass": (i32, [vp, vp, vp, vp]),
        "sem_apply": (i32, [vp, vp, vp, vp]),
        "sem_smooth": (i32, [vp, vp, vp, i32, vp]),
        "sem_vcycle": (i32, [vp, vp, vp, vp]),
        "sem_mg_solve": (i32, [vp, vp, vp, ctypes.POINTER(sem_result), dp, i32, vp]),
        "sem_pcg_solve": (i32, [vp, vp, vp, ctypes.POINTER(sem_result), dp, i32, vp]),
        "sem_inspect_level": (i32, [ctypes.POINTER(sem_config), i32, ctypes.POINTER(sem_level_info),
                                    ctypes.POINTER(ctypes.c_int32), dp, dp, dp, dp]),
        "sem_gll_tables": (i32, [i32, dp, dp, dp, dp]),
        "sem_profile": (i32, [vp, i32]),
        "sem_profile_read": (i32, [vp, dp, ctypes.POINTER(ctypes.c_int64)]),
        "sem_profile_read_level": (i32, [vp, i32, dp, ctypes.POINTER(ctypes.c_int64)]),
        "sem_schwarz_correction_noalloc": (i32, [ctypes.POINTER(sem_sweep_tables), ctypes.POINTER(sem_sweep_tables),
                                                 vp, vp, vp]),
        "sem_learned_features": (i32, [ctypes.POINTER(sem_config), vp, vp]),
        "sem_mlp_load": (i32, [vp, ctypes.POINTER(ctypes.c_float)]),
        "sem_mlp_forward": (i32, [vp, vp, i32, vp, i32, vp]),
        "sem_mlp_workspace_bytes": (ctypes.c_int64, [i32]),
        "sem_mlp_loss_grad": (i32, [vp, vp, vp, i32, vp, vp, vp, vp]),
        "sem_mlp_train": (i32, [vp, vp, vp, vp, vp, i32, i32, ctypes.c_float, i32, vp, vp, vp]),
        "sem_batch_create": (i32, [ctypes.POINTER(sem_config), i32, ctypes.POINTER(vp)]),
        "sem_batch_destroy": (None, [vp]),
        "sem_batch_info": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_int64)]),
        "sem_batch_solve": (i32, [vp, vp, vp, ctypes.POINTER(sem_result), vp]),
        "sem_batch_launches": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "sem_autotune": (i32, [vp, ctypes.c_char_p, vp]),
        "sem_get_tune": (i32, [vp, i32, ctypes.POINTER(sem_level_tune)]),
        "sem_set_tune": (i32, [vp, i32, ctypes.POINTER(sem_level_tune)]),
        "sem_batch_autotune": (i32, [vp, ctypes.c_char_p, vp]),
        "sem_set_low_cycle": (i32, [vp, i32]),
        "sem_get_low_cycle": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "sem_set_fused_prolongation": (i32, [vp, i32]),
        "sem_get_fused_prolongation": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "sem_set_fixed_point_operator": (i32, [vp, i32]),
        "sem_get_fixed_point_operator": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "sem3_default_config": (None, [ctypes.POINTER(sem3_config)]),
        "sem3_create": (i32, [ctypes.POINTER(sem3_config), ctypes.POINTER(vp)]),
        "sem3_destroy": (None, [vp]),
        "sem3_sizes": (i32, [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "sem3_coords": (i32, [vp, dp, dp, dp]),
        "sem3_mass": (i32, [vp, vp, vp, vp]),
        "sem3_apply": (i32, [vp, vp, vp, vp]),
        "sem3_smooth": (i32, [vp, vp, vp, i32, vp]),
        "sem3_vcycle": (i32, [vp, vp, vp, vp]),
        "sem3_pcg_solve": (i32, [vp, vp, vp, ctypes.POINTER(sem_result), dp, i32, vp]),
        "sem_status_string": (ctypes.c_char_p, [i32]),
        "sem_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_name(status: int) -> str:
    return load_library().sem_status_string(int(status)).decode()


def last_error() -> str:
    return load_library().sem_last_error().decode()


def _check(rc: int, allow=(SEM_OK,)):
    if rc not in allow:
        raise SemError(rc, last_error())
    return rc


def _ptr(t, n=None):
    """Device address of a CUDA float64 tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float64 tensor")
    if n is not None and t.numel() != n:
        raise ValueError("tensor has %d elements, the node grid has %d" % (t.numel(), n))
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def sem_default_config() -> sem_config:
    cfg = sem_config()
    load_library().sem_default_config(ctypes.byref(cfg))
    return cfg


def sem_create(cfg: sem_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().sem_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def sem_destroy(h) -> None:
    load_library().sem_destroy(h)


def sem_sizes(h):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().sem_sizes(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def sem_coords(h):
    _, nx, ny = sem_sizes(h)
    x = np.zeros(nx)
    y = np.zeros(ny)
    _check(load_library().sem_coords(h, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     y.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return x, y


def _n(h):
    _, nx, ny = sem_sizes(h)
    return nx * ny


def sem_mass(h, f_nodal, b, stream=None):
    n = _n(h)
    _check(load_library().sem_mass(h, _ptr(f_nodal, n), _ptr(b, n), _stream(stream)))


def sem_apply(h, u, Au, stream=None):
    n = _n(h)
    _check(load_library().sem_apply(h, _ptr(u, n), _ptr(Au, n), _stream(stream)))


def sem_smooth(h, u, f, n_it, stream=None):
    n = _n(h)
    _check(load_library().sem_smooth(h, _ptr(u, n), _ptr(f, n), int(n_it), _stream(stream)))


def sem_vcycle(h, u, f, stream=None):
    n = _n(h)
    _check(load_library().sem_vcycle(h, _ptr(u, n), _ptr(f, n), _stream(stream)))


def _solve(fn, h, u, f, history_len, stream):
    n = _n(h)
    res = sem_result()
    hist = np.zeros(max(0, int(history_len)))
    hp = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if history_len else None
    rc = fn(h, _ptr(u, n), _ptr(f, n), ctypes.byref(res), hp, int(history_len), _stream(stream))
    _check(rc, allow=(SEM_OK, SEM_NOT_CONVERGED, SEM_BREAKDOWN))
    return res, hist[: min(len(hist), res.iterations + 1)]


def sem_mg_solve(h, u, f, history_len=0, stream=None):
    return _solve(load_library().sem_mg_solve, h, u, f, history_len, stream)


def sem_pcg_solve(h, u, f, history_len=0, stream=None):
    return _solve(load_library().sem_pcg_solve, h, u, f, history_len, stream)


def sem_inspect_level(cfg: sem_config, level: int):
    """Host-side set-up tables of one level (x direction); needs no GPU."""
    lib = load_library()
    info = sem_level_info()
    _check(lib.sem_inspect_level(ctypes.byref(cfg), int(level), ctypes.byref(info), None, None, None, None, None))
    nt, m = info.n_tables_x, info.m
    tab = np.zeros(cfg.nx, dtype=np.int32)
    S = np.zeros(nt * m * m)
    lam = np.zeros(nt * m)
    w = np.zeros(nt * m)
    xc = np.zeros(info.nx_nodes)
    d = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib.sem_inspect_level(ctypes.byref(cfg), int(level), ctypes.byref(info),
                                 tab.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), d(S), d(lam), d(w), d(xc)))
    return dict(p=info.p, n_o=info.n_o, m=m, tab=tab, S=S.reshape(nt, m, m), lam=lam.reshape(nt, m),
                w=w.reshape(nt, m), coords=xc)


def sem_gll_tables(p: int):
    """(xi, w, D, L_ref) of order p as the library builds them; needs no GPU."""
    n = int(p) + 1
    xi, w, D, L = np.zeros(n), np.zeros(n), np.zeros((n, n)), np.zeros((n, n))
    d = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(load_library().sem_gll_tables(int(p), d(xi), d(w), d(D), d(L)))
    return xi, w, D, L


def sem_profile(h, enable: bool) -> None:
    _check(load_library().sem_profile(h, int(bool(enable))))


def sem_profile_read(h):
    """{class: (ms, launches)} since the last sem_profile call."""
    n = len(KERNEL_CLASSES)
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    _check(load_library().sem_profile_read(h, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}


def sem_profile_read_level(h, level: int):
    """{class: (ms, launches)} of one V-cycle level since the last sem_profile call."""
    n = len(KERNEL_CLASSES)
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    _check(load_library().sem_profile_read_level(h, int(level), ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}


def sem_schwarz_correction_noalloc(tx: sem_sweep_tables, ty: sem_sweep_tables, r, u, stream=None) -> None:
    """u += sum_s R_s^T W A_ss^{-1} R_s r without any allocation (see the C header for who needs this)."""
    def nodes(t):
        return t.n * t.p + (0 if t.periodic else 1)
    want = nodes(tx) * nodes(ty)
    for name, v in (("r", r), ("u", u)):
        if v.numel() != want:
            raise ValueError("%s has %d entries; the tables describe a %d x %d node grid"
                             % (name, v.numel(), nodes(ty), nodes(tx)))
    _check(load_library().sem_schwarz_correction_noalloc(ctypes.byref(tx), ctypes.byref(ty), _ptr(r), _ptr(u),
                                                         _stream(stream)))


def _fptr(t):
    """Device address of a contiguous CUDA float32 tensor (None passes through)."""
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float32 tensor")
    return t.data_ptr()


def sem_learned_features(cfg: sem_config):
    """Features [level][interface][4] of the x and y interface lines (host)."""
    L = int(np.log2(cfg.p))
    fx = np.zeros((L + 1, cfg.nx + 1, 4), dtype=np.float32)
    fy = np.zeros((L + 1, cfg.ny + 1, 4), dtype=np.float32)
    _check(load_library().sem_learned_features(ctypes.byref(cfg), fx.ctypes.data, fy.ctypes.data))
    return fx, fy


def sem_mlp_load(h, params) -> None:
    """Rebuild the handle's weights from the network parameters (HOST array)."""
    arr = np.ascontiguousarray(params, dtype=np.float32)
    if arr.size != SEM_MLP_PARAMS:
        raise ValueError("expected %d network parameters, got %d" % (SEM_MLP_PARAMS, arr.size))
    _check(load_library().sem_mlp_load(h, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))


def sem_mlp_forward(params, X, Y, transform=True, stream=None):
    _check(load_library().sem_mlp_forward(_fptr(params), _fptr(X), int(X.shape[0]), _fptr(Y), int(bool(transform)),
                                          _stream(stream)))


def sem_mlp_workspace_bytes(n: int) -> int:
    return int(load_library().sem_mlp_workspace_bytes(int(n)))


def sem_mlp_loss_grad(params, X, T, grad, loss, workspace, stream=None):
    _check(load_library().sem_mlp_loss_grad(_fptr(params), _fptr(X), _fptr(T), int(X.shape[0]), _fptr(grad),
                                            _fptr(loss), _fptr(workspace), _stream(stream)))


def sem_mlp_train(params, m, v, X, T, steps, lr, step0, loss_hist, workspace, stream=None):
    _check(load_library().sem_mlp_train(_fptr(params), _fptr(m), _fptr(v), _fptr(X), _fptr(T), int(X.shape[0]),
                                        int(steps), float(lr), int(step0), _fptr(loss_hist), _fptr(workspace),
                                        _stream(stream)))


def sem_batch_create(cfgs):
    arr = (sem_config * len(cfgs))(*cfgs)
    h = ctypes.c_void_p()
    _check(load_library().sem_batch_create(arr, len(cfgs), ctypes.byref(h)))
    return h


def sem_batch_destroy(b) -> None:
    load_library().sem_batch_destroy(b)


def sem_batch_info(b):
    g, u = ctypes.c_int32(), ctypes.c_int64()
    _check(load_library().sem_batch_info(b, ctypes.byref(g), ctypes.byref(u)))
    return g.value, u.value


def sem_batch_solve(b, us, fs, stream=None):
    n = len(us)
    up = (ctypes.c_void_p * n)(*[_ptr(x) for x in us])
    fp = (ctypes.c_void_p * n)(*[_ptr(x) for x in fs])
    res = (sem_result * n)()
    rc = load_library().sem_batch_solve(b, up, fp, res, _stream(stream))
    _check(rc, allow=(SEM_OK, SEM_NOT_CONVERGED, SEM_BREAKDOWN))
    return list(res)


def sem_batch_launches(b) -> int:
    v = ctypes.c_int64()
    _check(load_library().sem_batch_launches(b, ctypes.byref(v)))
    return v.value


def _path_arg(path):
    return None if path is None else os.fsencode(path)


def sem_autotune(h, cache_path=None, stream=None) -> None:
    """Time the launch-shape candidates of every level (or read them from the cache file)."""
    _check(load_library().sem_autotune(h, _path_arg(cache_path), _stream(stream)))


def sem_get_tune(h, level: int):
    """dict(fuse, spw, tc, tc_available, us) of level `level` (1..log2 p)."""
    t = sem_level_tune()
    _check(load_library().sem_get_tune(h, int(level), ctypes.byref(t)))
    return dict(fuse=t.fuse, spw=t.spw, tc=t.tc, tc_available=t.tc_available, eo=t.eo, us=t.us)


def sem_set_tune(h, level: int, fuse: int, spw: int = 1, tc: int = 0, eo: int = -1) -> None:
    t = sem_level_tune(int(fuse), int(spw), int(tc), 0, int(eo), 0.0)
    _check(load_library().sem_set_tune(h, int(level), ctypes.byref(t)))


def sem_batch_autotune(b, cache_path=None, stream=None) -> None:
    _check(load_library().sem_batch_autotune(b, _path_arg(cache_path), _stream(stream)))


def sem_set_low_cycle(h, enable: bool) -> None:
    _check(load_library().sem_set_low_cycle(h, int(bool(enable))))


def sem_get_low_cycle(h):
    """(available, enabled) of the persistent low-level cycle."""
    a, e = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().sem_get_low_cycle(h, ctypes.byref(a), ctypes.byref(e)))
    return bool(a.value), bool(e.value)


def sem_set_fused_prolongation(h, enable: bool) -> None:
    _check(load_library().sem_set_fused_prolongation(h, int(bool(enable))))


def sem_get_fused_prolongation(h):
    """(available, enabled) of the one-launch up-leg of the V-cycle."""
    a, e = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().sem_get_fused_prolongation(h, ctypes.byref(a), ctypes.byref(e)))
    return bool(a.value), bool(e.value)


def sem_set_fixed_point_operator(h, enable: bool) -> None:
    _check(load_library().sem_set_fixed_point_operator(h, int(bool(enable))))


def sem_get_fixed_point_operator(h):
    """(available, enabled) of the FP64 operator in exact integer arithmetic."""
    a, e = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().sem_get_fixed_point_operator(h, ctypes.byref(a), ctypes.byref(e)))
    return bool(a.value), bool(e.value)



# ---- three-dimensional extension (include/sem_schwarz3d.h) ---------------------

def sem3_default_config() -> sem3_config:
    cfg = sem3_config()
    load_library().sem3_default_config(ctypes.byref(cfg))
    return cfg


def sem3_create(cfg: sem3_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().sem3_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def sem3_destroy(h) -> None:
    load_library().sem3_destroy(h)


def sem3_sizes(h):
    v = [ctypes.c_int64() for _ in range(4)]
    _check(load_library().sem3_sizes(h, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def sem3_coords(h):
    _, nx, ny, nz = sem3_sizes(h)
    x, y, z = np.zeros(nx), np.zeros(ny), np.zeros(nz)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load_library().sem3_coords(h, x.ctypes.data_as(dp), y.ctypes.data_as(dp), z.ctypes.data_as(dp)))
    return x, y, z


def sem3_mass(h, f_nodal, b, stream=None) -> None:
    _check(load_library().sem3_mass(h, _ptr(f_nodal), _ptr(b), _stream(stream)))


def sem3_apply(h, u, Au, stream=None) -> None:
    _check(load_library().sem3_apply(h, _ptr(u), _ptr(Au), _stream(stream)))


def sem3_smooth(h, u, f, n_it=1, stream=None) -> None:
    _check(load_library().sem3_smooth(h, _ptr(u), _ptr(f), int(n_it), _stream(stream)))


def sem3_vcycle(h, u, f, stream=None) -> None:
    _check(load_library().sem3_vcycle(h, _ptr(u), _ptr(f), _stream(stream)))


def sem3_pcg_solve(h, u, f, history_len=0, stream=None):
    """(sem_result, residual norms) of Alg. 4 in 3D; non-OK statuses are returned, not raised."""
    res = sem_result()
    hist = np.zeros(max(1, history_len))
    rc = load_library().sem3_pcg_solve(h, _ptr(u), _ptr(f), ctypes.byref(res),
                                       hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if history_len else None,
                                       int(history_len), _stream(stream))
    _check(rc, allow=(SEM_OK, SEM_NOT_CONVERGED, SEM_BREAKDOWN))
    return res, hist[:res.iterations + 1] if history_len else None
