"""Thin ctypes binding of libnbody.so (C ABI in include/nbody.h).

Argument marshalling only: every function here checks dtypes/sizes, turns
torch tensors (device or host) or numpy arrays into raw pointers, calls the C
entry point of the same name and raises NbodyError on a non-OK status.  No
step of the computation runs in Python, and there is no CPU fallback: if the
CUDA library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

NBODY_OK, NBODY_EINVAL, NBODY_ENOMEM, NBODY_EOVERFLOW, NBODY_ETIMEOUT, NBODY_ECUDA, \
    NBODY_ENOTBUILT = range(7)
SCHED_MORTON, SCHED_MLP, SCHED_LASTCOST = 0, 1, 2
_STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "EOVERFLOW", 4: "ETIMEOUT", 5: "ECUDA",
                 6: "ENOTBUILT"}


class NbodyError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("G", C.c_float), ("eps", C.c_float), ("delta_acc", C.c_float),
                ("theta", C.c_float), ("leaf_cap", C.c_int32), ("group_size", C.c_int32),
                ("ipl", C.c_int32), ("list_depth", C.c_int32), ("stack_depth", C.c_int32),
                ("warps_per_block", C.c_int32), ("compensated", C.c_int32),
                ("want_potential", C.c_int32), ("schedule", C.c_int32),
                ("use_graph", C.c_int32), ("rebuild_interval", C.c_int32),
                ("quadrupole", C.c_int32), ("block_levels", C.c_int32),
                ("block_eta", C.c_float), ("walk_pipeline", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneSpace(C.Structure):
    _fields_ = [("n_leaf_cap", C.c_int32), ("leaf_cap", C.c_int32 * 4),
                ("n_group_size", C.c_int32), ("group_size", C.c_int32 * 6),
                ("n_ipl", C.c_int32), ("ipl", C.c_int32 * 3),
                ("n_list_depth", C.c_int32), ("list_depth", C.c_int32 * 4),
                ("n_warps_per_block", C.c_int32), ("warps_per_block", C.c_int32 * 4),
                ("repeats", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_groups", C.c_int64), ("interactions", C.c_int64),
                ("list_entries", C.c_int64), ("max_stack", C.c_int32), ("levels", C.c_int32),
                ("kernels", C.c_int64), ("ms_build", C.c_float), ("ms_walk", C.c_float),
                ("ms_walk_kernel", C.c_float), ("walk_launches", C.c_int32),
                ("rebuilds", C.c_int32), ("quad_interactions", C.c_int64),
                ("walk_warps", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()
EXPORTS = ("nbody_abi_version", "nbody_config_default", "nbody_create", "nbody_destroy",
           "nbody_set_config", "nbody_get_config", "nbody_build", "nbody_build_batched",
           "nbody_walk", "nbody_direct", "nbody_step", "nbody_step_batched", "nbody_diagnostics",
           "nbody_get_group_costs", "nbody_export", "nbody_last_error",
           "nbody_diagnostics_noalloc", "nbody_tune_space_default", "nbody_autotune",
           "nbody_mlp_set_params", "nbody_mlp_get_params", "nbody_mlp_train",
           "nbody_mlp_predict", "nbody_mlp_eval", "nbody_selftest",
           "nbody_refit", "nbody_rebuild_due", "nbody_sort_keys")
MLP_PARAMS, MLP_FEATURES = 1377, 8
EXPORT_PERM, EXPORT_KEYS, EXPORT_NODE_LEVEL, EXPORT_NODE_START, EXPORT_NODE_COUNT, \
    EXPORT_NODE_PARENT, EXPORT_NODE_A, EXPORT_NODE_B, EXPORT_GROUP_FIRST, EXPORT_GROUP_COUNT, \
    EXPORT_GROUP_SPHERE, EXPORT_SYS_BOX, EXPORT_NODE_Q = range(13)
_EXPORT_DTYPE = {0: (np.int32, 1), 1: (np.uint64, 1), 2: (np.int8, 1), 3: (np.int32, 1),
                 4: (np.int32, 1), 5: (np.int32, 1), 6: (np.float32, 4), 7: (np.float32, 4),
                 8: (np.int32, 1), 9: (np.int32, 1), 10: (np.float32, 4), 11: (np.float32, 4),
                 12: (np.float32, 8)}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libnbody.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and _build.stale():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise NbodyError(NBODY_ECUDA, f"CUDA library not found at {_build.LIB}")
        lib = C.CDLL(_build.LIB)
        vp, i64, i32, f32 = C.c_void_p, C.c_int64, C.c_int32, C.c_float
        st = C.c_int
        sig = {
            "nbody_abi_version": (C.c_int32, []),
            "nbody_config_default": (None, [C.POINTER(Config)]),
            "nbody_create": (st, [C.POINTER(vp), C.POINTER(Config), vp]),
            "nbody_destroy": (st, [vp]),
            "nbody_set_config": (st, [vp, C.POINTER(Config)]),
            "nbody_get_config": (st, [vp, C.POINTER(Config)]),
            "nbody_build": (st, [vp, i64, vp, vp, vp, vp]),
            "nbody_build_batched": (st, [vp, i32, vp, vp, vp, vp, vp, vp]),
            "nbody_walk": (st, [vp, vp, vp, vp, vp, vp, C.POINTER(Stats)]),
            "nbody_direct": (st, [i64, vp, vp, vp, vp, f32, f32, i32, vp, vp, vp, vp, vp]),
            "nbody_step": (st, [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, f32, i32,
                                C.POINTER(Stats)]),
            "nbody_step_batched": (st, [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                        f32, i32, C.POINTER(Stats)]),
            "nbody_diagnostics": (st, [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "nbody_diagnostics_noalloc": (st, [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "nbody_get_group_costs": (st, [vp, vp, i64, C.POINTER(i64)]),
            "nbody_export": (st, [vp, i32, vp, i64, C.POINTER(i64)]),
            "nbody_tune_space_default": (None, [C.POINTER(TuneSpace)]),
            "nbody_mlp_set_params": (st, [vp, vp]),
            "nbody_mlp_get_params": (st, [vp, vp]),
            "nbody_mlp_train": (st, [vp, i32, f32, i32, C.POINTER(f32)]),
            "nbody_mlp_predict": (st, [vp, vp, vp, i64, C.POINTER(i64)]),
            "nbody_mlp_eval": (st, [i64, vp, vp, vp, vp, vp, vp, vp, vp]),
            "nbody_autotune": (st, [vp, i32, vp, vp, vp, vp, vp, vp, vp, C.POINTER(TuneSpace),
                                    C.POINTER(Config), C.POINTER(f32), C.POINTER(i32)]),
            "nbody_selftest": (st, [i32, vp]),
            "nbody_sort_keys": (st, [vp, i32, vp, i64, vp, vp]),
            "nbody_refit": (st, [vp, vp, vp, vp, vp]),
            "nbody_rebuild_due": (i32, [C.POINTER(f32), i32]),
            "nbody_last_error": (st, [vp, C.c_char_p, C.c_size_t]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


# ---------------------------------------------------------------- marshalling
def _ptr(a, dtype: str, n=None, name="array", allow_none=False):
    """Raw pointer of a contiguous torch tensor or numpy array of `dtype`."""
    if a is None:
        if allow_none:
            return None
        raise NbodyError(NBODY_EINVAL, f"{name} is None")
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"]:
            raise NbodyError(NBODY_EINVAL, f"{name} must be a contiguous {dtype} array")
        if n is not None and a.size != n:
            raise NbodyError(NBODY_EINVAL, f"{name} has {a.size} elements, expected {n}")
        return a.ctypes.data
    import torch
    if not isinstance(a, torch.Tensor):
        raise NbodyError(NBODY_EINVAL, f"{name} must be a torch tensor or numpy array")
    want = {"float32": torch.float32, "float64": torch.float64, "int64": torch.int64,
            "int32": torch.int32}[dtype]
    if a.dtype != want or not a.is_contiguous():
        raise NbodyError(NBODY_EINVAL, f"{name} must be a contiguous {dtype} tensor")
    if n is not None and a.numel() != n:
        raise NbodyError(NBODY_EINVAL, f"{name} has {a.numel()} elements, expected {n}")
    return a.data_ptr()


def _size(a):
    return int(a.size if isinstance(a, np.ndarray) else a.numel())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _check(lib, ctx, status):
    if status != NBODY_OK:
        buf = C.create_string_buffer(512)
        lib.nbody_last_error(ctx, buf, 512)
        raise NbodyError(status, buf.value.decode(errors="replace"))


# ---------------------------------------------------------------- entry points
def nbody_abi_version() -> int:
    return int(load().nbody_abi_version())


def nbody_config_default(**overrides) -> Config:
    cfg = Config()
    load().nbody_config_default(C.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise NbodyError(NBODY_EINVAL, f"unknown config field {k}")
        setattr(cfg, k, v)
    return cfg


def nbody_create(cfg: Config | None = None, stream=None):
    """Returns an opaque context handle (c_void_p)."""
    lib = load()
    h = C.c_void_p()
    _check(lib, None, lib.nbody_create(C.byref(h), C.byref(cfg) if cfg is not None else None,
                                       _stream_ptr(stream)))
    return h


def nbody_destroy(ctx):
    lib = load()
    _check(lib, None, lib.nbody_destroy(ctx))


def nbody_set_config(ctx, cfg: Config):
    lib = load()
    _check(lib, ctx, lib.nbody_set_config(ctx, C.byref(cfg)))


def nbody_get_config(ctx) -> Config:
    lib = load()
    cfg = Config()
    _check(lib, ctx, lib.nbody_get_config(ctx, C.byref(cfg)))
    return cfg


def nbody_build(ctx, x, y, z, m):
    lib = load()
    n = _size(x)
    ps = [_ptr(a, "float32", n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (m, "m"))]
    _check(lib, ctx, lib.nbody_build(ctx, n, *ps))


def nbody_build_batched(ctx, offsets, eps_sys, x, y, z, m):
    """offsets: host int64 [nsys+1]; eps_sys: host float32 [nsys] or None."""
    lib = load()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nsys = off.size - 1
    eps = None if eps_sys is None else np.ascontiguousarray(eps_sys, dtype=np.float32)
    if eps is not None and eps.size != nsys:
        raise NbodyError(NBODY_EINVAL, "eps_sys must have nsys entries")
    n = int(off[-1])
    ps = [_ptr(a, "float32", n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (m, "m"))]
    _check(lib, ctx, lib.nbody_build_batched(ctx, nsys, off.ctypes.data,
                                             None if eps is None else eps.ctypes.data, *ps))


def nbody_walk(ctx, a_old, ax, ay, az, phi=None) -> Stats:
    lib = load()
    n = _size(ax)
    st = Stats()
    _check(lib, ctx, lib.nbody_walk(ctx, _ptr(a_old, "float32", n, "a_old", True),
                                    _ptr(ax, "float32", n, "ax"), _ptr(ay, "float32", n, "ay"),
                                    _ptr(az, "float32", n, "az"),
                                    _ptr(phi, "float32", n, "phi", True), C.byref(st)))
    return st


def nbody_direct(x, y, z, m, G, eps, compensated, ax, ay, az, phi=None, stream=None):
    lib = load()
    n = _size(x)
    ps = [_ptr(a, "float32", n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (m, "m"))]
    _check(lib, None, lib.nbody_direct(n, *ps, float(G), float(eps), int(compensated),
                                       _ptr(ax, "float32", n, "ax"), _ptr(ay, "float32", n, "ay"),
                                       _ptr(az, "float32", n, "az"),
                                       _ptr(phi, "float32", n, "phi", True), _stream_ptr(stream)))


def nbody_step(ctx, x, y, z, vx, vy, vz, m, ax, ay, az, dt, nsteps) -> Stats:
    lib = load()
    n = _size(x)
    st = Stats()
    d = [_ptr(a, "float64", n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"))]
    f = [_ptr(a, "float32", n, nm) for a, nm in ((vx, "vx"), (vy, "vy"), (vz, "vz"), (m, "m"),
                                                 (ax, "ax"), (ay, "ay"), (az, "az"))]
    _check(lib, ctx, lib.nbody_step(ctx, n, *d, *f, float(dt), int(nsteps), C.byref(st)))
    return st


def nbody_step_batched(ctx, offsets, eps_sys, x, y, z, vx, vy, vz, m, ax, ay, az, dt,
                       nsteps) -> Stats:
    lib = load()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nsys = off.size - 1
    eps = None if eps_sys is None else np.ascontiguousarray(eps_sys, dtype=np.float32)
    n = int(off[-1])
    st = Stats()
    d = [_ptr(a, "float64", n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"))]
    f = [_ptr(a, "float32", n, nm) for a, nm in ((vx, "vx"), (vy, "vy"), (vz, "vz"), (m, "m"),
                                                 (ax, "ax"), (ay, "ay"), (az, "az"))]
    _check(lib, ctx, lib.nbody_step_batched(ctx, nsys, off.ctypes.data,
                                            None if eps is None else eps.ctypes.data, *d, *f,
                                            float(dt), int(nsteps), C.byref(st)))
    return st


def nbody_diagnostics(ctx, x, y, z, vx, vy, vz, m, phi=None) -> np.ndarray:
    lib = load()
    n = _size(x)
    out = np.zeros(8, np.float64)
    d = [_ptr(a, "float64", n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"))]
    f = [_ptr(a, "float32", n, nm) for a, nm in ((vx, "vx"), (vy, "vy"), (vz, "vz"), (m, "m"))]
    _check(lib, ctx, lib.nbody_diagnostics(ctx, n, *d, *f, _ptr(phi, "float32", n, "phi", True),
                                           out.ctypes.data))
    return out


def nbody_diagnostics_noalloc(x, y, z, vx, vy, vz, m, phi=None, out=None,
                              stream=None) -> np.ndarray:
    """FP64 diagnostics computed in the library's fixed scratch array, with no
    device allocation; inputs must be device tensors.  `out` (8 doubles) may
    be a device tensor or None (then a host array is returned)."""
    lib = load()
    n = _size(x)
    res = np.zeros(8, np.float64) if out is None else out
    d = [_ptr(a, "float64", n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"))]
    f = [_ptr(a, "float32", n, nm) for a, nm in ((vx, "vx"), (vy, "vy"), (vz, "vz"), (m, "m"))]
    _check(lib, None, lib.nbody_diagnostics_noalloc(n, *d, *f, _ptr(phi, "float32", n, "phi", True),
                                                    _ptr(res, "float64", 8, "out"),
                                                    _stream_ptr(stream)))
    return res


def nbody_get_group_costs(ctx, counts) -> int:
    lib = load()
    ng = C.c_int64()
    _check(lib, ctx, lib.nbody_get_group_costs(ctx, _ptr(counts, "int32", None, "counts"),
                                               _size(counts), C.byref(ng)))
    return int(ng.value)


def nbody_tune_space_default(**overrides) -> TuneSpace:
    """Default autotuner space; overrides are lists, e.g. ipl=[1, 2]."""
    sp = TuneSpace()
    load().nbody_tune_space_default(C.byref(sp))
    for k, v in overrides.items():
        if k == "repeats":
            sp.repeats = int(v)
            continue
        arr = getattr(sp, k)
        if len(v) > len(arr):
            raise NbodyError(NBODY_EINVAL, f"at most {len(arr)} values for {k}")
        for i, x in enumerate(v):
            arr[i] = int(x)
        setattr(sp, "n_" + k, len(v))
    return sp


def nbody_autotune(ctx, offsets, eps_sys, x, y, z, m, a_old=None, space=None):
    """Grid search; returns (best Config, best build+walk ms, candidates timed)."""
    lib = load()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nsys = off.size - 1
    eps = None if eps_sys is None else np.ascontiguousarray(eps_sys, dtype=np.float32)
    n = int(off[-1])
    ps = [_ptr(a, "float32", n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (m, "m"))]
    best, ms, tried = Config(), C.c_float(), C.c_int32()
    _check(lib, ctx, lib.nbody_autotune(ctx, nsys, off.ctypes.data,
                                        None if eps is None else eps.ctypes.data, *ps,
                                        _ptr(a_old, "float32", n, "a_old", True),
                                        C.byref(space) if space is not None else None,
                                        C.byref(best), C.byref(ms), C.byref(tried)))
    return best, float(ms.value), int(tried.value)


def nbody_mlp_set_params(ctx, params):
    lib = load()
    _check(lib, ctx, lib.nbody_mlp_set_params(ctx, _ptr(params, "float32", MLP_PARAMS, "params")))


def nbody_mlp_get_params(ctx) -> np.ndarray:
    lib = load()
    out = np.empty(MLP_PARAMS, np.float32)
    _check(lib, ctx, lib.nbody_mlp_get_params(ctx, out.ctypes.data))
    return out


def nbody_mlp_train(ctx, epochs=1, lr=1e-3, batch=4096) -> float:
    lib = load()
    loss = C.c_float()
    _check(lib, ctx, lib.nbody_mlp_train(ctx, int(epochs), float(lr), int(batch), C.byref(loss)))
    return float(loss.value)


def nbody_mlp_predict(ctx, want_features=False):
    """(predicted log2 cost per group, features or None) of the last build."""
    lib = load()
    ng = C.c_int64()
    _check(lib, ctx, lib.nbody_mlp_predict(ctx, None, None, 0, C.byref(ng)))
    pred = np.empty(ng.value, np.float32)
    feat = np.empty((ng.value, MLP_FEATURES), np.float32) if want_features else None
    _check(lib, ctx, lib.nbody_mlp_predict(ctx, pred.ctypes.data if pred.size else None,
                                           feat.ctypes.data if feat is not None and pred.size else None,
                                           ng.value, C.byref(ng)))
    return pred, feat


def nbody_mlp_eval(features, targets, params, norm=None, stream=None):
    """Stateless forward/loss/gradient: returns (pred, grad, loss)."""
    lib = load()
    n = _size(targets)
    pred = np.empty(n, np.float32)
    grad = np.empty(MLP_PARAMS, np.float32)
    loss = np.empty(1, np.float32)
    _check(lib, None, lib.nbody_mlp_eval(n, _ptr(features, "float32", n * MLP_FEATURES, "features"),
                                         _ptr(targets, "float32", n, "targets"),
                                         _ptr(params, "float32", MLP_PARAMS, "params"),
                                         _ptr(norm, "float32", 16, "norm", True),
                                         pred.ctypes.data, grad.ctypes.data, loss.ctypes.data,
                                         _stream_ptr(stream)))
    return pred, grad, float(loss[0])


def nbody_export(ctx, what: int) -> np.ndarray:
    """Host copy of an internal array of the last build (see nbody_export_what)."""
    lib = load()
    cnt = C.c_int64()
    _check(lib, ctx, lib.nbody_export(ctx, int(what), None, 0, C.byref(cnt)))
    dt, width = _EXPORT_DTYPE[int(what)]
    out = np.empty(cnt.value * width, dt)
    _check(lib, ctx, lib.nbody_export(ctx, int(what), out.ctypes.data if out.size else None,
                                      cnt.value, C.byref(cnt)))
    return out.reshape(-1, width) if width > 1 else out


def nbody_refit(ctx, x, y, z, m):
    """Refit the last build's tree to new positions of the same particles."""
    lib = load()
    n = _size(x)
    ps = [_ptr(a, "float32", n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (m, "m"))]
    _check(lib, ctx, lib.nbody_refit(ctx, *ps))


def nbody_rebuild_due(cost_ms) -> bool:
    """Host-only rebuild policy of rebuild_interval = 0 (see nbody.h)."""
    a = np.ascontiguousarray(cost_ms, dtype=np.float32)
    return bool(load().nbody_rebuild_due(a.ctypes.data_as(C.POINTER(C.c_float)), a.size))


SELFTEST_SORT_WAIT = 1
SORT_RADIX, SORT_NEAR_ORDER = 0, 1


def nbody_sort_keys(ctx, method, keys, keys_out, perm_out) -> None:
    """Stable sort of 64-bit keys on the context's device (the tree build's
    ordering step): keys, keys_out int64 CUDA tensors [n] holding the key
    bits (compared as unsigned), perm_out int32 [n] (input index of each
    sorted key).  method: SORT_RADIX or SORT_NEAR_ORDER."""
    lib = load()
    n = _size(keys)
    _check(lib, ctx, lib.nbody_sort_keys(ctx, int(method), _ptr(keys, "int64", None, "keys"), n,
                                         _ptr(keys_out, "int64", n, "keys_out"),
                                         _ptr(perm_out, "int32", n, "perm_out")))




def nbody_selftest(which, stream=None) -> int:
    """Runs a self-test of a failure path; returns the status it produced
    (NBODY_ETIMEOUT for SELFTEST_SORT_WAIT when the wait bound works)."""
    return int(load().nbody_selftest(int(which), _stream_ptr(stream)))


def nbody_last_error(ctx=None) -> str:
    lib = load()
    buf = C.create_string_buffer(512)
    lib.nbody_last_error(ctx, buf, 512)
    return buf.value.decode(errors="replace")
