"""FP64 CPU oracle for the gravitational octree method -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The CUDA library and its Python
binding never import it; the two implementations share no code.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over targets).
This module compiles it with gcc on first use (``build()``) and wraps it with
ctypes, taking numpy arrays and returning numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAC_PARTICLE_ACC, MAC_GROUP_ACC, MAC_PARTICLE_GEO, MAC_GROUP_GEO = 0, 1, 2, 3
QUADRUPOLE = 16  # or-ed into a MAC mode: accepted nodes add their quadrupole


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, no fast-math, no FP contraction)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB)
        d, i64, f32, u32, u64, i32 = (C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_float), C.POINTER(C.c_uint32),
                                      C.POINTER(C.c_uint64), C.POINTER(C.c_int32))
        lib.oracle_direct.argtypes = [C.c_int64, d, d, d, d, C.c_double, C.c_double, d, d, d, d]
        lib.oracle_direct_targets.argtypes = [C.c_int64, d, d, d, d, C.c_int64, i64, C.c_double,
                                              C.c_double, d, d, d, d]
        lib.oracle_cube.argtypes = [C.c_int64, f32, f32, f32, f32]
        lib.oracle_cells.argtypes = [C.c_int64, f32, f32, f32, f32, C.c_int, u32, u32, u32]
        lib.oracle_interleave.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_int]
        lib.oracle_interleave.restype = C.c_uint64
        lib.oracle_sort.argtypes = [C.c_int64, u64, i64]
        lib.oracle_tree_build.argtypes = [C.c_int64, d, d, d, d, C.c_int, C.c_int]
        lib.oracle_tree_build.restype = C.c_void_p
        lib.oracle_tree_free.argtypes = [C.c_void_p]
        lib.oracle_tree_refit.argtypes = [C.c_void_p, d, d, d]
        lib.oracle_tree_quadrupoles.argtypes = [C.c_void_p, d]
        lib.oracle_tree_nnodes.argtypes = [C.c_void_p]
        lib.oracle_tree_nnodes.restype = C.c_int64
        lib.oracle_tree_cube.argtypes = [C.c_void_p, f32]
        lib.oracle_tree_nodes.argtypes = [C.c_void_p, i32, u64, i64, i64, i32, i64, d, d, d, d, d]
        lib.oracle_tree_order.argtypes = [C.c_void_p, i64]
        lib.oracle_tree_groups.argtypes = [C.c_void_p, C.c_int, i64, i64]
        lib.oracle_tree_groups.restype = C.c_int64
        lib.oracle_tree_walk.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_int, d, d, d, d, d, i64]
        lib.oracle_tree_walk_groups.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double,
                                                C.c_double, C.c_double, C.c_int, d, C.c_int64,
                                                i64, d, d, d, d, i64]
        lib.oracle_kick.argtypes = [C.c_int64, d, d, d, d, d, d, C.c_double]
        lib.oracle_drift.argtypes = [C.c_int64, d, d, d, d, d, d, C.c_double]
        lib.oracle_diagnostics.argtypes = [C.c_int64, d, d, d, d, d, d, d, d, d]
        lib.oracle_threads.restype = C.c_int
        lib.oracle_set_threads.argtypes = [C.c_int]
        lib.oracle_mlp_params.restype = C.c_int
        lib.oracle_mlp_eval.argtypes = [C.c_int64, d, d, d, d, d, d, d]
        _lib = lib
        return lib


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def set_threads(k: int) -> None:
    """Threads of later oracle calls (k < 1: all cores)."""
    _load().oracle_set_threads(int(k))


def threads() -> int:
    return int(_load().oracle_threads())


# ---------------------------------------------------------------------------
def direct(x, y, z, m, G=1.0, eps=0.0, want_phi=True):
    """Eq. 1 by direct summation in FP64.  Returns (ax, ay, az, phi|None)."""
    lib = _load()
    x, y, z, m = _f64(x), _f64(y), _f64(z), _f64(m)
    n = x.size
    ax, ay, az = np.empty(n), np.empty(n), np.empty(n)
    phi = np.empty(n) if want_phi else None
    lib.oracle_direct(n, _p(x, C.c_double), _p(y, C.c_double), _p(z, C.c_double),
                      _p(m, C.c_double), G, eps, _p(ax, C.c_double), _p(ay, C.c_double),
                      _p(az, C.c_double), _p(phi, C.c_double))
    return ax, ay, az, phi


def direct_targets(x, y, z, m, targets, G=1.0, eps=0.0, want_phi=False):
    """Eq. 1 for the given target indices against all sources."""
    lib = _load()
    x, y, z, m = _f64(x), _f64(y), _f64(z), _f64(m)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    nt = t.size
    ax, ay, az = np.empty(nt), np.empty(nt), np.empty(nt)
    phi = np.empty(nt) if want_phi else None
    lib.oracle_direct_targets(x.size, _p(x, C.c_double), _p(y, C.c_double), _p(z, C.c_double),
                              _p(m, C.c_double), nt, _p(t, C.c_int64), G, eps,
                              _p(ax, C.c_double), _p(ay, C.c_double), _p(az, C.c_double),
                              _p(phi, C.c_double))
    return ax, ay, az, phi


def cube(x, y, z):
    lib = _load()
    x, y, z = _f32(x), _f32(y), _f32(z)
    out = np.empty(4, np.float32)
    lib.oracle_cube(x.size, _p(x, C.c_float), _p(y, C.c_float), _p(z, C.c_float),
                    _p(out, C.c_float))
    return out


def cells(x, y, z, cube_, levels):
    lib = _load()
    x, y, z = _f32(x), _f32(y), _f32(z)
    cube_ = _f32(cube_)
    n = x.size
    q = [np.empty(n, np.uint32) for _ in range(3)]
    lib.oracle_cells(n, _p(x, C.c_float), _p(y, C.c_float), _p(z, C.c_float),
                     _p(cube_, C.c_float), levels, *[_p(a, C.c_uint32) for a in q])
    return q


def interleave(qx, qy, qz, levels):
    lib = _load()
    return np.array([lib.oracle_interleave(int(a), int(b), int(c), levels)
                     for a, b, c in zip(qx, qy, qz)], dtype=np.uint64)


def keys(x, y, z, levels=21, cube_=None):
    """Morton keys of the particles (cube from the particles unless given)."""
    if cube_ is None:
        cube_ = cube(x, y, z)
    qx, qy, qz = cells(x, y, z, cube_, levels)
    return interleave(qx, qy, qz, levels), cube_


def sort_order(k):
    lib = _load()
    k = np.ascontiguousarray(k, dtype=np.uint64)
    order = np.empty(k.size, np.int64)
    lib.oracle_sort(k.size, _p(k, C.c_uint64), _p(order, C.c_int64))
    return order


class Tree:
    """Octree built by recursive subdivision (FP64 moments)."""

    def __init__(self, x, y, z, m, levels=21, leaf_cap=16):
        self._lib = _load()
        self._x, self._y, self._z, self._m = _f64(x), _f64(y), _f64(z), _f64(m)
        self.n = self._x.size
        self.levels, self.leaf_cap = levels, leaf_cap
        self._h = self._lib.oracle_tree_build(self.n, _p(self._x, C.c_double),
                                              _p(self._y, C.c_double), _p(self._z, C.c_double),
                                              _p(self._m, C.c_double), levels, leaf_cap)
        if not self._h:
            raise MemoryError("oracle_tree_build failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_tree_free(h)
            self._h = None

    @property
    def nnodes(self):
        return int(self._lib.oracle_tree_nnodes(self._h))

    def cube(self):
        out = np.empty(4, np.float32)
        self._lib.oracle_tree_cube(self._h, _p(out, C.c_float))
        return out

    def nodes(self):
        nn = self.nnodes
        o = dict(level=np.empty(nn, np.int32), prefix=np.empty(nn, np.uint64),
                 first=np.empty(nn, np.int64), count=np.empty(nn, np.int64),
                 nchild=np.empty(nn, np.int32), child=np.empty(nn, np.int64),
                 cx=np.empty(nn), cy=np.empty(nn), cz=np.empty(nn), M=np.empty(nn), b=np.empty(nn))
        self._lib.oracle_tree_nodes(self._h, _p(o["level"], C.c_int32), _p(o["prefix"], C.c_uint64),
                                    _p(o["first"], C.c_int64), _p(o["count"], C.c_int64),
                                    _p(o["nchild"], C.c_int32), _p(o["child"], C.c_int64),
                                    _p(o["cx"], C.c_double), _p(o["cy"], C.c_double),
                                    _p(o["cz"], C.c_double), _p(o["M"], C.c_double),
                                    _p(o["b"], C.c_double))
        return o

    def quadrupoles(self):
        """Traceless quadrupole of every node, shape (nodes, 6): xx, yy, zz, xy, xz, yz."""
        out = np.empty((self.nnodes, 6))
        self._lib.oracle_tree_quadrupoles(self._h, _p(out, C.c_double))
        return out

    def order(self):
        out = np.empty(self.n, np.int64)
        self._lib.oracle_tree_order(self._h, _p(out, C.c_int64))
        return out

    def groups(self, group_size):
        f = np.empty(self.n, np.int64)
        c = np.empty(self.n, np.int64)
        ng = self._lib.oracle_tree_groups(self._h, group_size, _p(f, C.c_int64), _p(c, C.c_int64))
        return f[:ng].copy(), c[:ng].copy()

    def refit(self, x, y, z):
        """Replace the positions (same particles, caller order) and recompute
        the node moments on the same tree (no rebuild)."""
        self._x, self._y, self._z = _f64(x), _f64(y), _f64(z)
        self._lib.oracle_tree_refit(self._h, _p(self._x, C.c_double), _p(self._y, C.c_double),
                                    _p(self._z, C.c_double))

    def walk(self, mode=MAC_GROUP_ACC, G=1.0, eps=0.0, delta_acc=2.0 ** -9, theta=0.5,
             group_size=32, a_old=None, want_phi=True):
        """Tree accelerations (caller order).  Returns (ax, ay, az, phi|None, ninter)."""
        n = self.n
        ax, ay, az = np.empty(n), np.empty(n), np.empty(n)
        phi = np.empty(n) if want_phi else None
        nint = np.empty(n, np.int64)
        ao = _f64(a_old) if a_old is not None else None
        self._lib.oracle_tree_walk(self._h, mode, G, eps, delta_acc, theta, group_size,
                                   _p(ao, C.c_double), _p(ax, C.c_double), _p(ay, C.c_double),
                                   _p(az, C.c_double), _p(phi, C.c_double), _p(nint, C.c_int64))
        return ax, ay, az, phi, nint


    def walk_groups(self, groups, mode=MAC_GROUP_ACC, G=1.0, eps=0.0, delta_acc=2.0 ** -9,
                    theta=0.5, group_size=32, a_old=None):
        """Walk only the listed groups.  Returns (ax, ay, az, ninter) with NaN /
        -1 for particles outside them (caller order)."""
        n = self.n
        ax, ay, az = np.full(n, np.nan), np.full(n, np.nan), np.full(n, np.nan)
        nint = np.full(n, -1, np.int64)
        sel = np.ascontiguousarray(groups, dtype=np.int64)
        ao = _f64(a_old) if a_old is not None else None
        self._lib.oracle_tree_walk_groups(self._h, mode, G, eps, delta_acc, theta, group_size,
                                          _p(ao, C.c_double), sel.size, _p(sel, C.c_int64),
                                          _p(ax, C.c_double), _p(ay, C.c_double),
                                          _p(az, C.c_double), None, _p(nint, C.c_int64))
        return ax, ay, az, nint


def kick(v, a, h):
    """v += a h (in place; v and a are (vx, vy, vz) tuples of float64 arrays)."""
    lib = _load()
    lib.oracle_kick(v[0].size, *[_p(q, C.c_double) for q in v], *[_p(_f64(q), C.c_double) for q in a], h)


def drift(x, v, h):
    lib = _load()
    lib.oracle_drift(x[0].size, *[_p(q, C.c_double) for q in x], *[_p(_f64(q), C.c_double) for q in v], h)


def block_level(amag, eps, eta, dt, levels):
    """Time-step level of each particle under block time steps (the paper's
    code integrates with McMillan's block steps, Sect. 1; the step criterion
    is not given -- READING: dt_i = sqrt(2 eta eps / |a_i|), the level the
    smallest k in 0..levels with dt / 2^k <= dt_i; |a| = 0 gives level 0).
    The decision is taken in FP32 with the library's operation order, so equal
    inputs give equal levels."""
    a32 = np.atleast_1d(np.asarray(amag, np.float32))
    eps32 = np.broadcast_to(np.asarray(eps, np.float32), a32.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        dti = np.sqrt(np.float32(2.0) * np.float32(eta) * eps32 / a32).astype(np.float32)
    k = np.zeros(a32.shape, np.int64)
    h = np.full(a32.shape, np.float32(dt), np.float32)
    for _ in range(levels):
        finer = (k < levels) & (h > dti)
        h = np.where(finer, h * np.float32(0.5), h).astype(np.float32)
        k += finer
    return np.where(a32 > 0, k, 0)


def block_kdk(x, v, m, a, G, eps, dt, nsteps, levels, eta, force, trace=None):
    """Leapfrog kick-drift-kick with block time steps, FP64.

    Level k steps by dt / 2^k; the integer clock ticks in units of dt / 2^levels
    and a particle on level k is active at ticks that are multiples of
    2^(levels - k).  At tick 0 every particle takes the opening half kick of
    its level; at each tick where some particle is active, all positions
    drift to that tick, the active particles get new accelerations
    (force(x, index array) -> (ax, ay, az) for those), their closing half
    kick, a new level (coarser only where the tick is a multiple of the new
    step) and, unless it is the last tick, the opening half kick of the new
    step.  x, v, a: tuples of three float64 arrays (copied).  trace (a list,
    optional) receives (tick, active indices, their levels before the tick).
    Returns (x, v, a, levels of the last steps, number of force evaluations)."""
    x = [np.array(q, np.float64) for q in x]
    v = [np.array(q, np.float64) for q in v]
    a = [np.array(q, np.float64) for q in a]
    K = levels
    amag = np.sqrt(a[0] ** 2 + a[1] ** 2 + a[2] ** 2)
    lvl = block_level(amag, eps, eta, dt, K)
    for c in range(3):
        v[c] += a[c] * (dt / 2.0 ** lvl) * 0.5
    total, last, nforce = nsteps << K, 0, 0
    tau = dt / (1 << K)
    for T in range(1, total + 1):
        if T % (1 << (K - int(lvl.max()))):
            continue
        for c in range(3):
            x[c] += v[c] * ((T - last) * tau)
        last = T
        act = np.flatnonzero(T % (1 << (K - lvl)) == 0)
        if trace is not None:
            trace.append((T, act.copy(), lvl[act].copy()))
        fa = force(x, act)
        nforce += act.size
        for c in range(3):
            a[c][act] = fa[c]
            v[c][act] += fa[c] * (dt / 2.0 ** lvl[act]) * 0.5
        if T < total:
            am = np.sqrt(fa[0] ** 2 + fa[1] ** 2 + fa[2] ** 2)
            knew = block_level(am, eps, eta, dt, K)
            old = lvl[act]
            # a coarser level only where this tick is a multiple of its step
            while True:
                bad = (knew < old) & (T % (1 << (K - knew)) != 0)
                if not bad.any():
                    break
                knew = knew + bad
            lvl[act] = knew
            for c in range(3):
                v[c][act] += fa[c] * (dt / 2.0 ** knew) * 0.5
    return x, v, a, lvl, nforce


def diagnostics(x, y, z, vx, vy, vz, m, phi=None):
    """FP64 {E_kin, E_pot, Px, Py, Pz, Lx, Ly, Lz}."""
    lib = _load()
    arrs = [_f64(a) for a in (x, y, z, vx, vy, vz, m)]
    ph = _f64(phi) if phi is not None else None
    out = np.empty(8)
    lib.oracle_diagnostics(arrs[0].size, *[_p(a, C.c_double) for a in arrs], _p(ph, C.c_double),
                           _p(out, C.c_double))
    return out


def mlp_eval(feat, target, w, norm=None, want_grad=True):
    """FP64 MLP forward, MSE and gradient.  Returns (pred, grad|None, loss)."""
    lib = _load()
    feat = _f64(feat).reshape(-1, 8)
    target = _f64(target)
    w = _f64(w)
    n = target.size
    assert w.size == lib.oracle_mlp_params() and feat.shape[0] == n
    nm = _f64(norm) if norm is not None else None
    pred = np.empty(n)
    grad = np.empty(w.size) if want_grad else None
    loss = np.empty(1)
    lib.oracle_mlp_eval(n, _p(feat, C.c_double), _p(target, C.c_double), _p(w, C.c_double),
                        _p(nm, C.c_double), _p(pred, C.c_double), _p(grad, C.c_double),
                        _p(loss, C.c_double))
    return pred, grad, float(loss[0])


def rel_err(ax, ay, az, bx, by, bz):
    """Per-particle |a - b| / |b|."""
    num = np.sqrt((ax - bx) ** 2 + (ay - by) ** 2 + (az - bz) ** 2)
    den = np.sqrt(bx ** 2 + by ** 2 + bz ** 2)
    return num / den


def percentile_nearest_rank(e, p):
    """Nearest-rank percentile (p in [0, 100])."""
    s = np.sort(np.asarray(e))
    if s.size == 0:
        return float("nan")
    k = int(np.ceil(p / 100.0 * s.size)) - 1
    return float(s[min(max(k, 0), s.size - 1)])
