"""Seeded synthetic particle distributions (initial conditions).

These generators produce the inputs that both the CUDA path and the CPU
oracle consume.  They hold none of the force method's arithmetic: no Eq. 1,
no opening criterion, no tree.  Everything here is ordinary sampling from
textbook density profiles, done on the host in FP64 with numpy's
counter-based Philox generator (Philox4x64-10), then stored as FP32
structure-of-arrays (plus FP64 positions for the large workloads).

Units: G = 1, total mass 1 per system, equal particle masses 1/N.

Workloads
---------
plummer(n, seed)        Plummer sphere, scale radius 1 (Aarseth, Henon & Wielen
                        1974 sampling).  Stand-in for a small test system.
hernquist(n, seed, a)   Hernquist (1990) sphere, truncated at 100 a.
galaxy(n, seed)         Three-component disk galaxy (Hernquist bulge 15 %,
                        exponential disk 10 %, NFW halo 75 %), the synthetic
                        stand-in for the M31 model of the paper's Sect. 2.2,
                        which was built with an external tool not available
                        here.
batched(nsys, seed)     Many independent Plummer/Hernquist systems of
                        log-uniform size, concatenated in CSR order.
"""
from __future__ import annotations

import numpy as np

__all__ = ["plummer", "hernquist", "galaxy", "batched", "rng", "mlp_init"]


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Counter-based Philox generator for (seed, stream)."""
    ss = np.random.SeedSequence([int(seed), int(stream)])
    return np.random.Generator(np.random.Philox(ss))


def _isotropic(g: np.random.Generator, r: np.ndarray):
    cth = g.uniform(-1.0, 1.0, r.shape)
    phi = g.uniform(0.0, 2.0 * np.pi, r.shape)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return r * sth * np.cos(phi), r * sth * np.sin(phi), r * cth


def _bisect(f, target, lo, hi, iters=64):
    """Vectorised bisection for the monotone increasing f(x) = target."""
    lo = np.full_like(target, lo)
    hi = np.full_like(target, hi)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        up = f(mid) < target
        lo = np.where(up, mid, lo)
        hi = np.where(up, hi, mid)
    return 0.5 * (lo + hi)


def _pack(x, y, z, vx, vy, vz, m, keep64=False):
    out = {
        "x": x.astype(np.float32), "y": y.astype(np.float32), "z": z.astype(np.float32),
        "vx": vx.astype(np.float32), "vy": vy.astype(np.float32), "vz": vz.astype(np.float32),
        "m": m.astype(np.float32),
    }
    if keep64:
        out["x64"], out["y64"], out["z64"] = (np.ascontiguousarray(x, np.float64),
                                              np.ascontiguousarray(y, np.float64),
                                              np.ascontiguousarray(z, np.float64))
    return out


# ----------------------------------------------------------------------------
# Plummer sphere
# ----------------------------------------------------------------------------
def plummer(n: int, seed: int, rmax: float = 64.0, keep64: bool = False):
    """Plummer sphere (G = M = a = 1).

    Radius from the inverse cumulative mass r = (U^{-2/3} - 1)^{-1/2},
    redrawn while r > rmax; speed from the isotropic distribution function
    by rejection on g(q) = q^2 (1 - q^2)^{7/2}, v = q sqrt(2) (1 + r^2)^{-1/4}.
    """
    g = rng(seed, 1)
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        u = g.uniform(0.0, 1.0, todo.size)
        u = np.maximum(u, 1e-300)
        rr = 1.0 / np.sqrt(np.maximum(u ** (-2.0 / 3.0) - 1.0, 1e-300))
        ok = rr <= rmax
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    x, y, z = _isotropic(g, r)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = g.uniform(0.0, 1.0, todo.size)
        yy = g.uniform(0.0, 0.1, todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    v = q * np.sqrt(2.0) * (1.0 + r * r) ** -0.25
    vx, vy, vz = _isotropic(g, v)
    m = np.full(n, 1.0 / max(n, 1))
    return _pack(x, y, z, vx, vy, vz, m, keep64)


# ----------------------------------------------------------------------------
# Spherical Jeans velocities (isotropic Gaussian), shared by the spheroids
# ----------------------------------------------------------------------------
def _jeans_sigma2(rgrid, rho, mtot):
    """sigma^2(r) = 1/rho(r) * int_r^rmax rho(s) M(s)/s^2 ds on a log grid."""
    f = rho * mtot / (rgrid * rgrid)
    seg = 0.5 * (f[1:] + f[:-1]) * np.diff(rgrid)
    tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    with np.errstate(divide="ignore", invalid="ignore"):
        s2 = np.where(rho > 0, tail / rho, 0.0)
    return s2


def _hernquist_mass(r, a):
    return r * r / (r + a) ** 2


def _hernquist_rho(r, a):
    return a / (2.0 * np.pi * r * (r + a) ** 3)


def hernquist(n: int, seed: int, a: float = 1.0, rtrunc_over_a: float = 100.0,
              keep64: bool = False):
    """Hernquist sphere (G = M = 1), truncated at rtrunc_over_a * a and
    renormalised to unit mass; isotropic Gaussian velocities from the
    spherical Jeans equation of the truncated profile."""
    g = rng(seed, 2)
    rt = rtrunc_over_a * a
    umax = _hernquist_mass(rt, a)
    s = np.sqrt(g.uniform(0.0, umax, n))
    r = a * s / (1.0 - s)
    x, y, z = _isotropic(g, r)
    rgrid = np.geomspace(1e-6 * a, rt, 4096)
    mt = _hernquist_mass(rgrid, a) / umax
    rho = _hernquist_rho(rgrid, a) / umax
    s2 = _jeans_sigma2(rgrid, rho, mt)
    sig = np.sqrt(np.interp(r, rgrid, s2))
    vx, vy, vz = (g.normal(0.0, 1.0, n) * sig for _ in range(3))
    m = np.full(n, 1.0 / max(n, 1))
    return _pack(x, y, z, vx, vy, vz, m, keep64)


# ----------------------------------------------------------------------------
# Three-component galaxy
# ----------------------------------------------------------------------------
_BULGE_FRAC, _BULGE_A = 0.15, 0.6
_DISK_FRAC, _DISK_RD, _DISK_Z0 = 0.10, 5.4, 0.6
_HALO_FRAC, _HALO_RS, _HALO_C = 0.75, 12.0, 10.0


def _nfw_m(x):
    return np.log1p(x) - x / (1.0 + x)


def _disk_m(R, rd):
    t = R / rd
    return 1.0 - (1.0 + t) * np.exp(-t)


def _galaxy_mtot(r):
    """Spherically averaged enclosed mass of the three components (the disk
    counted by its cylindrical enclosed mass)."""
    mb = _hernquist_mass(r, _BULGE_A) / _hernquist_mass(100 * _BULGE_A, _BULGE_A)
    mb = np.where(r >= 100 * _BULGE_A, 1.0, mb)
    mh = _nfw_m(np.minimum(r / _HALO_RS, _HALO_C)) / _nfw_m(_HALO_C)
    md = _disk_m(np.minimum(r, 10 * _DISK_RD), _DISK_RD) / _disk_m(10 * _DISK_RD, _DISK_RD)
    return _BULGE_FRAC * mb + _HALO_FRAC * mh + _DISK_FRAC * md


def galaxy(n: int, seed: int, keep64: bool = True):
    """Hernquist bulge (15 %, a = 0.6, cut at 100 a), exponential disk
    (10 %, R_d = 5.4, sech^2 height 0.6, cut at 10 R_d and |z| <= 6) and NFW
    halo (75 %, r_s = 12, cut at 10 r_s); equal masses, total mass 1.

    Spheroid velocities: isotropic Gaussians with the Jeans dispersion of
    each component in the total spherically averaged potential.  Disk:
    v_phi = v_c(R) plus Gaussian scatter 0.1 v_c in R and phi, and
    sigma_z^2 = pi G Sigma(R) z0.  Components are sampled independently and
    shuffled together.
    """
    nb = int(round(_BULGE_FRAC * n))
    nd = int(round(_DISK_FRAC * n))
    nh = n - nb - nd
    rgrid = np.geomspace(1e-5, 10 * _HALO_RS * _HALO_C, 8192)
    mtot = _galaxy_mtot(rgrid)

    # bulge
    gb = rng(seed, 11)
    a = _BULGE_A
    umax = _hernquist_mass(100 * a, a)
    s = np.sqrt(gb.uniform(0.0, umax, nb))
    rb = a * s / (1.0 - s)
    xb, yb, zb = _isotropic(gb, rb)
    rho_b = np.where(rgrid < 100 * a, _hernquist_rho(rgrid, a), 0.0)
    sb = np.sqrt(np.interp(rb, rgrid, _jeans_sigma2(rgrid, rho_b, mtot)))
    vb = [gb.normal(0.0, 1.0, nb) * sb for _ in range(3)]

    # halo
    gh = rng(seed, 12)
    u = gh.uniform(0.0, 1.0, nh) * _nfw_m(_HALO_C)
    xh_ = _bisect(_nfw_m, u, 0.0, _HALO_C)
    rh = xh_ * _HALO_RS
    xh, yh, zh = _isotropic(gh, rh)
    xg = rgrid / _HALO_RS
    rho_h = np.where(xg < _HALO_C, 1.0 / (xg * (1.0 + xg) ** 2), 0.0)
    sh = np.sqrt(np.interp(rh, rgrid, _jeans_sigma2(rgrid, rho_h, mtot)))
    vh = [gh.normal(0.0, 1.0, nh) * sh for _ in range(3)]

    # disk
    gd = rng(seed, 13)
    rd = _DISK_RD
    u = gd.uniform(0.0, 1.0, nd) * _disk_m(10 * rd, rd)
    R = _bisect(lambda t: _disk_m(t, rd), u, 0.0, 10 * rd)
    zd = np.empty(nd)
    todo = np.arange(nd)
    while todo.size:
        w = gd.uniform(-1.0, 1.0, todo.size)
        zz = _DISK_Z0 * np.arctanh(np.clip(w, -1 + 1e-16, 1 - 1e-16))
        ok = np.abs(zz) <= 6.0
        zd[todo[ok]] = zz[ok]
        todo = todo[~ok]
    ph = gd.uniform(0.0, 2.0 * np.pi, nd)
    xd, yd = R * np.cos(ph), R * np.sin(ph)
    vc = np.sqrt(np.interp(R, rgrid, mtot) / np.maximum(R, 1e-12))
    sig_surf = _DISK_FRAC / (2.0 * np.pi * rd * rd * _disk_m(10 * rd, rd)) * np.exp(-R / rd)
    sz = np.sqrt(np.pi * sig_surf * _DISK_Z0)
    vR = gd.normal(0.0, 1.0, nd) * 0.1 * vc
    vphi = vc + gd.normal(0.0, 1.0, nd) * 0.1 * vc
    vzd = gd.normal(0.0, 1.0, nd) * sz
    vxd = vR * np.cos(ph) - vphi * np.sin(ph)
    vyd = vR * np.sin(ph) + vphi * np.cos(ph)

    x = np.concatenate([xb, xd, xh])
    y = np.concatenate([yb, yd, yh])
    z = np.concatenate([zb, zd, zh])
    vx = np.concatenate([vb[0], vxd, vh[0]])
    vy = np.concatenate([vb[1], vyd, vh[1]])
    vz = np.concatenate([vb[2], vzd, vh[2]])
    perm = rng(seed, 14).permutation(n)
    m = np.full(n, 1.0 / n)
    return _pack(x[perm], y[perm], z[perm], vx[perm], vy[perm], vz[perm], m, keep64)


# ----------------------------------------------------------------------------
# Many independent systems
# ----------------------------------------------------------------------------
def batched(nsys: int, seed: int, log2_min: float = 10.0, log2_max: float = 16.0,
            sizes=None):
    """nsys independent systems, N_s = round(2^(log2_min + (log2_max-log2_min) U)),
    each a Plummer or a Hernquist sphere (probability 1/2 each, unit mass,
    unit scale radius), with softening eps_s = 4 / N_s^(1/3).

    Returns the concatenated SoA arrays (system s occupies
    offsets[s]:offsets[s+1]), the int64 offsets and the float32 eps_s.
    """
    g = rng(seed, 21)
    if sizes is None:
        sizes = np.rint(2.0 ** g.uniform(log2_min, log2_max, nsys)).astype(np.int64)
    else:
        sizes = np.asarray(sizes, np.int64)
    kinds = g.integers(0, 2, nsys)
    parts = []
    for s in range(nsys):
        ns = int(sizes[s])
        sub = (plummer(ns, seed * 100003 + s) if kinds[s] == 0
               else hernquist(ns, seed * 100003 + s))
        parts.append(sub)
    out = {k: np.concatenate([p[k] for p in parts]) for k in ("x", "y", "z", "vx", "vy", "vz", "m")}
    out["offsets"] = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    # eps_s = 4 / N_s^(1/3); an empty system gets eps = 1 (it has no particles)
    out["eps"] = (4.0 / np.maximum(sizes, 1).astype(np.float64) ** (1.0 / 3.0)).astype(np.float32)
    out["eps"][sizes == 0] = 1.0
    out["kind"] = kinds.astype(np.int32)
    return out


# ----------------------------------------------------------------------------
# Initial weights of the cost model (seeded random numbers are inputs too)
# ----------------------------------------------------------------------------
def mlp_init(seed: int):
    """He-uniform weights for the 8 -> 32 -> 32 -> 1 ReLU network, zero
    biases, flattened as W1[8][32], b1[32], W2[32][32], b2[32], W3[32], b3."""
    g = rng(seed, 31)

    def he(fan_in, shape):
        lim = np.sqrt(6.0 / fan_in)
        return g.uniform(-lim, lim, shape)
    parts = [he(8, (8, 32)).ravel(), np.zeros(32), he(32, (32, 32)).ravel(), np.zeros(32),
             g.uniform(-1 / np.sqrt(32), 1 / np.sqrt(32), 32), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)
