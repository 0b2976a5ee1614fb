"""Pins of the FP64 CPU oracle against things other than itself.

Every check here is fixed by the paper or by mathematics: hand-derived closed
forms (tests/golden/closed_forms.json), symmetry, Newton's third law,
analytic density profiles, a library stable sort, higher-precision brute
force on tiny inputs, special cases where the tree must reduce to the direct
sum, and conservation properties of the leapfrog.  A plausible mistake in
the oracle (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import ics
import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(np.asarray(b)), 1e-300))


# --------------------------------------------------------------------------- Eq. 1
@pytest.mark.parametrize("case", ["two_body_pythagorean", "two_body_unsoftened"])
def test_direct_two_body_closed_form(case):
    c = GOLD[case]
    ax, ay, az, phi = oracle.direct(c["x"], c["y"], c["z"], c["m"], c["G"], c["eps"])
    for got, want in ((ax, c["ax"]), (ay, c["ay"]), (phi, c["phi"])):
        assert np.allclose(got, want, rtol=1e-14, atol=0)
    assert np.all(az == 0.0)


def _cube():
    v = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], float)
    return v


def test_direct_cube_vertices():
    v = _cube()
    m = np.ones(8)
    ax, ay, az, _ = oracle.direct(v[:, 0], v[:, 1], v[:, 2], m, 1.0, 0.0)
    want = GOLD["cube_vertices"]["component_magnitude"]
    a = np.stack([ax, ay, az], 1)
    # every component has the closed-form magnitude and points to the centre
    assert np.allclose(np.abs(a), want, rtol=1e-14)
    assert np.all(np.sign(a) == -np.sign(v))


def test_direct_cube_plus_centre_symmetry():
    v = np.vstack([_cube(), [[0, 0, 0]]])
    m = np.ones(9)
    ax, ay, az, _ = oracle.direct(v[:, 0], v[:, 1], v[:, 2], m, 1.0, 0.0)
    assert abs(ax[8]) < 1e-15 and abs(ay[8]) < 1e-15 and abs(az[8]) < 1e-15
    want = GOLD["cube_vertices_plus_centre"]["component_magnitude"]
    assert np.allclose(np.abs(ax[:8]), want, rtol=1e-14)


def test_direct_octahedron_centre_zero():
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [0, 0, 0]], float)
    ax, ay, az, _ = oracle.direct(v[:, 0], v[:, 1], v[:, 2], np.ones(7), 1.0, 0.1)
    assert max(abs(ax[6]), abs(ay[6]), abs(az[6])) < 1e-15
    mags = np.sqrt(ax[:6] ** 2 + ay[:6] ** 2 + az[:6] ** 2)
    assert np.allclose(mags, mags[0], rtol=1e-14)


def test_direct_longdouble_bruteforce():
    """Brute force in extended precision for N <= 64."""
    g = ics.rng(7)
    n = 48
    x, y, z = (g.normal(size=n) for _ in range(3))
    m = g.uniform(0.5, 2.0, n)
    eps = 0.05
    ax, ay, az, phi = oracle.direct(x, y, z, m, 1.0, eps)
    L = np.longdouble
    X, Y, Z, Mm = (np.asarray(a, dtype=L) for a in (x, y, z, m))
    for i in range(n):
        dx, dy, dz = X - X[i], Y - Y[i], Z - Z[i]
        r2 = dx * dx + dy * dy + dz * dz + L(eps) * L(eps)
        w = Mm / (r2 * np.sqrt(r2))
        w[i] = 0
        pw = Mm / np.sqrt(r2)
        pw[i] = 0
        assert abs(float((w * dx).sum()) - ax[i]) <= 1e-14 * float(np.abs(w * dx).sum())
        assert abs(float((w * dy).sum()) - ay[i]) <= 1e-14 * float(np.abs(w * dy).sum())
        assert abs(float((w * dz).sum()) - az[i]) <= 1e-14 * float(np.abs(w * dz).sum())
        assert abs(-float(pw.sum()) - phi[i]) <= 1e-14 * float(pw.sum())


def test_direct_third_law():
    p = ics.plummer(2000, 3)
    ax, ay, az, _ = oracle.direct(p["x"], p["y"], p["z"], p["m"], 1.0, 1 / 128)
    m = p["m"].astype(float)
    for a in (ax, ay, az):
        assert abs((m * a).sum()) <= 1e-13 * np.abs(m * a).sum()


def test_direct_G_scaling_and_softened_point_mass():
    # a test particle of negligible mass at distance r from a mass M
    M, r, eps, G = 3.0, 2.5, 0.7, 4.0
    ax, ay, az, phi = oracle.direct([0.0, r], [0.0, 0.0], [0.0, 0.0], [M, 1e-30], G, eps)
    assert np.isclose(ax[1], -G * M * r / (r * r + eps * eps) ** 1.5, rtol=1e-15)
    assert np.isclose(phi[1], -G * M / np.sqrt(r * r + eps * eps), rtol=1e-15)


def _shell_checks(p, seed, eps):
    """Per target: direct-sum radial acceleration over -G M_enc(r)/r^2 and the
    potential over -G M_enc(r)/r - G sum_{r_j > r} m_j/r_j, both from the
    sample's own radial mass profile (Newton's shell theorem)."""
    x, y, z, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    n = x.size
    tg = ics.rng(seed, 5).choice(n, 3000, replace=False)
    ax, ay, az, phi = oracle.direct_targets(x, y, z, m, tg, 1.0, eps, want_phi=True)
    R = np.sqrt(x * x + y * y + z * z)
    o = np.argsort(R)
    Rs = R[o]
    cm = np.cumsum(m[o])
    outer = np.cumsum((m[o] / Rs)[::-1])[::-1]
    r = R[tg]
    k = np.searchsorted(Rs, r, side="left")
    menc = np.where(k > 0, cm[np.maximum(k - 1, 0)], 0.0)
    out = np.where(k + 1 < n, outer[np.minimum(k + 1, n - 1)], 0.0)
    ar = (ax * x[tg] + ay * y[tg] + az * z[tg]) / r
    return r, ar / (-menc / r ** 2), phi / (-menc / r - out)


@pytest.mark.parametrize("gen,seed", [(ics.plummer, 11), (ics.hernquist, 12)])
def test_direct_shell_theorem_profiles(gen, seed):
    """Plummer and Hernquist spheres: shell-averaged radial acceleration and
    potential of the direct sum match the monopole of the sample's own
    spherical mass profile, away from the softening scale."""
    r, ra, rp = _shell_checks(gen(1 << 15, seed), seed, 1 / 256)
    edges = [0.15, 0.4, 0.8, 1.5, 3.0, 8.0]
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (r >= lo) & (r < hi)
        assert sel.sum() > 100
        for q in (ra[sel], rp[sel]):
            sem = q.std() / np.sqrt(sel.sum())
            assert abs(q.mean() - 1) < 4 * sem + 1e-3, (lo, hi, q.mean(), sem)


def test_ic_profiles_follow_analytic_mass():
    """The samplers draw from the stated profiles: enclosed-mass fractions
    agree with M(<r) within binomial noise (Plummer r^3/(1+r^2)^{3/2};
    truncated Hernquist (r/(r+1))^2 / (100/101)^2)."""
    n = 1 << 15
    for gen, seed, M in ((ics.plummer, 11, lambda r: r ** 3 / (1 + r * r) ** 1.5),
                         (ics.hernquist, 12, lambda r: (r / (r + 1)) ** 2 / (100 / 101) ** 2)):
        p = gen(n, seed)
        R = np.sqrt(p["x"].astype(float) ** 2 + p["y"] ** 2 + p["z"] ** 2)
        for r in (0.3, 1.0, 3.0):
            f = (R < r).mean()
            assert abs(f - M(r)) < 5 * np.sqrt(M(r) * (1 - M(r)) / n) + 1e-4


# --------------------------------------------------------------------------- keys and order
def test_interleave_golden():
    for c in GOLD["morton_keys"]["cases"]:
        got = oracle.interleave([c["q"][0]], [c["q"][1]], [c["q"][2]], c["levels"])[0]
        assert int(got) == c["key"], c


def test_cells_fp32_quantisation_bounds():
    p = ics.galaxy(5000, 4)
    cube = oracle.cube(p["x"], p["y"], p["z"])
    lo = np.array([p["x"].min(), p["y"].min(), p["z"].min()], np.float32)
    assert np.array_equal(cube[:3], lo)
    ext = max(np.float32(p["x"].max() - lo[0]), np.float32(p["y"].max() - lo[1]),
              np.float32(p["z"].max() - lo[2]))
    assert cube[3] == np.float32(ext * np.float32(1 + 2.0 ** -20))
    q = oracle.cells(p["x"], p["y"], p["z"], cube, 21)
    for a, c in zip(q, (p["x"], p["y"], p["z"])):
        assert a.max() <= (1 << 21) - 1
        # the cell index is the FP32 floor of the scaled offset (monotone in x)
        o = np.argsort(c, kind="stable")
        assert np.all(np.diff(a[o].astype(np.int64)) >= 0)


def test_sort_matches_library_stable_sort():
    p = ics.galaxy(20000, 5)
    k, _ = oracle.keys(p["x"], p["y"], p["z"], 21)
    k[::7] = k[3]  # force many ties
    assert np.array_equal(oracle.sort_order(k), np.argsort(k, kind="stable"))


# --------------------------------------------------------------------------- tree
@pytest.fixture(scope="module")
def gal_tree():
    n = 1 << 14
    p = ics.galaxy(n, 6)
    t = oracle.Tree(p["x"], p["y"], p["z"], p["m"], levels=21, leaf_cap=16)
    return p, t


def test_tree_order_is_sorted_morton_order(gal_tree):
    """The recursive subdivision visits particles in (key, index) order, the
    order a stable radix sort of the keys produces."""
    p, t = gal_tree
    k, _ = oracle.keys(p["x"], p["y"], p["z"], 21)
    assert np.array_equal(t.order(), np.argsort(k, kind="stable"))


def test_tree_invariants(gal_tree):
    p, t = gal_tree
    nd = t.nodes()
    n, cap = t.n, t.leaf_cap
    order = t.order()
    leaf = nd["nchild"] == 0
    # every particle in exactly one leaf
    cover = np.zeros(n, np.int64)
    for f, c in zip(nd["first"][leaf], nd["count"][leaf]):
        cover[f:f + c] += 1
    assert np.all(cover == 1)
    # leaf sizes, internal sizes
    assert np.all((nd["count"][leaf] <= cap) | (nd["level"][leaf] == 21))
    assert np.all(nd["count"][~leaf] > cap)
    x, y, z, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    for i in np.flatnonzero(~leaf):
        ch = np.arange(nd["child"][i], nd["child"][i] + nd["nchild"][i])
        assert nd["count"][ch].sum() == nd["count"][i]
        assert np.all(nd["level"][ch] == nd["level"][i] + 1)
        assert np.all(nd["prefix"][ch] >> np.uint64(3) == nd["prefix"][i])
        assert np.isclose(nd["M"][ch].sum(), nd["M"][i], rtol=1e-14)
        assert nd["first"][ch[0]] == nd["first"][i]
    # moments against the definition, and b >= the exact member radius
    for i in range(0, nd["M"].size, 7):
        mem = order[nd["first"][i]:nd["first"][i] + nd["count"][i]]
        M = m[mem].sum()
        com = np.array([(m[mem] * q[mem]).sum() / M for q in (x, y, z)])
        assert np.isclose(nd["M"][i], M, rtol=1e-14)
        assert np.allclose([nd["cx"][i], nd["cy"][i], nd["cz"][i]], com, rtol=1e-14, atol=1e-14)
        rmax = np.sqrt((x[mem] - com[0]) ** 2 + (y[mem] - com[1]) ** 2 + (z[mem] - com[2]) ** 2).max()
        if leaf[i]:
            assert np.isclose(nd["b"][i], rmax, rtol=1e-14, atol=1e-15)
        else:
            assert nd["b"][i] >= rmax * (1 - 1e-14)


def test_tree_groups_partition(gal_tree):
    p, t = gal_tree
    nd = t.nodes()
    for G in (16, 32, 64):
        f, c = t.groups(G)
        assert np.all(c <= G) and np.all(c >= 1)
        assert f[0] == 0 and np.all(f[1:] == f[:-1] + c[:-1]) and f[-1] + c[-1] == t.n
        # each group is a run of consecutive siblings, each holding at most G,
        # under a parent holding more than G; runs are packed greedily, so the
        # next sibling after a run does not fit into it
        by_first = {}
        for i in range(nd["M"].size):
            by_first.setdefault(int(nd["first"][i]), []).append(i)
        parent = np.full(nd["M"].size, -1)
        for i in np.flatnonzero(nd["nchild"] > 0):
            parent[nd["child"][i]:nd["child"][i] + nd["nchild"][i]] = i
        for a, b in zip(f, c):
            # the deepest node starting at a whose parent holds more than G
            cands = [i for i in by_first[int(a)] if parent[i] >= 0 and nd["count"][parent[i]] > G]
            i = max(cands, key=lambda q: nd["level"][q])
            par = parent[i]
            sib = np.arange(nd["child"][par], nd["child"][par] + nd["nchild"][par])
            k0 = int(np.flatnonzero(sib == i)[0])
            tot, k = 0, k0
            while k < sib.size and nd["count"][sib[k]] <= G and tot + nd["count"][sib[k]] <= G:
                tot += nd["count"][sib[k]]
                k += 1
            assert tot == b, (a, b, tot)


@pytest.mark.parametrize("mode", [oracle.MAC_PARTICLE_ACC, oracle.MAC_GROUP_ACC])
def test_tree_dacc_zero_is_direct(mode):
    """With delta_acc = 0 Eq. 2 accepts only single-particle nodes, so the
    tree sum reduces to the direct sum of Eq. 1."""
    p = ics.plummer(3000, 8)
    x, y, z, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    ax, ay, az, phi = oracle.direct(x, y, z, m, 1.0, 1 / 64)
    t = oracle.Tree(x, y, z, m, 21, 8)
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2)
    bx, by, bz, bphi, nint = t.walk(mode, 1.0, 1 / 64, 0.0, 0.5, 32, amag)
    assert np.max(oracle.rel_err(bx, by, bz, ax, ay, az)) < 1e-13
    assert np.allclose(bphi, phi, rtol=1e-13)
    assert np.all(nint == 3000)


# --------------------------------------------------------------------------- refit
def _moved(p, seed, scale):
    """Positions displaced by seeded Gaussian steps of `scale`, plus a few
    particles thrown across the system (far outside their cells)."""
    g = np.random.default_rng(seed)
    x, y, z = (p[k].astype(float) + g.normal(scale=scale, size=p[k].size) for k in ("x", "y", "z"))
    far = g.choice(x.size, 16, replace=False)
    x[far], y[far], z[far] = -x[far], z[far], y[far]
    return x, y, z


def test_refit_moments_follow_the_definition():
    """After a refit the tree keeps its membership; the moments must be those
    of the members at their new positions (mass, centre of mass by
    definition, b_J >= the exact largest member distance, exact for leaves)."""
    p = ics.galaxy(6000, 9)
    x0, y0, z0, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    t = oracle.Tree(x0, y0, z0, m, 21, 8)
    before = t.nodes()
    x, y, z = _moved(p, 1, 0.05)
    t.refit(x, y, z)
    nd = t.nodes()
    order = t.order()
    for k in ("level", "first", "count", "nchild", "child"):
        assert np.array_equal(nd[k], before[k])
    leaf = nd["nchild"] == 0
    moved_away = 0
    for i in range(nd["M"].size):
        mem = order[nd["first"][i]:nd["first"][i] + nd["count"][i]]
        M = m[mem].sum()
        com = np.array([(m[mem] * q[mem]).sum() / M for q in (x, y, z)])
        assert np.isclose(nd["M"][i], M, rtol=1e-14)
        assert np.allclose([nd["cx"][i], nd["cy"][i], nd["cz"][i]], com, rtol=1e-13, atol=1e-13)
        rmax = np.sqrt((x[mem] - com[0]) ** 2 + (y[mem] - com[1]) ** 2 + (z[mem] - com[2]) ** 2).max()
        if leaf[i]:
            assert np.isclose(nd["b"][i], rmax, rtol=1e-14, atol=1e-15)
        else:
            assert nd["b"][i] >= rmax * (1 - 1e-14)
            moved_away += nd["b"][i] > before["b"][i]
    assert moved_away > 0  # the thrown particles enlarge their ancestors


def test_refit_at_the_same_positions_keeps_mass_and_centre():
    """Refitting to unchanged positions reproduces M and the centre of mass
    exactly; b_J can only grow (the cell-corner bound is dropped)."""
    p = ics.plummer(4000, 10)
    x, y, z, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    t = oracle.Tree(x, y, z, m, 21, 16)
    a = t.nodes()
    t.refit(x, y, z)
    b = t.nodes()
    for k in ("M", "cx", "cy", "cz"):
        assert np.array_equal(a[k], b[k])
    leaf = a["nchild"] == 0
    assert np.array_equal(a["b"][leaf], b["b"][leaf])
    assert np.all(b["b"][~leaf] >= a["b"][~leaf])


@pytest.mark.parametrize("mode", [oracle.MAC_PARTICLE_ACC, oracle.MAC_GROUP_ACC])
def test_refit_dacc_zero_is_direct_at_the_new_positions(mode):
    """With delta_acc = 0 the walk of a refitted tree is the direct sum of
    Eq. 1 over the new positions: a refit that kept any stale position or
    moment would fail."""
    p = ics.plummer(2500, 11)
    x0, y0, z0, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    t = oracle.Tree(x0, y0, z0, m, 21, 8)
    x, y, z = _moved(p, 2, 0.1)
    t.refit(x, y, z)
    ax, ay, az, phi = oracle.direct(x, y, z, m, 1.0, 1 / 64)
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2)
    bx, by, bz, bphi, _ = t.walk(mode, 1.0, 1 / 64, 0.0, 0.5, 32, amag)
    assert np.max(oracle.rel_err(bx, by, bz, ax, ay, az)) < 1e-13
    assert np.allclose(bphi, phi, rtol=1e-13)


def test_refit_error_stays_bounded_by_the_mac():
    """After one leapfrog-sized displacement the refitted tree's errors at
    delta_acc = 2^-9 stay close to a fresh tree's: the MAC still bounds them
    because b_J still bounds every member's distance."""
    p = ics.plummer(8192, 12)
    x0, y0, z0, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    t = oracle.Tree(x0, y0, z0, m, 21, 16)
    dt = 1.0 / 256
    x, y, z = (p[k].astype(float) + dt * p["v" + k].astype(float) for k in ("x", "y", "z"))
    t.refit(x, y, z)
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, 1 / 128, want_phi=False)
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2)
    rx, ry, rz, _, nr = t.walk(oracle.MAC_GROUP_ACC, 1.0, 1 / 128, 2.0 ** -9, 0.5, 64, amag,
                               want_phi=False)
    f = oracle.Tree(x, y, z, m, 21, 16)
    fx, fy, fz, _, nf = f.walk(oracle.MAC_GROUP_ACC, 1.0, 1 / 128, 2.0 ** -9, 0.5, 64, amag,
                               want_phi=False)
    er = oracle.rel_err(rx, ry, rz, ax, ay, az)
    ef = oracle.rel_err(fx, fy, fz, ax, ay, az)
    for q in (50, 99):
        assert oracle.percentile_nearest_rank(er, q) <= 1.5 * oracle.percentile_nearest_rank(ef, q)
    assert nr.sum() >= 0.9 * nf.sum()


def test_tree_tiny_theta_is_direct():
    p = ics.plummer(2000, 9)
    x, y, z, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, 0.01)
    t = oracle.Tree(x, y, z, m, 21, 16)
    bx, by, bz, _, _ = t.walk(oracle.MAC_GROUP_GEO, 1.0, 0.01, 0.0, 1e-9, 32, None)
    assert np.max(oracle.rel_err(bx, by, bz, ax, ay, az)) < 1e-12


def test_tree_distant_cluster_is_its_monopole():
    """A compact cluster far from the target is accepted as one node and
    contributes exactly its monopole: G M (com - r)/(d^2 + eps^2)^{3/2}."""
    g = ics.rng(10)
    k = 12
    cl = g.normal(scale=0.01, size=(k, 3)) + np.array([100.0, 50.0, -20.0])
    mc = g.uniform(1.0, 2.0, k)
    x = np.concatenate([cl[:, 0], [0.0]])
    y = np.concatenate([cl[:, 1], [0.0]])
    z = np.concatenate([cl[:, 2], [0.0]])
    m = np.concatenate([mc, [1e-6]])
    t = oracle.Tree(x, y, z, m, 21, 8)
    aold = np.full(k + 1, 1e3)
    eps = 0.3
    ax, ay, az, phi, nint = t.walk(oracle.MAC_PARTICLE_ACC, 1.0, eps, 2 ** -9, 0.5, 1, aold)
    M = mc.sum()
    com = (mc[:, None] * cl).sum(0) / M
    d = com  # target at the origin
    r2 = (d * d).sum() + eps * eps
    want = M * d / r2 ** 1.5
    assert nint[k] < k  # the cluster was not opened particle by particle
    assert np.allclose([ax[k], ay[k], az[k]], want, rtol=1e-12)


def _eq1(src, ms, tgt, G):
    """Eq. 1 with eps = 0 written out for a handful of sources (test-side)."""
    d = np.asarray(src, float) - np.asarray(tgt, float)
    r = np.sqrt((d * d).sum(1))
    keep = r > 0
    return G * (np.asarray(ms)[keep, None] * d[keep] / r[keep, None] ** 3).sum(0)


@pytest.mark.parametrize("case", GOLD["mac_threshold"]["cases"], ids=lambda c: c["name"])
def test_mac_threshold_hand_cases(case):
    """Eq. 2 at its boundary: hand-derived node/target pairs for which both
    sides are exact in FP64 decide accept on equality, reject one ulp below,
    the powers of b_J (2) and d (4), the factor G, the strict d > b_J and the
    group-mode distance |com - c_g| - r_g (tests/golden/closed_forms.json)."""
    anchors = [[0.0, 0.0, 0.0], [64.0, 64.0, 64.0]]
    ma = 2.0 ** -40
    cl, tg = case["cluster"], case["targets"]
    pos = np.array(anchors + cl + tg, float)
    m = np.array([ma, ma] + [0.25] * len(cl) + [0.25] * len(tg))
    nt = len(tg)
    t = oracle.Tree(pos[:, 0], pos[:, 1], pos[:, 2], m, 21, 2)
    nd = t.nodes()
    # the cluster is one leaf with the exact centre of mass and b_J
    com = np.mean(np.array(cl, float), 0)
    bJ = np.sqrt(((np.array(cl, float) - com) ** 2).sum(1)).max()
    hit = [k for k in range(t.nnodes) if nd["nchild"][k] == 0 and nd["count"][k] == 2 and
           nd["cx"][k] == com[0] and nd["cy"][k] == com[1] and nd["cz"][k] == com[2]]
    assert len(hit) == 1 and nd["b"][hit[0]] == bJ and nd["M"][hit[0]] == 0.5
    aold = np.ones(pos.shape[0])
    aold[-nt:] = case["a_old"]
    mode = oracle.MAC_GROUP_ACC if case["mode"] == "group" else oracle.MAC_PARTICLE_ACC
    gs = case.get("group_size", 1)
    ax, ay, az, _, nint = t.walk(mode, case["G"], 0.0, case["dacc"], 0.5, gs, aold, want_phi=False)
    assert list(nint[-nt:]) == case["ninter"]
    # the accepted cluster adds its monopole, an opened one its members
    for j in range(nt):
        i = pos.shape[0] - nt + j
        others = [p for k, p in enumerate(tg) if k != j]
        src = anchors + others + ([list(com)] if case["accept"] else cl)
        ms = [ma, ma] + [0.25] * len(others) + ([0.5] if case["accept"] else [0.25] * len(cl))
        want = _eq1(src, ms, tg[j], case["G"])
        assert np.allclose([ax[i], ay[i], az[i]], want, rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------------- quadrupoles
def _far_cluster_walk(cl, mc, eps, quad, target=(0.0, 0.0, 0.0), leaf_cap=1):
    """Walk for one light target far from a cluster; returns its acceleration
    and interaction count (2 when the cluster is accepted as one node: that
    node plus the target's own leaf, whose zero self term is counted)."""
    x = np.concatenate([cl[:, 0], [target[0]]])
    y = np.concatenate([cl[:, 1], [target[1]]])
    z = np.concatenate([cl[:, 2], [target[2]]])
    m = np.concatenate([mc, [1e-9]])
    t = oracle.Tree(x, y, z, m, 21, leaf_cap)
    mode = oracle.MAC_PARTICLE_GEO | (oracle.QUADRUPOLE if quad else 0)
    ax, ay, az, phi, nint = t.walk(mode, 1.0, eps, 0.0, 0.5, 1, None)
    k = mc.size
    return np.array([ax[k], ay[k], az[k]]), phi[k], nint[k], t


def test_quadrupole_dumbbell_closed_form():
    """Two masses m at com +- b x, target at distance D on the axis, eps = 0:
    Q = diag(4 m b^2, -2 m b^2, -2 m b^2) and the quadrupole-corrected pull is
    2m/D^2 + 6 m b^2/D^4 (the first two terms of m/(D-b)^2 + m/(D+b)^2, hand
    expansion), the potential -2m/D - 2 m b^2/D^3."""
    m, b, D = 1.5, 0.01, 60.0
    cl = np.array([[D - b, 0.0, 0.0], [D + b, 0.0, 0.0]])
    a, phi, nint, t = _far_cluster_walk(cl, np.array([m, m]), 0.0, True)
    assert nint == 2
    assert np.isclose(a[0], 2 * m / D ** 2 + 6 * m * b ** 2 / D ** 4, rtol=1e-13)
    assert abs(a[1]) < 1e-18 and abs(a[2]) < 1e-18
    assert np.isclose(phi, -2 * m / D - 2 * m * b ** 2 / D ** 3, rtol=1e-13)
    nd = t.nodes()
    Q = t.quadrupoles()
    node = int(np.flatnonzero((nd["count"] == 2) & np.isclose(nd["M"], 2 * m))[0])
    assert np.allclose(Q[node], [4 * m * b * b, -2 * m * b * b, -2 * m * b * b, 0, 0, 0],
                       rtol=1e-9, atol=1e-18)
    # its error against the exact pull is fourth order, the monopole's second
    exact = m / (D - b) ** 2 + m / (D + b) ** 2
    mono, _, _, _ = _far_cluster_walk(cl, np.array([m, m]), 0.0, False)
    assert abs(a[0] - exact) / exact < 6 * (b / D) ** 4
    assert abs(mono[0] - exact) / exact > 2.9 * (b / D) ** 2


def test_quadrupole_far_field_convergence_order():
    """For a generic compact cluster the monopole's relative error falls as
    (b/D)^2 and the quadrupole's as (b/D)^3 (the dipole vanishes about the
    centre of mass; the octupole is next): doubling D divides them by about 4
    and 8."""
    g = ics.rng(31)
    k = 24
    u = np.array([0.6, -0.48, 0.64])
    off = g.normal(scale=0.05, size=(k, 3))
    mc = g.uniform(0.5, 2.0, k)
    errs = {}
    for quad in (False, True):
        e = []
        for D in (40.0, 80.0, 160.0):
            cl = off + D * u
            a, _, nint, _ = _far_cluster_walk(cl, mc, 0.0, quad)
            assert nint == 2
            d = cl  # target at the origin
            want = (mc[:, None] * d / (d * d).sum(1, keepdims=True) ** 1.5).sum(0)
            e.append(np.linalg.norm(a - want) / np.linalg.norm(want))
        errs[quad] = e
    for e0, e1 in zip(errs[False], errs[False][1:]):
        assert 3.5 < e0 / e1 < 4.5
    for e0, e1 in zip(errs[True], errs[True][1:]):
        assert 7.0 < e0 / e1 < 9.0
    assert errs[True][0] < 0.1 * errs[False][0]


def test_quadrupole_vanishes_for_cubic_symmetry():
    """Equal masses on the vertices of a cube have zero quadrupole: the
    quadrupole walk equals the monopole walk."""
    v = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], float) * 0.02
    cl = v + np.array([50.0, 20.0, -30.0])
    mc = np.full(8, 0.7)
    aq, pq, nq, t = _far_cluster_walk(cl, mc, 0.1, True, leaf_cap=4)
    am, pm, nm, _ = _far_cluster_walk(cl, mc, 0.1, False, leaf_cap=4)
    assert nq == nm == 2
    nd = t.nodes()
    node = int(np.flatnonzero(nd["count"] == 8)[-1])
    # zero up to the rounding of the offsets (|s| = 0.035 at coordinates ~60)
    assert np.max(np.abs(t.quadrupoles()[node])) < 1e-11 * (mc * (v * v).sum(1)).sum()
    assert np.allclose(aq, am, rtol=1e-12) and np.isclose(pq, pm, rtol=1e-12)


def test_quadrupoles_are_traceless_and_lower_the_error(gal_tree):
    """Every node's quadrupole is traceless; with the same MAC the quadrupole
    walk's error percentiles are below the monopole walk's."""
    p, t = gal_tree
    Q = t.quadrupoles()
    nd = t.nodes()
    scale = nd["M"] * nd["b"] ** 2 + 1e-300
    assert np.all(np.abs(Q[:, 0] + Q[:, 1] + Q[:, 2]) <= 1e-12 * scale)
    x, y, z, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, 1 / 64, want_phi=False)
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2)
    e = {}
    for quad in (0, oracle.QUADRUPOLE):
        bx, by, bz, _, _ = t.walk(oracle.MAC_GROUP_ACC | quad, 1.0, 1 / 64, 2.0 ** -9, 0.5, 64,
                                  amag, want_phi=False)
        e[quad] = oracle.rel_err(bx, by, bz, ax, ay, az)
    for q in (50, 99):
        assert (oracle.percentile_nearest_rank(e[oracle.QUADRUPOLE], q) <
                0.7 * oracle.percentile_nearest_rank(e[0], q))


def test_tree_error_decreases_with_dacc():
    n = 1 << 13
    p = ics.plummer(n, 1)
    x, y, z, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, 1 / 128, want_phi=False)
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2)
    t = oracle.Tree(x, y, z, m, 21, 16)
    prev = np.inf
    prev_n = 0
    for k in (2, 5, 8, 11, 14):
        bx, by, bz, _, nint = t.walk(oracle.MAC_GROUP_ACC, 1.0, 1 / 128, 2.0 ** -k, 0.5, 32, amag,
                                     want_phi=False)
        e50 = np.percentile(oracle.rel_err(bx, by, bz, ax, ay, az), 50)
        assert e50 < prev
        assert nint.sum() > prev_n
        prev, prev_n = e50, nint.sum()


def test_tree_walk_groups_subset_equals_full_walk():
    p = ics.galaxy(6000, 15)
    x, y, z, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    t = oracle.Tree(x, y, z, m, 21, 16)
    aold = np.full(6000, 0.5)
    fx, fy, fz, _, fn = t.walk(oracle.MAC_GROUP_ACC, 1.0, 0.01, 2 ** -7, 0.5, 32, aold)
    f, c = t.groups(32)
    sel = np.arange(0, f.size, 5)
    gx, gy, gz, gn = t.walk_groups(sel, oracle.MAC_GROUP_ACC, 1.0, 0.01, 2 ** -7, 0.5, 32, aold)
    members = np.concatenate([t.order()[f[g]:f[g] + c[g]] for g in sel])
    assert np.array_equal(gx[members], fx[members]) and np.array_equal(gn[members], fn[members])
    others = np.setdiff1d(np.arange(6000), members)
    assert np.all(np.isnan(gx[others]))


def test_tree_group_mac_not_looser_than_particle_mac():
    """The group distance |com - c_g| - r_g is a lower bound of every member's
    distance and amin <= |a_i|, so a group accepts a node only if every member
    would: group-mode lists are at least as long as particle-mode lists."""
    n = 1 << 12
    p = ics.plummer(n, 2)
    x, y, z, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, 1 / 128, want_phi=False)
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2)
    t = oracle.Tree(x, y, z, m, 21, 16)
    _, _, _, _, ng = t.walk(oracle.MAC_GROUP_ACC, 1.0, 1 / 128, 2 ** -9, 0.5, 32, amag)
    _, _, _, _, npart = t.walk(oracle.MAC_PARTICLE_ACC, 1.0, 1 / 128, 2 ** -9, 0.5, 32, amag)
    assert np.all(ng >= npart)


def test_tree_coincident_particles():
    """More coincident particles than a leaf holds: the finest-level leaf keeps
    them all, groups are chunked, and with eps > 0 the sum stays the direct one."""
    p = ics.plummer(500, 13)
    x, y, z, m = (p[k].astype(float) for k in ("x", "y", "z", "m"))
    x[:100], y[:100], z[:100] = 0.25, -0.5, 0.125
    t = oracle.Tree(x, y, z, m, 21, 8)
    nd = t.nodes()
    assert nd["count"][(nd["nchild"] == 0)].max() == 100
    f, c = t.groups(32)
    assert c.max() <= 32 and c.sum() == 500
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, 0.05)
    bx, by, bz, _, _ = t.walk(oracle.MAC_GROUP_ACC, 1.0, 0.05, 0.0, 0.5, 32,
                              np.sqrt(ax ** 2 + ay ** 2 + az ** 2))
    assert np.max(oracle.rel_err(bx, by, bz, ax, ay, az)) < 1e-12


# --------------------------------------------------------------------------- leapfrog, diagnostics
def _kdk(x, v, m, eps, dt, steps):
    a = oracle.direct(*x, m, 1.0, eps, want_phi=False)[:3]
    for _ in range(steps):
        oracle.kick(v, a, dt / 2)
        oracle.drift(x, v, dt)
        a = oracle.direct(*x, m, 1.0, eps, want_phi=False)[:3]
        oracle.kick(v, a, dt / 2)
    return x, v


def test_leapfrog_time_reversible():
    p = ics.plummer(64, 14)
    x = [p[k].astype(float) for k in ("x", "y", "z")]
    v = [p[k].astype(float) for k in ("vx", "vy", "vz")]
    m = p["m"].astype(float)
    x0 = [a.copy() for a in x]
    v0 = [a.copy() for a in v]
    _kdk(x, v, m, 0.05, 1 / 256, 20)
    _kdk(x, v, m, 0.05, -1 / 256, 20)
    for a, b in zip(x + v, x0 + v0):
        assert np.max(np.abs(a - b)) < 1e-11


def test_leapfrog_kepler_energy_second_order():
    """Two-body circular orbit: the energy error of KDK falls as dt^2."""
    def run(dt):
        x = [np.array([0.5, -0.5]), np.array([0.0, 0.0]), np.array([0.0, 0.0])]
        vc = np.sqrt(1.0 / 2.0 / 2.0)  # m = 1 each, separation 1
        v = [np.array([0.0, 0.0]), np.array([vc, -vc]), np.array([0.0, 0.0])]
        m = np.array([1.0, 1.0])
        phi = oracle.direct(*x, m, 1.0, 0.0)[3]
        e0 = oracle.diagnostics(*x, *v, m, phi)
        emax = 0.0
        T = 2 * np.pi / np.sqrt(2.0)
        steps = int(round(T / dt))
        for _ in range(steps // 8):
            _kdk(x, v, m, 0.0, dt, 8)
            phi = oracle.direct(*x, m, 1.0, 0.0)[3]
            e = oracle.diagnostics(*x, *v, m, phi)
            emax = max(emax, abs((e[0] + e[1]) - (e0[0] + e0[1])))
        return emax

    e1, e2 = run(2 ** -6), run(2 ** -7)
    assert 3.0 < e1 / e2 < 5.0


# --------------------------------------------------------------------------- block time steps
def test_block_level_thresholds():
    """dt_i = sqrt(2 eta eps / |a|) <= dt / 2^k: with eta = 1/40, eps = 1/64 and
    dt = 1/256 the level-0 threshold is |a| = 2 eta eps / dt^2 = 51.2 (hand
    value) and every factor 4 above it adds a level, up to the deepest."""
    eta, eps, dt, K = 0.025, 1.0 / 64, 1.0 / 256, 5
    a0 = 2 * eta * eps / dt ** 2
    assert np.isclose(a0, 51.2)
    amag = np.array([0.0, a0 * 0.999, a0 * 1.001, 4 * a0 * 0.999, 4 * a0 * 1.001, 16 * a0 * 1.001,
                     1e9])
    assert list(oracle.block_level(amag, eps, eta, dt, K)) == [0, 0, 1, 1, 2, 3, 5]


def _shared_kdk(x, v, a, m, eps, h, steps):
    x, v, a = [q.copy() for q in x], [q.copy() for q in v], [q.copy() for q in a]
    for _ in range(steps):
        for c in range(3):
            v[c] += a[c] * (h * 0.5)
            x[c] += v[c] * h
        a = list(oracle.direct(*x, m, 1.0, eps, want_phi=False)[:3])
        for c in range(3):
            v[c] += a[c] * (h * 0.5)
    return x, v, a


def _direct_force(m, eps):
    def f(x, idx):
        return oracle.direct_targets(*x, m, idx, 1.0, eps)[:3]
    return f


@pytest.mark.parametrize("eta,fine", [(1e30, False), (1e-30, True)])
def test_block_kdk_single_level_is_shared_kdk(eta, fine):
    """All particles on one level: the block scheme performs exactly the
    operations of the shared-step leapfrog (step dt, or dt/2^K with 2^K times
    as many steps), so the states agree bit for bit."""
    p = ics.plummer(300, 51)
    m = p["m"].astype(float)
    x = [p[k].astype(float) for k in ("x", "y", "z")]
    v = [p[k].astype(float) for k in ("vx", "vy", "vz")]
    eps, dt, K = 1 / 32, 1 / 64, 3
    a = list(oracle.direct(*x, m, 1.0, eps, want_phi=False)[:3])
    bx, bv, ba, lvl, nf = oracle.block_kdk(x, v, m, a, 1.0, eps, dt, 2, K, eta, _direct_force(m, eps))
    assert np.all(lvl == (K if fine else 0))
    sx, sv, sa = _shared_kdk(x, v, a, m, eps, dt / 2 ** K if fine else dt, 2 * 2 ** K if fine else 2)
    for q, r in zip(bx + bv + ba, sx + sv + sa):
        assert np.array_equal(q, r)


def test_block_kdk_every_step_lasts_its_level():
    """The defining invariant of block steps: a particle's consecutive force
    evaluations are exactly one step of its level apart (levels change only at
    the end of a step, and a coarser level only where the clock is a multiple
    of the new step).  An eccentric binary (levels refine towards pericentre
    and coarsen after it) exercises both directions."""
    mb, apo, ecc = 0.5, 0.2, 0.9
    vapo = np.sqrt(2 * mb / apo * (1 - ecc) / 2)  # apocentre speed of each body, reduced-mass orbit
    x = [np.array([-apo / 2, apo / 2, 5.0]), np.zeros(3), np.zeros(3)]
    v = [np.zeros(3), np.array([-vapo / 2 * 2 ** 0.5, vapo / 2 * 2 ** 0.5, 0.3]), np.zeros(3)]
    m = np.array([mb, mb, 1e-6])
    eps, dt, K, eta = 1e-4, 1 / 8, 8, 15.0
    a = list(oracle.direct(*x, m, 1.0, eps, want_phi=False)[:3])
    tr = []
    oracle.block_kdk(x, v, m, a, 1.0, eps, dt, 4, K, eta, _direct_force(m, eps), trace=tr)
    last = {}
    coarsened = refined = 0
    for T, act, lv in tr:
        for i, k in zip(act, lv):
            assert T % (1 << (K - k)) == 0
            if i in last:  # the step [T0, T] ran at level k (recorded at its end)
                T0, k0 = last[i]
                assert T - T0 == 1 << (K - k)
                coarsened += k < k0
                refined += k > k0
            last[i] = (T, k)
    assert coarsened > 0 and refined > 0


def test_block_kdk_binary_and_distant_particles():
    """A tight binary (fine levels) beside a loose cluster (coarse levels):
    the binary's energy is conserved as well as with the fine shared step,
    and the whole system ends close to the fine shared-step run, with far
    fewer force evaluations."""
    g = ics.rng(52)
    nc = 40
    cl = g.normal(scale=1.0, size=(nc, 3)) + np.array([30.0, 0.0, 0.0])
    sep, mb = 0.02, 0.5
    vb = np.sqrt(mb * 2 / sep) / 2  # circular: each moves at sqrt(G M_tot / r) / 2
    x = [np.concatenate([[-sep / 2, sep / 2], cl[:, c]]) for c in range(3)]
    v = [np.concatenate([[0.0, 0.0], np.zeros(nc)]),
         np.concatenate([[-vb, vb], g.normal(scale=0.05, size=nc)]),
         np.concatenate([[0.0, 0.0], np.zeros(nc)])]
    m = np.concatenate([[mb, mb], np.full(nc, 1e-3)])
    eps, dt, K, eta = 1e-4, 1 / 64, 6, 0.02
    a = list(oracle.direct(*x, m, 1.0, eps, want_phi=False)[:3])
    bx, bv, _, lvl, nf = oracle.block_kdk(x, v, m, a, 1.0, eps, dt, 2, K, eta, _direct_force(m, eps))
    assert lvl[:2].min() >= 4 and lvl[2:].max() <= 2
    sx, sv, _ = _shared_kdk(x, v, a, m, eps, dt / 2 ** K, 2 * 2 ** K)
    assert nf < 0.2 * (2 * 2 ** K) * m.size

    def ebin(x_, v_):
        ke = 0.5 * mb * sum(v_[c][0] ** 2 + v_[c][1] ** 2 for c in range(3))
        r = np.sqrt(sum((x_[c][0] - x_[c][1]) ** 2 for c in range(3)) + eps ** 2)
        return ke - mb * mb / r
    e0 = ebin(x, v)
    assert abs(ebin(bx, bv) - e0) / abs(e0) < 2 * abs(ebin(sx, sv) - e0) / abs(e0) + 1e-6
    for c in range(3):
        assert np.max(np.abs(bx[c][2:] - sx[c][2:])) < 1e-6
        assert np.max(np.abs(bx[c][:2] - sx[c][:2])) < 1e-3 * sep


def test_diagnostics_two_body_closed_form():
    x, y, z = np.array([0.0, 3.0]), np.array([0.0, 4.0]), np.zeros(2)
    vx, vy, vz = np.array([1.0, -0.5]), np.array([0.0, 2.0]), np.array([0.5, 0.0])
    m = np.array([1.0, 2.0])
    phi = oracle.direct(x, y, z, m, 1.0, 12.0)[3]
    d = oracle.diagnostics(x, y, z, vx, vy, vz, m, phi)
    ek = 0.5 * 1.0 * (1 + 0.25) + 0.5 * 2.0 * (0.25 + 4)
    ep = -1.0 * 2.0 / 13.0
    assert np.isclose(d[0], ek, rtol=1e-15) and np.isclose(d[1], ep, rtol=1e-15)
    assert np.allclose(d[2:5], [1.0 - 1.0, 0.0 + 4.0, 0.5], rtol=1e-15)
    # L = sum m r x v ; particle 1: r = (3,4,0), v = (-0.5, 2, 0) -> (0, 0, 3*2 - 4*-0.5) = 8, times 2
    assert np.allclose(d[5:], [0.0, 0.0, 16.0], rtol=1e-15)


# --------------------------------------------------------------------------- cost-model MLP
def _mlp_case(seed, n=40):
    g = ics.rng(seed, 3)
    w = ics.mlp_init(seed).astype(np.float64)
    w[8 * 32:8 * 32 + 32] = g.normal(scale=0.1, size=32)          # b1
    w[-1] = 0.3                                                    # b3
    feat = g.normal(size=(n, 8))
    target = g.normal(size=n)
    norm = np.concatenate([g.normal(scale=0.1, size=8), g.uniform(0.5, 2.0, 8)])
    return feat, target, w, norm


def test_mlp_gradient_matches_finite_differences():
    feat, target, w, norm = _mlp_case(1)
    _, grad, loss = oracle.mlp_eval(feat, target, w, norm)
    h = 1e-6
    g = ics.rng(2, 4)
    for p in g.choice(w.size, 60, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[p] += h
        wm[p] -= h
        fd = (oracle.mlp_eval(feat, target, wp, norm, False)[2] -
              oracle.mlp_eval(feat, target, wm, norm, False)[2]) / (2 * h)
        assert abs(fd - grad[p]) <= 1e-6 * max(1.0, abs(grad[p])) + 1e-9, (p, fd, grad[p])


def test_mlp_closed_forms():
    feat, target, w, norm = _mlp_case(3)
    # all weights zero: y = b3, loss = mean (b3 - t)^2, only b3 has a gradient
    z = np.zeros_like(w)
    z[-1] = 0.7
    pred, grad, loss = oracle.mlp_eval(feat, target, z, norm)
    assert np.all(pred == 0.7)
    assert np.isclose(loss, np.mean((0.7 - target) ** 2), rtol=1e-14)
    assert np.isclose(grad[-1], 2 * np.mean(0.7 - target), rtol=1e-14)
    assert np.all(grad[:-1] == 0)
    # a hidden unit with a very negative bias is dead: its weights get no gradient
    w2 = w.copy()
    w2[8 * 32 + 5] = -1e6                                          # b1[5]
    _, g2, _ = oracle.mlp_eval(feat, target, w2, norm)
    assert np.all(g2[5:8 * 32:32] == 0) and g2[8 * 32 + 5] == 0
