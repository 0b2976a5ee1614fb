"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer work (keys, sort, tree structure, groups) must match bit for bit;
floating-point results within the tolerances stated in each test:
  * GPU direct vs FP64 direct: max relative error <= 1e-5 (compensated);
  * GPU tree error percentiles (p50, p99) vs FP64 direct within 1.1x the
    oracle tree's percentiles + 1e-6 (same MAC reading, group mode);
  * the walk against the oracle's walk of the same tree, group by group:
    equal interaction-list lengths except for a few groups, each explained
    by a MAC decision within 1e-5 (relative) of its threshold, and per-
    particle agreement to FP32 rounding (p50 < 1e-6, p99 < 5e-6, max < 1e-4)
    for every member of a group with an equal list.
"""
import numpy as np
import pytest

import ics
import oracle
from _walk_parity import compare_groups, group_entries, group_spheres, visited_margin

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1811_02761_gb300 as nb  # noqa: E402

EPS = 1.0 / 128
DACC = 2.0 ** -9


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def f64(p):
    return [p[k].astype(np.float64) for k in ("x", "y", "z", "m")]


@pytest.fixture(scope="module")
def plummer8k():
    p = ics.plummer(8192, 1)
    x, y, z, m = f64(p)
    ax, ay, az, phi = oracle.direct(x, y, z, m, 1.0, EPS)
    return p, (ax, ay, az, phi)


def gpu_walk(p, cfg, a_old=None, want_phi=False, offsets=None, eps_sys=None):
    ctx = nb.nbody_create(cfg)
    try:
        X = [dev(p[k]) for k in ("x", "y", "z", "m")]
        if offsets is None:
            nb.nbody_build(ctx, *X)
        else:
            nb.nbody_build_batched(ctx, offsets, eps_sys, *X)
        n = X[0].numel()
        out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(4)]
        st = nb.nbody_walk(ctx, None if a_old is None else dev(a_old.astype(np.float32)),
                           out[0], out[1], out[2], out[3] if want_phi else None)
        exports = {w: nb.nbody_export(ctx, w) for w in range(12)}  # all but the quadrupoles
        costs = torch.zeros(max(int(st.n_groups), 1), dtype=torch.int32, device="cuda")
        ng = nb.nbody_get_group_costs(ctx, costs)
        exports["costs"] = host(costs)[:ng]
        return [host(o) for o in out], st, exports
    finally:
        nb.nbody_destroy(ctx)


# --------------------------------------------------------------------------- direct
@pytest.mark.parametrize("compensated", [1, 0])
def test_direct_vs_fp64(plummer8k, compensated):
    p, (ax, ay, az, phi) = plummer8k
    n = p["x"].size
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(4)]
    X = [dev(p[k]) for k in ("x", "y", "z", "m")]
    nb.nbody_direct(*X, 1.0, EPS, compensated, *out)
    gx, gy, gz, gphi = (host(o).astype(np.float64) for o in out)
    e = oracle.rel_err(gx, gy, gz, ax, ay, az)
    if compensated:
        assert e.max() <= 1e-5, e.max()
    else:
        assert e.max() <= 1e-4, e.max()
    assert np.max(np.abs(gphi - phi) / np.abs(phi)) < 1e-5


def test_direct_host_buffers_match_device(plummer8k):
    p, _ = plummer8k
    n = 2000
    q = {k: np.ascontiguousarray(p[k][:n]) for k in ("x", "y", "z", "m")}
    hout = [np.empty(n, np.float32) for _ in range(3)]
    nb.nbody_direct(q["x"], q["y"], q["z"], q["m"], 1.0, EPS, 1, *hout)
    dout = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    nb.nbody_direct(*[dev(q[k]) for k in ("x", "y", "z", "m")], 1.0, EPS, 1, *dout)
    for a, b in zip(hout, dout):
        assert np.array_equal(a, host(b))


# --------------------------------------------------------------------------- keys, sort, tree
def test_keys_and_sort_bit_exact(plummer8k):
    p, (ax, ay, az, _) = plummer8k
    cfg = nb.nbody_config_default(eps=EPS)
    _, _, ex = gpu_walk(p, cfg, a_old=np.sqrt(ax ** 2 + ay ** 2 + az ** 2))
    k, cube = oracle.keys(p["x"], p["y"], p["z"], 21)
    order = oracle.sort_order(k)
    assert np.array_equal(ex[nb.nbody.EXPORT_SYS_BOX][0], cube)
    assert np.array_equal(ex[nb.nbody.EXPORT_PERM], order.astype(np.int32))
    assert np.array_equal(ex[nb.nbody.EXPORT_KEYS], k[order])


def _gpu_nodes(ex):
    lev = ex[nb.nbody.EXPORT_NODE_LEVEL].astype(np.int64)
    start = ex[nb.nbody.EXPORT_NODE_START].astype(np.int64)
    cnt = ex[nb.nbody.EXPORT_NODE_COUNT].astype(np.int64)
    B = ex[nb.nbody.EXPORT_NODE_B]
    leaf = (B[:, 3].view(np.int32) & 1).astype(bool)
    return lev, start, cnt, leaf, ex[nb.nbody.EXPORT_NODE_A], B


@pytest.mark.parametrize("gen,n,cap", [(ics.plummer, 8192, 16), (ics.galaxy, 20000, 8),
                                       (ics.hernquist, 5000, 32)])
def test_tree_structure_and_moments(gen, n, cap):
    p = gen(n, 3)
    cfg = nb.nbody_config_default(eps=EPS, leaf_cap=cap, group_size=max(cap, 32))
    _, _, ex = gpu_walk(p, cfg, a_old=np.ones(n))
    t = oracle.Tree(*f64(p), levels=21, leaf_cap=cap)
    on = t.nodes()
    lev, start, cnt, leaf, A, B = _gpu_nodes(ex)
    # identical node sets (the oracle's tree order equals the sorted order)
    g = sorted(zip(lev, start, cnt, leaf))
    o = sorted(zip(on["level"].astype(np.int64), on["first"], on["count"], on["nchild"] == 0))
    assert g == o
    # level-major order with contiguous children
    assert np.all(np.diff(lev) >= 0)
    # moments: match nodes by (level, start)
    key_o = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(on["level"], on["first"]))}
    idx = np.array([key_o[(int(a), int(b))] for a, b in zip(lev, start)])
    assert np.allclose(A[:, 3], on["M"][idx], rtol=2e-6)
    for c, k in ((0, "cx"), (1, "cy"), (2, "cz")):
        scale = np.maximum(np.abs(on[k][idx]), on["b"][idx] + 1e-3)
        assert np.all(np.abs(A[:, c] - on[k][idx]) <= 2e-6 * scale)
    # b_J is an upper bound (Eq. 2's node size; the MAC's d > b_J must never
    # accept a node that can hold the target): the GPU's b_J covers, with no
    # slack, the exact (FP64) largest distance of the node's members from the
    # GPU's own FP32 centre of mass, and exceeds the oracle's b_J by rounding only
    perm = ex[nb.nbody.EXPORT_PERM].astype(np.int64)
    P = np.stack([p[k][perm].astype(np.float64) for k in ("x", "y", "z")], 1)
    rows = np.repeat(np.arange(lev.size), cnt)
    mem = np.concatenate([np.arange(a, a + c) for a, c in zip(start, cnt)])
    dist = np.sqrt(((P[mem] - A[rows, :3].astype(np.float64)) ** 2).sum(1))
    exact = np.zeros(lev.size)
    np.maximum.at(exact, rows, dist)
    assert np.all(B[:, 0].astype(np.float64) >= exact), np.min(B[:, 0] - exact)
    b_o = on["b"][idx]
    ulp = np.spacing(np.max(np.abs(A[:, :3]), axis=1).astype(np.float32)).astype(np.float64)
    assert np.all(B[:, 0] <= b_o * (1 + 1e-5) + 8 * ulp)


def test_groups_bit_exact(plummer8k):
    p, _ = plummer8k
    for G, ipl in ((32, 1), (64, 2), (128, 4)):
        cfg = nb.nbody_config_default(eps=EPS, group_size=G, ipl=ipl)
        _, _, ex = gpu_walk(p, cfg, a_old=np.ones(p["x"].size))
        t = oracle.Tree(*f64(p), levels=21, leaf_cap=16)
        f, c = t.groups(G)
        assert np.array_equal(ex[nb.nbody.EXPORT_GROUP_FIRST], f.astype(np.int32))
        assert np.array_equal(ex[nb.nbody.EXPORT_GROUP_COUNT], c.astype(np.int32))


# --------------------------------------------------------------------------- walk
def _pcts(e):
    return oracle.percentile_nearest_rank(e, 50), oracle.percentile_nearest_rank(e, 99)


@pytest.mark.parametrize("ipl,G", [(1, 32), (2, 64), (4, 128), (2, 32)])
def test_walk_error_vs_oracle_tree(plummer8k, ipl, G):
    p, (ax, ay, az, phi) = plummer8k
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2)
    aold32 = amag.astype(np.float32)
    cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC, ipl=ipl, group_size=G)
    (gx, gy, gz, _), st, ex = gpu_walk(p, cfg, a_old=aold32)
    t = oracle.Tree(*f64(p), levels=21, leaf_cap=16)
    ox, oy, oz, _, nint = t.walk(oracle.MAC_GROUP_ACC, 1.0, EPS, DACC, 0.5, G,
                                 aold32.astype(np.float64))
    eg = oracle.rel_err(gx.astype(float), gy.astype(float), gz.astype(float), ax, ay, az)
    eo = oracle.rel_err(ox, oy, oz, ax, ay, az)
    g50, g99 = _pcts(eg)
    o50, o99 = _pcts(eo)
    assert g50 <= 1.1 * o50 + 1e-6, (g50, o50)
    assert g99 <= 1.1 * o99 + 1e-6, (g99, o99)
    # same tree, same groups, same MAC: group by group, the list lengths are
    # the oracle's except where a MAC decision is within FP32 rounding of its
    # threshold, and the accelerations agree per particle up to FP32 rounding
    check_walk_against_oracle_tree(p, t, ex, nint, aold32, G, (gx, gy, gz), (ox, oy, oz))
    assert abs(st.interactions - nint.sum()) <= 0.01 * nint.sum()


def check_walk_against_oracle_tree(p, t, ex, nint, aold32, G, gpu_acc, ora_acc, dacc=DACC,
                                   grav=1.0):
    """Per-group list lengths and per-particle accelerations of a GPU walk
    against the oracle's walk of the same tree (group mode, same a_old)."""
    first = ex[nb.nbody.EXPORT_GROUP_FIRST].astype(np.int64)
    count = ex[nb.nbody.EXPORT_GROUP_COUNT].astype(np.int64)
    f, c = t.groups(G)
    assert np.array_equal(first, f) and np.array_equal(count, c)
    order = t.order()
    ora = group_entries(nint, order, first)
    x, y, z, _ = f64(p)
    cen, rad, amin = group_spheres(x, y, z, order, first, count, aold32.astype(np.float64))
    nodes = t.nodes()
    flipped, margins = compare_groups(
        ex["costs"], ora, flipped_budget=max(3, first.size // 200),
        explain=lambda g: visited_margin(nodes, cen[g], rad[g], dacc * amin[g], grav))
    d = oracle.rel_err(*[a.astype(float) for a in gpu_acc], *ora_acc)
    same = np.ones(d.size, bool)
    for g in flipped:
        same[order[first[g]:first[g] + count[g]]] = False
    ds = d[same]
    print(f"groups {first.size}, flipped {flipped.size} (margins {margins}); "
          f"same-list particles: p50 {np.median(ds):.2e} p99 {np.percentile(ds, 99):.2e} "
          f"max {ds.max():.2e}; all: max {d.max():.2e}")
    assert np.median(ds) < 1e-6 and np.percentile(ds, 99) < 5e-6 and ds.max() < 1e-4


def test_walk_bootstrap_without_a_old(plummer8k):
    p, (ax, ay, az, _) = plummer8k
    cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC)
    (gx, gy, gz, _), st, _ = gpu_walk(p, cfg, a_old=None)
    t = oracle.Tree(*f64(p), levels=21, leaf_cap=16)
    bx, by, bz, _, _ = t.walk(oracle.MAC_GROUP_GEO, 1.0, EPS, 0.0, 0.5, 64, None, want_phi=False)
    a0 = np.sqrt(bx ** 2 + by ** 2 + bz ** 2).astype(np.float32).astype(np.float64)
    ox, oy, oz, _, _ = t.walk(oracle.MAC_GROUP_ACC, 1.0, EPS, DACC, 0.5, 64, a0, want_phi=False)
    eg = oracle.rel_err(gx.astype(float), gy.astype(float), gz.astype(float), ax, ay, az)
    eo = oracle.rel_err(ox, oy, oz, ax, ay, az)
    (g50, g99), (o50, o99) = _pcts(eg), _pcts(eo)
    assert g50 <= 1.1 * o50 + 1e-6 and g99 <= 1.1 * o99 + 1e-6


def test_walk_potential_and_compensation(plummer8k):
    p, (ax, ay, az, phi) = plummer8k
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2).astype(np.float32)
    t = oracle.Tree(*f64(p), levels=21, leaf_cap=16)
    ox, oy, oz, ophi, _ = t.walk(oracle.MAC_GROUP_ACC, 1.0, EPS, DACC, 0.5, 64, amag.astype(float))
    res = {}
    for comp in (0, 1):
        cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC, want_potential=1, compensated=comp)
        (gx, gy, gz, gphi), _, _ = gpu_walk(p, cfg, a_old=amag, want_phi=True)
        assert np.median(np.abs(gphi - ophi) / np.abs(ophi)) < 2e-6
        res[comp] = oracle.rel_err(gx.astype(float), gy.astype(float), gz.astype(float), ox, oy, oz)
    # compensation cannot make the agreement with the FP64 tree worse on average
    assert np.mean(res[1]) <= np.mean(res[0]) * 1.05 + 1e-9


def test_walk_deterministic(plummer8k):
    p, (ax, ay, az, _) = plummer8k
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2).astype(np.float32)
    cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC)
    (a1, _, _, _), _, _ = gpu_walk(p, cfg, a_old=amag)
    (a2, _, _, _), _, _ = gpu_walk(p, cfg, a_old=amag)
    assert np.array_equal(a1, a2)


@pytest.mark.parametrize("wpb,stack,depth", [(3, 97, 96), (1, 65, 64), (16, 130, 128)])
def test_walk_launch_shape_does_not_change_forces(plummer8k, wpb, stack, depth):
    """Warps per CTA, stack depth (also ones that are not a multiple of 4) and
    list depth change only how the groups are laid out on the GPU, and the
    flush points, never a group's traversal: the MAC decisions and the
    interaction count are identical and the forces agree to rounding."""
    p, (ax, ay, az, _) = plummer8k
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2).astype(np.float32)
    base = nb.nbody_config_default(eps=EPS, delta_acc=DACC)
    (a1, _, _, _), st1, _ = gpu_walk(p, base, a_old=amag)
    cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC, warps_per_block=wpb,
                                  stack_depth=stack, list_depth=depth)
    (a2, _, _, _), st2, _ = gpu_walk(p, cfg, a_old=amag)
    assert st1.interactions == st2.interactions
    assert np.max(np.abs(a1 - a2)) <= 1e-5 * np.max(np.abs(a1))


# --------------------------------------------------------------------------- edge cases
@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 100, 8192 + 13])
def test_walk_small_and_ragged_n(n):
    p = ics.plummer(n, 5)
    x, y, z, m = f64(p)
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, 0.05)
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2)
    cfg = nb.nbody_config_default(eps=0.05, delta_acc=DACC)
    a32 = amag.astype(np.float32)
    (gx, gy, gz, _), _, ex = gpu_walk(p, cfg, a_old=a32)
    if n == 1:
        assert gx[0] == 0 and gy[0] == 0 and gz[0] == 0
        return
    t = oracle.Tree(x, y, z, m, 21, 16)
    ox, oy, oz, _, nint = t.walk(oracle.MAC_GROUP_ACC, 1.0, 0.05, DACC, 0.5, 64,
                                 a32.astype(float))
    check_walk_against_oracle_tree(p, t, ex, nint, a32, 64, (gx, gy, gz), (ox, oy, oz))


def test_walk_coincident_particles():
    p = ics.plummer(3000, 6)
    for k in ("x", "y", "z"):
        p[k][:200] = p[k][0]
    x, y, z, m = f64(p)
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, 0.05)
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2)
    cfg = nb.nbody_config_default(eps=0.05, delta_acc=0.0)
    (gx, gy, gz, _), _, ex = gpu_walk(p, cfg, a_old=amag)
    assert ex[nb.nbody.EXPORT_GROUP_COUNT].max() <= 64
    e = oracle.rel_err(gx.astype(float), gy.astype(float), gz.astype(float), ax, ay, az)
    assert e.max() < 1e-4


def test_walk_zero_softening():
    g = ics.rng(9)
    n = 2000
    p = {k: g.normal(size=n).astype(np.float32) for k in ("x", "y", "z")}
    p["m"] = np.full(n, 1.0 / n, np.float32)
    x, y, z, m = f64(p)
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, 0.0)
    cfg = nb.nbody_config_default(eps=0.0, delta_acc=0.0)
    (gx, gy, gz, _), _, _ = gpu_walk(p, cfg, a_old=np.sqrt(ax ** 2 + ay ** 2 + az ** 2))
    e = oracle.rel_err(gx.astype(float), gy.astype(float), gz.astype(float), ax, ay, az)
    assert np.all(np.isfinite(gx)) and np.median(e) < 1e-5


# --------------------------------------------------------------------------- batched
def test_batched_forest_matches_per_system_oracle():
    sizes = [1, 20, 700, 3000, 65, 1, 0, 4096]
    b = ics.batched(len(sizes), 7, sizes=sizes)
    off, eps = b["offsets"], b["eps"]
    n = int(off[-1])
    cfg = nb.nbody_config_default(delta_acc=DACC)
    # |a_old| from each system's own direct sum
    aold = np.zeros(n)
    for s in range(len(sizes)):
        sl = slice(off[s], off[s + 1])
        if off[s + 1] - off[s] < 2:
            continue
        ax, ay, az, _ = oracle.direct(*[b[k][sl].astype(float) for k in ("x", "y", "z", "m")],
                                      1.0, float(eps[s]), want_phi=False)
        aold[sl] = np.sqrt(ax ** 2 + ay ** 2 + az ** 2)
    (gx, gy, gz, _), _, ex = gpu_walk(b, cfg, a_old=aold, offsets=off, eps_sys=eps)
    levels = 63 // 3 if len(sizes) == 1 else (63 - int(np.ceil(np.log2(len(sizes))))) // 3
    for s in range(len(sizes)):
        sl = slice(off[s], off[s + 1])
        ns = off[s + 1] - off[s]
        if ns == 0:
            continue
        if ns == 1:
            assert gx[sl][0] == 0
            continue
        t = oracle.Tree(*[b[k][sl].astype(float) for k in ("x", "y", "z", "m")], levels=levels,
                        leaf_cap=16)
        a32 = aold[sl].astype(np.float32)
        ox, oy, oz, _, nint = t.walk(oracle.MAC_GROUP_ACC, 1.0, float(eps[s]), DACC, 0.5, 64,
                                     a32.astype(float), want_phi=False)
        # this system's groups of the forest (sorted order keeps each system in
        # its own index range), renumbered from the system's first particle
        gf = ex[nb.nbody.EXPORT_GROUP_FIRST].astype(np.int64)
        mine = (gf >= off[s]) & (gf < off[s + 1])
        sub = {nb.nbody.EXPORT_GROUP_FIRST: gf[mine] - off[s],
               nb.nbody.EXPORT_GROUP_COUNT: ex[nb.nbody.EXPORT_GROUP_COUNT][mine],
               "costs": ex["costs"][mine]}
        ps = {k: b[k][sl] for k in ("x", "y", "z", "m")}
        check_walk_against_oracle_tree(ps, t, sub, nint, a32, 64,
                                       (gx[sl], gy[sl], gz[sl]), (ox, oy, oz))


# --------------------------------------------------------------------------- step, diagnostics
def test_step_one_kdk_vs_oracle():
    p = ics.plummer(4096, 8)
    n = p["x"].size
    x, y, z, m = f64(p)
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, EPS)
    a0 = [a.astype(np.float32) for a in (ax, ay, az)]
    dt = 1.0 / 256
    cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC)
    ctx = nb.nbody_create(cfg)
    try:
        X = [dev(a) for a in (x, y, z)]
        V = [dev(p[k]) for k in ("vx", "vy", "vz")]
        A = [dev(a) for a in a0]
        nb.nbody_step(ctx, *X, *V, dev(p["m"]), *A, dt, 1)
        gx, gy, gz = (host(t) for t in X)
        gv = [host(t) for t in V]
        ga = [host(t) for t in A]
    finally:
        nb.nbody_destroy(ctx)
    # oracle leapfrog with the same entry accelerations and the oracle tree force
    vh = [p[k].astype(float) + a.astype(float) * dt / 2 for k, a in zip(("vx", "vy", "vz"), a0)]
    x1 = [q + v * dt for q, v in zip((x, y, z), vh)]
    assert np.max(np.abs(gx - x1[0])) < 1e-9 and np.max(np.abs(gz - x1[2])) < 1e-9
    t = oracle.Tree(*x1, m, 21, 16)
    amag = np.sqrt(sum(a.astype(float) ** 2 for a in a0)).astype(np.float32).astype(float)
    ox, oy, oz, _, _ = t.walk(oracle.MAC_GROUP_ACC, 1.0, EPS, DACC, 0.5, 64, amag, want_phi=False)
    d = oracle.rel_err(ga[0].astype(float), ga[1].astype(float), ga[2].astype(float), ox, oy, oz)
    assert np.median(d) < 5e-6 and np.percentile(d, 99) < 1e-4, (np.median(d), np.percentile(d, 99))
    v1 = [v + a * dt / 2 for v, a in zip(vh, (ox, oy, oz))]
    assert np.max(np.abs(gv[0] - v1[0])) < 1e-5 * np.max(np.abs(v1[0]))


def test_diagnostics_vs_oracle(plummer8k):
    p, (_, _, _, phi) = plummer8k
    x, y, z, m = f64(p)
    ref = oracle.diagnostics(x, y, z, p["vx"], p["vy"], p["vz"], m, phi.astype(np.float32))
    ctx = nb.nbody_create(nb.nbody_config_default())
    try:
        got = nb.nbody_diagnostics(ctx, dev(x), dev(y), dev(z), dev(p["vx"]), dev(p["vy"]),
                                   dev(p["vz"]), dev(p["m"]), dev(phi.astype(np.float32)))
    finally:
        nb.nbody_destroy(ctx)
    scale = np.array([abs(ref[0]), abs(ref[1])] + [np.abs(ref[2:5]).max() + 1e-3] * 3 +
                     [np.abs(ref[5:]).max() + 1e-3] * 3)
    assert np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-15)


def test_bad_arguments_rejected_on_gpu():
    ctx = nb.nbody_create(nb.nbody_config_default())
    try:
        out = [torch.empty(4, device="cuda") for _ in range(3)]
        with pytest.raises(nb.NbodyError) as e:
            nb.nbody_walk(ctx, None, *out)
        assert e.value.status == nb.NBODY_ENOTBUILT
        with pytest.raises(nb.NbodyError) as e:
            nb.nbody_build_batched(ctx, [0, 5, 3], None, *[torch.zeros(3, device="cuda")] * 4)
        assert e.value.status == nb.NBODY_EINVAL
    finally:
        nb.nbody_destroy(ctx)


def test_sort_lookback_wait_is_bounded(plummer8k):
    """The one-sweep sort's look-back is the library's only device wait.  The
    self-test gives it a predecessor tile that never publishes: the wait must
    run out, be reported as ETIMEOUT, and leave the device usable."""
    import time
    t0 = time.perf_counter()
    assert nb.nbody_selftest(nb.nbody.SELFTEST_SORT_WAIT) == nb.NBODY_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert "ran out" in nb.nbody_last_error()
    assert nb.nbody_selftest(99) == nb.NBODY_EINVAL
    # the device still answers: a normal build and walk afterwards succeed
    p, _ = plummer8k
    X = [dev(p[k]) for k in ("x", "y", "z", "m")]
    ctx = nb.nbody_create(nb.nbody_config_default(eps=1 / 128))
    try:
        nb.nbody_build(ctx, *X)
        out = [torch.empty(X[0].numel(), device="cuda") for _ in range(3)]
        nb.nbody_walk(ctx, None, *out)
        assert all(torch.isfinite(o).all() for o in out)
    finally:
        nb.nbody_destroy(ctx)


# --------------------------------------------------------------------------- CUDA graph
@pytest.mark.parametrize("nsteps,schedule", [(4, 0), (5, 0), (4, 1), (5, 2)])
def test_step_graph_equals_eager(nsteps, schedule):
    """The two-step CUDA graph replays exactly the eager launch sequence, also
    with a cost-ordered queue (the ordering reads the group count on the
    device, so it is captured with the step)."""
    sizes = [3000, 1, 700, 5000, 20000]
    b = ics.batched(len(sizes), 9, sizes=sizes)
    n = int(b["offsets"][-1])
    res = []
    for graph in (0, 1):
        ctx = nb.nbody_create(nb.nbody_config_default(delta_acc=DACC, use_graph=graph,
                                                      group_size=32, ipl=1, schedule=schedule))
        if schedule == nb.SCHED_MLP:
            nb.nbody_mlp_set_params(ctx, ics.mlp_init(3))
        try:
            X = [dev(b[k].astype(np.float64)) for k in ("x", "y", "z")]
            V = [dev(b[k]) for k in ("vx", "vy", "vz")]
            A = [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(3)]
            m = dev(b["m"])
            nb.nbody_step_batched(ctx, b["offsets"], b["eps"], *X, *V, m, *A, 1.0 / 256, 1)
            st = nb.nbody_step_batched(ctx, b["offsets"], b["eps"], *X, *V, m, *A, 1.0 / 256, nsteps)
            # a second call replays the cached graph
            st2 = nb.nbody_step_batched(ctx, b["offsets"], b["eps"], *X, *V, m, *A, 1.0 / 256, nsteps)
            res.append([host(t) for t in X + V + A] + [st.interactions, st2.interactions])
        finally:
            nb.nbody_destroy(ctx)
    for a, g in zip(res[0][:-2], res[1][:-2]):
        assert np.array_equal(a, g)
    assert res[0][-2:] == res[1][-2:]


# --------------------------------------------------------------------------- checkpoint / resume
def test_resume_from_saved_state_is_bit_identical(tmp_path):
    """The library keeps no integrator state between nbody_step calls: the
    caller's arrays (FP64 positions, velocities, accelerations) are the whole
    state, so saving them and resuming in a new context continues the
    trajectory bit for bit -- also with the learned queue order, whose
    parameters round-trip through nbody_mlp_get/set_params."""
    n = 12000
    p = ics.plummer(n, 91)
    for schedule in (nb.SCHED_MORTON, nb.SCHED_MLP):
        cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC, group_size=32, ipl=1,
                                      schedule=schedule)

        def fresh():
            ctx = nb.nbody_create(cfg)
            if schedule == nb.SCHED_MLP:
                nb.nbody_mlp_set_params(ctx, ics.mlp_init(5))
            return ctx

        def start():
            X = [dev(p[k].astype(np.float64)) for k in ("x", "y", "z")]
            V = [dev(p[k]) for k in ("vx", "vy", "vz")]
            A = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
            return X, V, A

        M = dev(p["m"])
        # reference: four steps in one call
        ctx = fresh()
        X, V, A = start()
        nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z")], M)
        nb.nbody_walk(ctx, None, *A)
        A0 = [a.clone() for a in A]
        nb.nbody_step(ctx, *X, *V, M, *A, 1.0 / 256, 4)
        ref = [host(t) for t in X + V + A]
        nb.nbody_destroy(ctx)
        # two steps, a checkpoint on disk, a new context, two more steps
        ctx = fresh()
        X, V, A = start()
        for a, a0 in zip(A, A0):
            a.copy_(a0)
        nb.nbody_step(ctx, *X, *V, M, *A, 1.0 / 256, 2)
        params = nb.nbody_mlp_get_params(ctx) if schedule == nb.SCHED_MLP else None
        ck = tmp_path / f"state{schedule}.npz"
        np.savez(ck, *[host(t) for t in X + V + A])
        nb.nbody_destroy(ctx)
        saved = np.load(ck)
        T = [dev(saved[f"arr_{k}"]) for k in range(9)]
        ctx = nb.nbody_create(cfg)
        if params is not None:
            nb.nbody_mlp_set_params(ctx, params)
        nb.nbody_step(ctx, *T[:3], *T[3:6], M, *T[6:9], 1.0 / 256, 2)
        nb.nbody_destroy(ctx)
        for r, t in zip(ref, T):
            assert np.array_equal(r, host(t))


def test_step_on_host_arrays_matches_device_arrays():
    """nbody_step on page-locked host tensors (read and written in place by the
    state load and the closing gather) and on pageable numpy arrays (staged
    through device copies) leaves the same state, bit for bit, as the same
    steps on device tensors."""
    n = 20000
    p = ics.plummer(n, 17)
    cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC)

    def run(kind):
        ctx = nb.nbody_create(cfg)
        A = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
        nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z")], dev(p["m"]))
        nb.nbody_walk(ctx, None, *A)
        arrs = [p[k].astype(np.float64) for k in ("x", "y", "z")]
        arrs += [p[k].copy() for k in ("vx", "vy", "vz")] + [host(a) for a in A]
        m = np.ascontiguousarray(p["m"])
        if kind == "device":
            T, mt = [dev(a) for a in arrs], dev(m)
        elif kind == "pinned":
            T = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrs]
            mt = torch.from_numpy(m).pin_memory()
        else:
            T, mt = [np.ascontiguousarray(a) for a in arrs], m
        nb.nbody_step(ctx, *T[:3], *T[3:6], mt, *T[6:9], 1.0 / 256, 3)
        nb.nbody_destroy(ctx)
        return [t.cpu().numpy() if isinstance(t, torch.Tensor) else t for t in T]

    ref = run("device")
    for kind in ("pinned", "pageable"):
        for r, g in zip(ref, run(kind)):
            assert np.array_equal(r, g), kind


def test_batched_step_on_host_arrays_matches_device_arrays():
    """The same for nbody_step_batched over a forest of uneven systems."""
    sizes = [3000, 1, 700, 5000]
    b = ics.batched(len(sizes), 13, sizes=sizes)
    n = int(b["offsets"][-1])
    cfg = nb.nbody_config_default(delta_acc=DACC)

    def run(kind):
        arrs = [b[k].astype(np.float64) for k in ("x", "y", "z")]
        arrs += [b[k].copy() for k in ("vx", "vy", "vz")] + [np.zeros(n, np.float32)] * 3
        m = np.ascontiguousarray(b["m"])
        if kind == "device":
            T, mt = [dev(a) for a in arrs], dev(m)
        elif kind == "pinned":
            T = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrs]
            mt = torch.from_numpy(m).pin_memory()
        else:
            T, mt = [np.array(a) for a in arrs], m
        ctx = nb.nbody_create(cfg)
        try:
            for _ in range(2):
                nb.nbody_step_batched(ctx, b["offsets"], b["eps"], *T[:3], *T[3:6], mt, *T[6:9],
                                      1.0 / 256, 2)
        finally:
            nb.nbody_destroy(ctx)
        return [t.cpu().numpy() if isinstance(t, torch.Tensor) else t for t in T]

    ref = run("device")
    for kind in ("pinned", "pageable"):
        for r, g in zip(ref, run(kind)):
            assert np.array_equal(r, g), kind
