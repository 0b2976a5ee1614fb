"""Parity at the benchmark's full size (three-component galaxy, N = 2^23), in
the launch configuration bench.py times, on sampled outputs the oracle can
compute one by one:
  * GPU tree accelerations vs FP64 direct summation on 384 seeded targets;
  * the same targets through the FP64 oracle tree (walking only the groups
    that hold them) -- p50/p99 of the GPU within 1.1x the oracle's + 1e-6;
  * group by group over those groups: the GPU's list lengths equal the
    oracle's except where a MAC decision sits within FP32 rounding of its
    threshold, and every member of a group with an equal list agrees with
    the oracle tree per particle to FP32 rounding (p50, p99 and max);
  * tree invariants that hold at any size (node count, leaf coverage).
"""
import numpy as np
import pytest

import ics
import oracle
from _walk_parity import compare_groups, group_entries, group_spheres, visited_margin

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1811_02761_gb300 as nb  # noqa: E402

N = 1 << 23
EPS, DACC, DT = 1.0 / 64, 2.0 ** -9, 1.0 / 256


@pytest.fixture(scope="module")
def full():
    """One leapfrog step exactly as the benchmark launches it (default config,
    bootstrap accelerations first), then the accelerations the step returns
    at its final positions."""
    p = ics.galaxy(N, 2)

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    X64 = [D(p[k]) for k in ("x64", "y64", "z64")]
    V = [D(p[k]) for k in ("vx", "vy", "vz")]
    M = D(p["m"])
    A = [torch.empty(N, dtype=torch.float32, device="cuda") for _ in range(3)]
    ctx = nb.nbody_create(nb.nbody_config_default(eps=EPS, delta_acc=DACC))
    try:
        nb.nbody_build(ctx, *[D(p[k]) for k in ("x", "y", "z")], M)
        nb.nbody_walk(ctx, None, *A)                         # bootstrap |a|
        amag = torch.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2).cpu().numpy()
        nb.nbody_step(ctx, *X64, *V, M, *A, DT, 1)          # walk with |a| inside
        g = [a.cpu().numpy().astype(np.float64) for a in A]
        P32 = [x.float() for x in X64]
        pos = [x.cpu().numpy().astype(np.float64) for x in P32]
        # the step leaves no caller-order tree behind: rebuild at the final
        # positions (same FP32 rounding as inside the step) for the exports
        nb.nbody_build(ctx, *P32, M)
        W = [torch.empty_like(a) for a in A]
        st = nb.nbody_walk(ctx, torch.from_numpy(amag).cuda(), *W)
        w = [a.cpu().numpy().astype(np.float64) for a in W]
        ex = {k: nb.nbody_export(ctx, k) for k in (nb.nbody.EXPORT_NODE_COUNT,
                                                   nb.nbody.EXPORT_NODE_B,
                                                   nb.nbody.EXPORT_GROUP_FIRST,
                                                   nb.nbody.EXPORT_GROUP_COUNT)}
        costs = torch.zeros(int(st.n_groups), dtype=torch.int32, device="cuda")
        ng = nb.nbody_get_group_costs(ctx, costs)
        ex["costs"] = costs.cpu().numpy()[:ng]
    finally:
        nb.nbody_destroy(ctx)
    return pos, p["m"].astype(np.float64), g, w, amag, st, ex


def test_fullsize_tree_invariants(full):
    pos, m, g, w, amag, st, ex = full
    cnt = ex[nb.nbody.EXPORT_NODE_COUNT].astype(np.int64)
    leaf = (ex[nb.nbody.EXPORT_NODE_B][:, 3].view(np.int32) & 1).astype(bool)
    assert cnt[leaf].sum() == N                    # every particle in one leaf
    assert cnt[0] == N                             # the root holds everything
    assert ex[nb.nbody.EXPORT_GROUP_COUNT].sum() == N
    assert st.max_stack < nb.nbody_config_default().stack_depth
    assert np.all(np.isfinite(g[0]))
    # a plain build + walk at the step's final positions reproduces the step
    d = oracle.rel_err(*g, *w)
    # (summation order inside leaves and ulp-level |a_old| may differ; a MAC
    # decision flipped by one ulp moves a particle by about the tree error)
    assert np.median(d) < 1e-6 and np.percentile(d, 99) < 1e-5 and d.max() < 1e-2, \
        (np.median(d), np.percentile(d, 99), d.max())


def test_fullsize_sampled_parity(full):
    (x, y, z), m, g, w, amag, st, ex = full
    tg = ics.rng(2, 77).choice(N, 384, replace=False)
    bx, by, bz, _ = oracle.direct_targets(x, y, z, m, tg, 1.0, EPS)
    eg = oracle.rel_err(g[0][tg], g[1][tg], g[2][tg], bx, by, bz)
    # the oracle tree on the groups holding the targets, same a_old
    t = oracle.Tree(x, y, z, m, 21, 16)
    f, c = t.groups(64)
    pos = np.empty(N, np.int64)
    pos[t.order()] = np.arange(N)
    sel = np.unique(np.searchsorted(f, pos[tg], side="right") - 1)
    ox, oy, oz, nint = t.walk_groups(sel, oracle.MAC_GROUP_ACC, 1.0, EPS, DACC, 0.5, 64,
                                     amag.astype(np.float64))
    eo = oracle.rel_err(ox[tg], oy[tg], oz[tg], bx, by, bz)
    for q in (50, 99):
        pg = oracle.percentile_nearest_rank(eg, q)
        po = oracle.percentile_nearest_rank(eo, q)
        assert pg <= 1.1 * po + 1e-6, (q, pg, po)
    d = oracle.rel_err(g[0][tg], g[1][tg], g[2][tg], ox[tg], oy[tg], oz[tg])
    assert np.median(d) < 5e-6
    # the GPU's groups are the oracle's groups
    assert np.array_equal(ex[nb.nbody.EXPORT_GROUP_FIRST], f.astype(np.int32))
    assert np.array_equal(ex[nb.nbody.EXPORT_GROUP_COUNT], c.astype(np.int32))
    # group by group over the walked groups: the list lengths of the plain
    # walk at these positions are the oracle's except at near-threshold MAC
    # decisions, and its accelerations agree per particle up to FP32 rounding
    order = t.order()
    ora = group_entries(nint, order, f[sel])
    cen, rad, amin = group_spheres(x, y, z, order, f[sel], c[sel], amag.astype(np.float64))
    nodes = t.nodes()
    flipped, margins = compare_groups(
        ex["costs"][sel], ora, flipped_budget=max(3, sel.size // 100),
        explain=lambda k: visited_margin(nodes, cen[k], rad[k], DACC * amin[k], 1.0))
    keep = np.setdiff1d(np.arange(sel.size), flipped)
    members = np.concatenate([order[f[gi]:f[gi] + c[gi]] for gi in sel[keep]])
    dw = oracle.rel_err(w[0][members], w[1][members], w[2][members],
                        ox[members], oy[members], oz[members])
    print(f"walked groups {sel.size}, flipped {flipped.size} (margins {margins}); same-list "
          f"particles {members.size}: p50 {np.median(dw):.2e} p99 {np.percentile(dw, 99):.2e} "
          f"max {dw.max():.2e}")
    assert np.median(dw) < 1e-6 and np.percentile(dw, 99) < 5e-6 and dw.max() < 1e-4


def test_fullsize_batched_sampled_parity():
    """The batched workload at its full size (512 Plummer/Hernquist systems,
    about 6.9M particles, the benchmark's seed): one forest step exactly as the
    benchmark launches its steps (one sort, one forest, one persistent walk),
    then sampled accelerations of 24 seeded systems against each system's
    FP64 direct sum and its own oracle tree (same a_old, the forest's depth
    of 18 levels), by the p50/p99 rule."""
    b = ics.batched(512, 4)
    off, eps = b["offsets"], b["eps"]
    n = int(off[-1])

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    X64 = [D(b[k].astype(np.float64)) for k in ("x", "y", "z")]
    V = [D(b[k]) for k in ("vx", "vy", "vz")]
    M = D(b["m"])
    A = [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    ctx = nb.nbody_create(nb.nbody_config_default(delta_acc=DACC))
    try:
        nb.nbody_build_batched(ctx, off, eps, *[D(b[k]) for k in ("x", "y", "z")], M)
        nb.nbody_walk(ctx, None, *A)
        amag = torch.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2).cpu().numpy()
        nb.nbody_step_batched(ctx, off, eps, *X64, *V, M, *A, DT, 1)
        g = [a.cpu().numpy().astype(np.float64) for a in A]
        pos = [x.float().cpu().numpy().astype(np.float64) for x in X64]
    finally:
        nb.nbody_destroy(ctx)
    m = b["m"].astype(np.float64)
    levels = (63 - 9) // 3
    r = ics.rng(4, 78)
    systems = r.choice(512, 24, replace=False)
    eg, eo = [], []
    for s in systems:
        sl = slice(int(off[s]), int(off[s + 1]))
        ns = off[s + 1] - off[s]
        if ns < 2:
            continue
        xs = [q[sl] for q in pos]
        tg = r.choice(ns, min(16, ns), replace=False)
        bx, by, bz, _ = oracle.direct_targets(*xs, m[sl], tg, 1.0, float(eps[s]))
        eg.append(oracle.rel_err(g[0][sl][tg], g[1][sl][tg], g[2][sl][tg], bx, by, bz))
        t = oracle.Tree(*xs, m[sl], levels, 16)
        f, c = t.groups(64)
        where = np.empty(ns, np.int64)
        where[t.order()] = np.arange(ns)
        sel = np.unique(np.searchsorted(f, where[tg], side="right") - 1)
        ox, oy, oz, _ = t.walk_groups(sel, oracle.MAC_GROUP_ACC, 1.0, float(eps[s]), DACC, 0.5, 64,
                                      amag[sl].astype(np.float64))
        eo.append(oracle.rel_err(ox[tg], oy[tg], oz[tg], bx, by, bz))
    eg, eo = np.concatenate(eg), np.concatenate(eo)
    assert eg.size >= 300
    for q in (50, 99):
        pg, po = oracle.percentile_nearest_rank(eg, q), oracle.percentile_nearest_rank(eo, q)
        assert pg <= 1.1 * po + 1e-6, (q, pg, po)
