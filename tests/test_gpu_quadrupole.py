"""Quadrupole nodes on the GPU (quadrupole = 1) against the FP64 oracle's
quadrupole mode: node quadrupoles after a build and after a refit, and walk
errors by the same rule as the monopole walk (p50/p99 within 1.1x the oracle
tree's + 1e-6, interaction counts within 1 %)."""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1811_02761_gb300 as nb  # noqa: E402

EPS, DACC = 1.0 / 64, 2.0 ** -9


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def node_index(ctx, t):
    lev = nb.nbody_export(ctx, nb.nbody.EXPORT_NODE_LEVEL).astype(np.int64)
    start = nb.nbody_export(ctx, nb.nbody.EXPORT_NODE_START).astype(np.int64)
    on = t.nodes()
    key = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(on["level"], on["first"]))}
    return np.array([key[(int(a), int(b))] for a, b in zip(lev, start)]), on


def check_quads(ctx, t):
    idx, on = node_index(ctx, t)
    Qg = nb.nbody_export(ctx, nb.nbody.EXPORT_NODE_Q)[:, :6].astype(np.float64)
    Qo = t.quadrupoles()[idx]
    scale = on["M"][idx] * on["b"][idx] ** 2 + 1e-30
    err = np.abs(Qg - Qo).max(axis=1) / scale
    assert np.percentile(err, 99) < 2e-5 and err.max() < 2e-4, (np.percentile(err, 99), err.max())
    assert np.all(np.abs(Qg[:, 0] + Qg[:, 1] + Qg[:, 2]) <= 1e-4 * scale)


@pytest.mark.parametrize("gen,n,cap", [(ics.galaxy, 20000, 16), (ics.plummer, 8192, 8)])
def test_quadrupole_moments_and_walk_vs_oracle(gen, n, cap):
    p = gen(n, 41)
    x, y, z, m = (p[k].astype(np.float64) for k in ("x", "y", "z", "m"))
    ax, ay, az, phi = oracle.direct(x, y, z, m, 1.0, EPS)
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2).astype(np.float32)
    cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC, leaf_cap=cap, quadrupole=1,
                                  want_potential=1)
    ctx = nb.nbody_create(cfg)
    t = oracle.Tree(x, y, z, m, 21, cap)
    try:
        nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z", "m")])
        check_quads(ctx, t)
        out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(4)]
        st = nb.nbody_walk(ctx, dev(amag), *out)
        g = [o.cpu().numpy().astype(np.float64) for o in out]
    finally:
        nb.nbody_destroy(ctx)
    mode = oracle.MAC_GROUP_ACC | oracle.QUADRUPOLE
    ox, oy, oz, ophi, nint = t.walk(mode, 1.0, EPS, DACC, 0.5, cfg.group_size, amag.astype(np.float64))
    eg = oracle.rel_err(*g[:3], ax, ay, az)
    eo = oracle.rel_err(ox, oy, oz, ax, ay, az)
    for q in (50, 99):
        pg, po = oracle.percentile_nearest_rank(eg, q), oracle.percentile_nearest_rank(eo, q)
        assert pg <= 1.1 * po + 1e-6, (q, pg, po)
    assert abs(st.interactions - nint.sum()) <= 0.01 * nint.sum()
    assert 0 < st.quad_interactions < st.interactions
    # the potential with quadrupole nodes follows the oracle's
    assert np.percentile(np.abs(g[3] - ophi) / np.abs(ophi), 99) < 1e-4
    # with the same MAC the quadrupole walk is more accurate than the monopole walk
    mono = nb.nbody_config_default(eps=EPS, delta_acc=DACC, leaf_cap=cap)
    ctx = nb.nbody_create(mono)
    try:
        nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z", "m")])
        out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
        nb.nbody_walk(ctx, dev(amag), *out)
        gm = [o.cpu().numpy().astype(np.float64) for o in out]
    finally:
        nb.nbody_destroy(ctx)
    em = oracle.rel_err(*gm, ax, ay, az)
    for q in (50, 99):
        assert oracle.percentile_nearest_rank(eg, q) < 0.7 * oracle.percentile_nearest_rank(em, q)


def test_quadrupoles_after_refit_vs_oracle():
    n = 12000
    p = ics.galaxy(n, 42)
    m = p["m"]
    g = np.random.default_rng(5)
    X1 = [(p[k] + g.normal(scale=0.02, size=n)).astype(np.float32) for k in ("x", "y", "z")]
    ctx = nb.nbody_create(nb.nbody_config_default(eps=EPS, quadrupole=1))
    t = oracle.Tree(p["x"], p["y"], p["z"], m, 21, 16)
    t.refit(*[a.astype(np.float64) for a in X1])
    try:
        nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z", "m")])
        nb.nbody_refit(ctx, *[dev(a) for a in X1], dev(m))
        check_quads(ctx, t)
    finally:
        nb.nbody_destroy(ctx)


def test_quadrupole_step_runs_and_export_needs_the_option():
    n = 1 << 13
    p = ics.plummer(n, 43)
    X = [dev(p[k].astype(np.float64)) for k in ("x", "y", "z")]
    V = [dev(p[k]) for k in ("vx", "vy", "vz")]
    M = dev(p["m"])
    A = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    ctx = nb.nbody_create(nb.nbody_config_default(eps=1 / 128, quadrupole=1, rebuild_interval=2))
    try:
        nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z")], M)
        nb.nbody_walk(ctx, None, *A)
        st = nb.nbody_step(ctx, *X, *V, M, *A, 1.0 / 256, 4)
        assert st.rebuilds == 2 and st.quad_interactions > 0
        assert all(torch.isfinite(a).all() for a in A)
    finally:
        nb.nbody_destroy(ctx)
    ctx = nb.nbody_create(nb.nbody_config_default())
    try:
        nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z")], M)
        with pytest.raises(nb.NbodyError) as e:
            nb.nbody_export(ctx, nb.nbody.EXPORT_NODE_Q)
        assert e.value.status == nb.NBODY_EINVAL
    finally:
        nb.nbody_destroy(ctx)
