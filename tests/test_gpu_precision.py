"""Precision of the FP32 walk across the accuracy parameter of Eq. 2, plain and
compensated, against FP64 direct summation and the FP64 oracle tree; and the
FP64 energy history of a multi-step leapfrog run against the oracle's own
leapfrog with the oracle tree force."""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1811_02761_gb300 as nb  # noqa: E402

EPS = 1.0 / 64


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def sweep():
    n = 1 << 15
    p = ics.galaxy(n, 12)
    x, y, z, m = (p[k].astype(np.float64) for k in ("x", "y", "z", "m"))
    bx, by, bz, _ = oracle.direct(x, y, z, m, 1.0, EPS, want_phi=False)
    ctx = nb.nbody_create(nb.nbody_config_default(eps=EPS))
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    res = {}
    try:
        nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z", "m")])
        nb.nbody_walk(ctx, None, *out)
        amag = torch.sqrt(out[0] ** 2 + out[1] ** 2 + out[2] ** 2).contiguous()
        for k in (3, 9, 15):
            for comp in (0, 1):
                cfg = nb.nbody_get_config(ctx)
                cfg.delta_acc, cfg.compensated, cfg.stack_depth = 2.0 ** -k, comp, 1024
                nb.nbody_set_config(ctx, cfg)
                st = nb.nbody_walk(ctx, amag, *out)
                g = [o.cpu().numpy().astype(np.float64) for o in out]
                res[k, comp] = (oracle.rel_err(*g, bx, by, bz), st.interactions)
    finally:
        nb.nbody_destroy(ctx)
    t = oracle.Tree(x, y, z, m, 21, 16)
    am = amag.cpu().numpy().astype(np.float64)
    for k in (3, 9, 15):
        ox, oy, oz, _, ni = t.walk(oracle.MAC_GROUP_ACC, 1.0, EPS, 2.0 ** -k, 0.5, 64, am,
                                   want_phi=False)
        res[k, "oracle"] = (oracle.rel_err(ox, oy, oz, bx, by, bz), int(ni.sum()))
    return res


@pytest.mark.parametrize("k", [3, 9, 15])
@pytest.mark.parametrize("comp", [0, 1])
def test_error_percentiles_track_the_oracle_tree(sweep, k, comp):
    e, ni = sweep[k, comp]
    eo, nio = sweep[k, "oracle"]
    for q in (50, 99):
        pg, po = oracle.percentile_nearest_rank(e, q), oracle.percentile_nearest_rank(eo, q)
        assert pg <= 1.1 * po + 1e-6, (k, comp, q, pg, po)
    assert abs(ni - nio) <= 0.01 * nio


def test_error_falls_with_delta_acc(sweep):
    for comp in (0, 1):
        p50 = [np.median(sweep[k, comp][0]) for k in (3, 9, 15)]
        assert p50[0] > 4 * p50[1] > 16 * p50[2], p50


def test_compensation_is_never_worse_at_the_tight_end(sweep):
    plain, comp = sweep[15, 0][0], sweep[15, 1][0]
    assert np.median(comp) <= 1.05 * np.median(plain) + 1e-8
    assert np.max(comp) <= 1.05 * np.max(plain) + 1e-8


def test_energy_history_matches_oracle_leapfrog():
    """32 KDK steps of the N = 2^13 Plummer sphere (eps = 1/128, dt = 1/256):
    the FP64 energy every 8 steps from the GPU (tree potential, FP64
    reductions) and from the oracle's leapfrog with the oracle tree force
    agree, and stay close to the initial energy."""
    p = ics.plummer(1 << 13, 4)
    n, eps, dt, dacc = p["x"].size, 1.0 / 128, 1.0 / 256, 2.0 ** -9
    x = [p[k].astype(np.float64) for k in ("x", "y", "z")]
    v = [p[k].astype(np.float64) for k in ("vx", "vy", "vz")]
    m = p["m"].astype(np.float64)

    def oracle_force(xs, a_old):
        t = oracle.Tree(*xs, m, 21, 16)
        if a_old is None:
            gx, gy, gz, _, _ = t.walk(oracle.MAC_GROUP_GEO, 1.0, eps, 0.0, 0.5, 64, None,
                                      want_phi=False)
            a_old = np.sqrt(gx ** 2 + gy ** 2 + gz ** 2)
        ax, ay, az, ph, _ = t.walk(oracle.MAC_GROUP_ACC, 1.0, eps, dacc, 0.5, 64, a_old)
        return [ax, ay, az], ph

    # oracle run
    a, ph = oracle_force(x, None)
    e_or = [oracle.diagnostics(*x, *v, m, ph)]
    for s in range(1, 33):
        oracle.kick(v, a, dt / 2)
        oracle.drift(x, v, dt)
        a, ph = oracle_force(x, np.sqrt(sum(q ** 2 for q in a)))
        oracle.kick(v, a, dt / 2)
        if s % 8 == 0:
            e_or.append(oracle.diagnostics(*x, *v, m, ph))

    # GPU run
    cfg = nb.nbody_config_default(eps=eps, delta_acc=dacc)
    ctx = nb.nbody_create(cfg)
    try:
        X = [dev(p[k].astype(np.float64)) for k in ("x", "y", "z")]
        V = [dev(p[k]) for k in ("vx", "vy", "vz")]
        M = dev(p["m"])
        A = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
        At = [torch.empty_like(q) for q in A]
        phi = torch.empty(n, dtype=torch.float32, device="cuda")

        def energy(a_old):
            c2 = nb.nbody_get_config(ctx)
            c2.want_potential = 1
            nb.nbody_set_config(ctx, c2)
            nb.nbody_build(ctx, *[q.float() for q in X], M)
            nb.nbody_walk(ctx, a_old, *At, phi)
            c2.want_potential = 0
            nb.nbody_set_config(ctx, c2)
            return nb.nbody_diagnostics(ctx, *X, *V, M, phi)

        nb.nbody_build(ctx, *[q.float() for q in X], M)
        nb.nbody_walk(ctx, None, *A)
        boot = torch.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2).contiguous()
        nb.nbody_walk(ctx, boot, *A)
        e_gpu = [energy(boot)]
        for s in range(1, 33):
            # the step's walk takes |a| of the previous step; so does the
            # oracle's potential
            prev = torch.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2).contiguous()
            nb.nbody_step(ctx, *X, *V, M, *A, dt, 1)
            if s % 8 == 0:
                e_gpu.append(energy(prev))
    finally:
        nb.nbody_destroy(ctx)
    e0 = e_or[0][0] + e_or[0][1]
    assert len(e_gpu) == len(e_or) == 5
    for go, gg in zip(e_or, e_gpu):
        eo, eg = go[0] + go[1], gg[0] + gg[1]
        # the tree force error moves E by ~1e-5 over these steps; the GPU and
        # the oracle trees differ by ~1e-6 per particle, far less in the sum
        assert abs(eg - eo) <= 3e-6 * abs(e0), (eg, eo, e0)
        assert abs(eo - e0) <= 1e-4 * abs(e0)
        # P wanders by about the force error (the tree force is not exactly
        # antisymmetric); both runs wander alike
        assert np.linalg.norm(gg[2:5] - go[2:5]) <= 2e-5


def test_automatic_compensation_follows_the_mac():
    """compensated = 2 (the default) sums plain at a loose MAC and with
    compensation where the MAC is tight (delta_acc <= 2^-18): its forces equal
    the explicit setting's bit for bit on each side of the threshold, and the
    two settings differ there."""
    n = 1 << 13
    p = ics.plummer(n, 5)
    ctx = nb.nbody_create(nb.nbody_config_default(eps=EPS))
    assert nb.nbody_get_config(ctx).compensated == 2
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    try:
        nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z", "m")])
        nb.nbody_walk(ctx, None, *out)
        amag = torch.sqrt(out[0] ** 2 + out[1] ** 2 + out[2] ** 2).contiguous()
        forces = {}
        for k in (9, 18):
            for comp in (0, 1, 2):
                cfg = nb.nbody_get_config(ctx)
                cfg.delta_acc, cfg.compensated, cfg.stack_depth = 2.0 ** -k, comp, 1024
                nb.nbody_set_config(ctx, cfg)
                nb.nbody_walk(ctx, amag, *out)
                forces[k, comp] = np.stack([o.cpu().numpy() for o in out])
        cfg = nb.nbody_get_config(ctx)
        cfg.compensated = 3
        with pytest.raises(nb.NbodyError) as e:
            nb.nbody_set_config(ctx, cfg)
        assert e.value.status == nb.NBODY_EINVAL
    finally:
        nb.nbody_destroy(ctx)
    assert np.array_equal(forces[9, 2], forces[9, 0])
    assert np.array_equal(forces[18, 2], forces[18, 1])
    assert not np.array_equal(forces[18, 0], forces[18, 1])
