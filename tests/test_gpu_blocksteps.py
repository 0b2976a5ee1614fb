"""Block time steps on the GPU (block_levels) against the FP64 oracle's block
kick-drift-kick: with delta_acc = 0 the walk is the direct sum, so the GPU
trajectory follows the oracle's up to FP32 rounding (and the rare particle
whose level decision flips on that rounding); with every particle on one
level the block path repeats the shared-step path bit for bit."""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1811_02761_gb300 as nb  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_run(p, cfg, dt, nsteps, offsets=None, eps_sys=None):
    n = p["x"].size
    X = [dev(p[k].astype(np.float64)) for k in ("x", "y", "z")]
    V = [dev(p[k]) for k in ("vx", "vy", "vz")]
    M = dev(p["m"])
    A = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    ctx = nb.nbody_create(cfg)
    try:
        if offsets is None:
            nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z")], M)
            nb.nbody_walk(ctx, None, *A)
            st = nb.nbody_step(ctx, *X, *V, M, *A, dt, nsteps)
        else:
            nb.nbody_build_batched(ctx, offsets, eps_sys, *[dev(p[k]) for k in ("x", "y", "z")], M)
            nb.nbody_walk(ctx, None, *A)
            st = nb.nbody_step_batched(ctx, offsets, eps_sys, *X, *V, M, *A, dt, nsteps)
    finally:
        nb.nbody_destroy(ctx)
    return [t.cpu().numpy() for t in X], [t.cpu().numpy() for t in V], [t.cpu().numpy() for t in A], st


def test_block_steps_follow_the_oracle():
    n, eps, dt, K, eta = 4096, 1.0 / 64, 1.0 / 8, 3, 0.05
    p = ics.plummer(n, 61)
    cfg = nb.nbody_config_default(eps=eps, delta_acc=0.0, block_levels=K, block_eta=eta)
    # initial accelerations as the GPU starts from them: an exact (delta_acc = 0) walk
    X0, V0, A0, _ = gpu_run(p, cfg, dt, 0)
    gx, gv, ga, st = gpu_run(p, cfg, dt, 2)
    m = p["m"].astype(np.float64)
    x0 = [p[k].astype(np.float64) for k in ("x", "y", "z")]
    v0 = [p[k].astype(np.float64) for k in ("vx", "vy", "vz")]
    a0 = [a.astype(np.float64) for a in A0]

    def force(x, idx):
        return oracle.direct_targets(*x, m, idx, 1.0, eps)[:3]

    ox, ov, oa, lvl, nforce = oracle.block_kdk(x0, v0, m, a0, 1.0, eps, dt, 2, K, eta, force)
    assert np.bincount(lvl, minlength=K + 1)[1:].sum() > 0.1 * n  # several levels in use
    dx = np.sqrt(sum((gx[c] - ox[c]) ** 2 for c in range(3)))
    dv = np.sqrt(sum((gv[c] - ov[c]) ** 2 for c in range(3)))
    vs = np.sqrt(sum(ov[c] ** 2 for c in range(3)))
    assert np.median(dx) < 1e-6 and np.percentile(dx, 99) < 1e-4, (np.median(dx), np.percentile(dx, 99))
    assert np.median(dv / vs) < 1e-5 and np.percentile(dv / vs, 99) < 1e-3
    # fewer walks than a shared step at the finest level would need
    assert st.interactions < 0.8 * n * n * 2 * (1 << K)


def test_block_steps_on_one_level_equal_the_shared_step():
    n = 6000
    p = ics.galaxy(n, 62)
    base = dict(eps=1.0 / 64, delta_acc=2.0 ** -9)
    sx, sv, sa, _ = gpu_run(p, nb.nbody_config_default(**base), 1.0 / 128, 3)
    bx, bv, ba, st = gpu_run(p, nb.nbody_config_default(**base, block_levels=2, block_eta=1e30),
                             1.0 / 128, 3)
    assert st.rebuilds == 3
    for q, r in zip(sx + sv + sa, bx + bv + ba):
        assert np.array_equal(q, r)


def test_block_steps_batched_systems_and_refit():
    sizes = [3000, 500, 1500]
    parts = [ics.plummer(k, 63 + i) for i, k in enumerate(sizes)]
    p = {k: np.concatenate([q[k] for q in parts]) for k in ("x", "y", "z", "vx", "vy", "vz", "m")}
    for i in range(1, 3):  # move the systems apart
        s0 = sum(sizes[:i])
        p["x"][s0:s0 + sizes[i]] += 50.0 * i
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    eps_sys = np.array([1 / 32, 1 / 16, 1 / 24], np.float32)
    cfg = nb.nbody_config_default(delta_acc=2.0 ** -9, block_levels=3, block_eta=0.05,
                                  rebuild_interval=0)
    gx, gv, ga, st = gpu_run(p, cfg, 1.0 / 8, 2, offsets, eps_sys)
    assert all(np.isfinite(a).all() for a in gx + gv + ga)
    assert 1 <= st.rebuilds
    # each system's accelerations at the end agree with its own FP64 direct sum
    for i in range(3):
        s0, s1 = offsets[i], offsets[i + 1]
        xs = [gx[c][s0:s1].astype(np.float32).astype(np.float64) for c in range(3)]
        ax, ay, az, _ = oracle.direct(*xs, p["m"][s0:s1].astype(np.float64), 1.0, float(eps_sys[i]),
                                      want_phi=False)
        e = oracle.rel_err(*[ga[c][s0:s1].astype(np.float64) for c in range(3)], ax, ay, az)
        assert oracle.percentile_nearest_rank(e, 99) < 1e-2
