"""The warp-specialised walk (walk_pipeline = 1: a traversal warp hands
interaction lists to an evaluation warp) builds the same lists, flushes them
at the same points and sums in the same order as the one-warp walk, so its
accelerations must equal the one-warp walk's bit for bit."""
import numpy as np
import pytest

import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1811_02761_gb300 as nb  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def walk(p, pipeline, a_old=None, offsets=None, eps_sys=None, **cfg):
    n = p["x"].size
    ctx = nb.nbody_create(nb.nbody_config_default(walk_pipeline=pipeline, **cfg))
    try:
        X = [dev(p[k]) for k in ("x", "y", "z", "m")]
        if offsets is None:
            nb.nbody_build(ctx, *X)
        else:
            nb.nbody_build_batched(ctx, offsets, eps_sys, *X)
        out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
        st = nb.nbody_walk(ctx, None if a_old is None else dev(a_old), *out)
        return [o.cpu().numpy() for o in out], st
    finally:
        nb.nbody_destroy(ctx)


@pytest.fixture(scope="module")
def galaxy():
    p = ics.galaxy(40000, 71)
    ref, _ = walk(p, 0, eps=1 / 64)
    amag = np.sqrt(sum(a.astype(np.float64) ** 2 for a in ref)).astype(np.float32)
    return p, amag


@pytest.mark.parametrize("ipl,G,comp,wpb", [(1, 32, 0, 4), (2, 64, 0, 2), (3, 64, 0, 4), (3, 96, 1, 4),
                                            (4, 128, 0, 8)])
def test_pipelined_walk_equals_one_warp_walk(galaxy, ipl, G, comp, wpb):
    p, amag = galaxy
    cfg = dict(eps=1 / 64, delta_acc=2.0 ** -9, ipl=ipl, group_size=G, compensated=comp,
               warps_per_block=wpb)
    a0, s0 = walk(p, 0, amag, **cfg)
    a1, s1 = walk(p, 1, amag, **cfg)
    for u, v in zip(a0, a1):
        assert np.array_equal(u, v)
    assert s0.interactions == s1.interactions and s0.list_entries == s1.list_entries
    assert s0.max_stack == s1.max_stack


def test_pipelined_bootstrap_walk_equals_one_warp_walk(galaxy):
    p, _ = galaxy
    a0, _ = walk(p, 0, None, eps=1 / 64, list_depth=64)
    a1, _ = walk(p, 1, None, eps=1 / 64, list_depth=64)
    for u, v in zip(a0, a1):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("n", [1, 2, 17, 100, 5003])
def test_pipelined_walk_small_ragged_and_unsoftened(n):
    p = ics.plummer(n, 72)
    for eps in (1 / 128, 0.0):
        a0, _ = walk(p, 0, eps=eps)
        a1, _ = walk(p, 1, eps=eps)
        for u, v in zip(a0, a1):
            assert np.array_equal(u, v)


def test_pipelined_batched_forest_and_steps():
    sizes = [3000, 1, 700, 9000]
    b = ics.batched(len(sizes), 11, sizes=sizes)
    a0, _ = walk(b, 0, offsets=b["offsets"], eps_sys=b["eps"])
    a1, _ = walk(b, 1, offsets=b["offsets"], eps_sys=b["eps"])
    for u, v in zip(a0, a1):
        assert np.array_equal(u, v)
    n = int(b["offsets"][-1])
    res = []
    for pipeline in (0, 1):
        ctx = nb.nbody_create(nb.nbody_config_default(delta_acc=2.0 ** -9, walk_pipeline=pipeline))
        try:
            X = [dev(b[k].astype(np.float64)) for k in ("x", "y", "z")]
            V = [dev(b[k]) for k in ("vx", "vy", "vz")]
            A = [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(3)]
            nb.nbody_step_batched(ctx, b["offsets"], b["eps"], *X, *V, dev(b["m"]), *A, 1.0 / 256, 3)
            res.append([t.cpu().numpy() for t in X + V + A])
        finally:
            nb.nbody_destroy(ctx)
    for u, v in zip(*res):
        assert np.array_equal(u, v)


def test_pipeline_needs_warp_pairs():
    with pytest.raises(nb.NbodyError) as e:
        nb.nbody_create(nb.nbody_config_default(walk_pipeline=1, warps_per_block=3))
    assert e.value.status == nb.NBODY_EINVAL
