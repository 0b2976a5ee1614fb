"""The first sort of a step call, started from the previous call's order.

A step call receives its particles in the caller's order, so its first build
sorts them from scratch.  When the context's last step call had the same
particle count, that call's final Morton order (as caller indices) is a
nearly sorted starting point: the keys are gathered into it and sorted by
(key, caller index) with the near-order sort, which is exactly the stable
sort of the caller's order that the radix sort gives.  So a call must end in
the same state, bit for bit, whether or not the context saw a call before --
also when the previous call held different particles (the hint is then just
some permutation) and when particles share Morton keys (ties go by caller
index either way).
"""
import numpy as np
import pytest

import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1811_02761_gb300 as nb  # noqa: E402

DT = 1.0 / 256


def _state(p):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s = [dev(p[k].astype(np.float64)) for k in ("x", "y", "z")]
    s += [dev(p[k].astype(np.float32)) for k in ("vx", "vy", "vz", "m")]
    s += [torch.zeros(len(p["x"]), dtype=torch.float32, device="cuda") for _ in range(3)]
    return s


def _clone(s):
    return [a.clone() for a in s]


def _run(ctx, s, nsteps):
    nb.nbody_step(ctx, *s, DT, nsteps)
    torch.cuda.synchronize()
    return s


def _equal(a, b):
    return all(torch.equal(u, v) for u, v in zip(a, b))


def _fresh(s, nsteps, **cfg):
    ctx = nb.nbody_create(nb.nbody_config_default(eps=1.0 / 64, **cfg))
    try:
        return _run(ctx, _clone(s), nsteps)
    finally:
        nb.nbody_destroy(ctx)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_second_call_equals_a_fresh_context(use_graph):
    s0 = _state(ics.galaxy(1 << 17, 7))
    ctx = nb.nbody_create(nb.nbody_config_default(eps=1.0 / 64, use_graph=use_graph))
    try:
        s1 = _run(ctx, _clone(s0), 2)          # no hint yet: radix sort
        s2 = _run(ctx, _clone(s1), 4)          # hint: the first call's final order
        other = _state(ics.plummer(1 << 17, 9))
        _run(ctx, other, 1)                    # a different set of particles...
        s3 = _run(ctx, _clone(s1), 4)          # ...leaves an unrelated hint
    finally:
        nb.nbody_destroy(ctx)
    ref = _fresh(s1, 4, use_graph=use_graph)
    assert _equal(s2, ref)
    assert _equal(s3, ref)


def test_ties_in_morton_keys_go_by_caller_index():
    p = ics.plummer(1 << 14, 11)
    # every particle twice, at the same position: pairs of equal keys
    q = {k: np.concatenate([v, v]) for k, v in p.items() if k in ("x", "y", "z", "vx", "vy", "vz", "m")}
    g = np.random.default_rng(3)
    perm = g.permutation(len(q["x"]))
    q = {k: v[perm] for k, v in q.items()}
    s0 = _state(q)
    ctx = nb.nbody_create(nb.nbody_config_default(eps=1.0 / 64))
    try:
        s1 = _run(ctx, _clone(s0), 1)
        s2 = _run(ctx, _clone(s1), 2)
    finally:
        nb.nbody_destroy(ctx)
    assert _equal(s2, _fresh(s1, 2))


@pytest.mark.parametrize("block_levels", [0, 3])
def test_batched_second_call_equals_a_fresh_context(block_levels):
    """The same for a forest of systems (the keys carry the system id), with
    shared steps and with block time steps."""
    b = ics.batched(24, 5, 8.0, 12.0)
    off, eps = b["offsets"], b["eps"]
    s0 = _state(b)

    def step(ctx, s, k):
        nb.nbody_step_batched(ctx, off, eps, *s, DT, k)
        torch.cuda.synchronize()
        return s

    cfg = dict(eps=1.0 / 64, block_levels=block_levels)
    ctx = nb.nbody_create(nb.nbody_config_default(**cfg))
    try:
        s1 = step(ctx, _clone(s0), 1)
        s2 = step(ctx, _clone(s1), 3)
    finally:
        nb.nbody_destroy(ctx)
    ctx = nb.nbody_create(nb.nbody_config_default(**cfg))
    try:
        ref = step(ctx, _clone(s1), 3)
    finally:
        nb.nbody_destroy(ctx)
    assert _equal(s2, ref)
