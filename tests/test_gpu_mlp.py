"""Learned cost model (MLP) on the GPU: gradients against the FP64 oracle,
online training on the walk's own cost log, and schedule invariance of the
forces."""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1811_02761_gb300 as nb  # noqa: E402


def bf16_round(a):
    """Round FP32 values to BF16 (nearest even), kept in FP32 storage."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_mlp_eval_matches_fp64_oracle():
    """GPU forward/backward (BF16 weights, FP32 accumulation) against the FP64
    oracle evaluated on the same BF16-rounded weights."""
    g = ics.rng(5, 6)
    n = 3000
    feat = g.normal(size=(n, 8)).astype(np.float32)
    target = g.normal(size=n).astype(np.float32)
    w = ics.mlp_init(5)
    w[8 * 32:8 * 32 + 32] = g.normal(scale=0.1, size=32)
    w[-1] = 0.2
    norm = np.concatenate([g.normal(scale=0.1, size=8), g.uniform(0.5, 2.0, 8)]).astype(np.float32)
    pred, grad, loss = nb.nbody_mlp_eval(feat, target, w, norm)
    wr = bf16_round(w).astype(np.float64)
    opred, ograd, oloss = oracle.mlp_eval(feat.astype(np.float64), target.astype(np.float64), wr,
                                          norm.astype(np.float64))
    assert np.max(np.abs(pred - opred)) <= 1e-4 * (1 + np.max(np.abs(opred)))
    assert abs(loss - oloss) <= 1e-4 * oloss
    sl = {"W1": slice(0, 256), "b1": slice(256, 288), "W2": slice(288, 1312),
          "b2": slice(1312, 1344), "W3": slice(1344, 1376), "b3": slice(1376, 1377)}
    for name, s in sl.items():
        a, b = grad[s].astype(np.float64), ograd[s]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        assert rel <= 1e-2 and cos >= 0.999, (name, rel, cos)


@pytest.fixture(scope="module")
def trained():
    # enough groups (~12k) to outnumber the resident walk warps, so the
    # cost-ordered queue is really used
    n = 1 << 18
    p = ics.galaxy(n, 8)
    X = [dev(p[k]) for k in ("x", "y", "z", "m")]
    ctx = nb.nbody_create(nb.nbody_config_default(eps=1 / 64, group_size=32, ipl=1))
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    nb.nbody_build(ctx, *X)
    nb.nbody_walk(ctx, None, *out)
    amag = torch.sqrt(out[0] ** 2 + out[1] ** 2 + out[2] ** 2).cpu().numpy()
    nb.nbody_walk(ctx, dev(amag), *out)
    ng = nb.nbody_export(ctx, nb.nbody.EXPORT_GROUP_FIRST).size
    cost = np.empty(ng, np.int32)
    nb.nbody_get_group_costs(ctx, cost)
    nb.nbody_mlp_set_params(ctx, ics.mlp_init(1))
    losses = [nb.nbody_mlp_train(ctx, epochs=1, lr=3e-3, batch=512) for _ in range(40)]
    yield ctx, X, amag, out, cost, losses
    nb.nbody_destroy(ctx)


def test_mlp_training_learns_the_walk_cost(trained):
    ctx, X, amag, out, cost, losses = trained
    assert losses[-1] < 0.5 * losses[0], losses[::8]
    pred, feat = nb.nbody_mlp_predict(ctx, want_features=True)
    assert pred.size == cost.size and np.all(np.isfinite(feat))
    r = np.corrcoef(pred, np.log2(np.maximum(cost, 1)))[0, 1]
    assert r >= 0.8, r


def test_schedules_give_bitwise_identical_forces(trained):
    ctx, X, amag, out, cost, losses = trained
    res = {}
    for sched in (nb.SCHED_MORTON, nb.SCHED_MLP, nb.SCHED_LASTCOST):
        cfg = nb.nbody_get_config(ctx)
        cfg.schedule = sched
        nb.nbody_set_config(ctx, cfg)
        nb.nbody_walk(ctx, dev(amag), *out)
        res[sched] = [o.cpu().numpy().copy() for o in out]
    for s in (nb.SCHED_MLP, nb.SCHED_LASTCOST):
        for a, b in zip(res[nb.SCHED_MORTON], res[s]):
            assert np.array_equal(a, b)
    cfg = nb.nbody_get_config(ctx)
    cfg.schedule = nb.SCHED_MORTON
    nb.nbody_set_config(ctx, cfg)


def test_mlp_schedule_needs_parameters():
    ctx = nb.nbody_create(nb.nbody_config_default(schedule=nb.SCHED_MLP))
    try:
        p = ics.plummer(2000, 3)
        nb.nbody_build(ctx, *[dev(p[k]) for k in ("x", "y", "z", "m")])
        out = [torch.empty(2000, dtype=torch.float32, device="cuda") for _ in range(3)]
        with pytest.raises(nb.NbodyError) as e:
            nb.nbody_walk(ctx, None, *out)
        assert e.value.status == nb.NBODY_EINVAL
    finally:
        nb.nbody_destroy(ctx)
