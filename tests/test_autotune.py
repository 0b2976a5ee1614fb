"""Autotuner: the JSON cache (CPU) and the native grid search (GPU)."""
import json

import numpy as np
import pytest

from paper_1811_02761_gb300 import autotune


def test_cache_key_buckets_and_roundtrip(tmp_path):
    k1 = autotune.cache_key("NVIDIA GB300", 1 << 23, 1, 2.0 ** -9)
    k2 = autotune.cache_key("NVIDIA GB300", (1 << 23) + 1000, 1, 2.0 ** -9)
    k3 = autotune.cache_key("NVIDIA GB300", 1 << 23, 512, 2.0 ** -9)
    assert k1 == k2 and k1 != k3
    path = str(tmp_path / "tune.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache(path, {k1: {"ipl": 2, "group_size": 64}})
    assert json.load(open(path))[k1]["ipl"] == 2

    class Cfg:
        leaf_cap, group_size, ipl, list_depth, warps_per_block = 16, 32, 1, 128, 2
    c = autotune.apply(Cfg(), {"ipl": 4, "group_size": 128, "ms": 3.0})
    assert c.ipl == 4 and c.group_size == 128 and c.leaf_cap == 16


@pytest.mark.gpu
def test_autotune_picks_a_candidate_and_keeps_parity(tmp_path):
    torch = pytest.importorskip("torch")
    import ics
    import oracle
    import paper_1811_02761_gb300 as nb
    n = 1 << 15
    p = ics.galaxy(n, 7)
    x, y, z, m = (p[k].astype(np.float64) for k in ("x", "y", "z", "m"))
    ax, ay, az, _ = oracle.direct(x, y, z, m, 1.0, 1 / 64, want_phi=False)
    amag = np.sqrt(ax ** 2 + ay ** 2 + az ** 2).astype(np.float32)

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    X = [D(p[k]) for k in ("x", "y", "z", "m")]
    ctx = nb.nbody_create(nb.nbody_config_default(eps=1 / 64))
    try:
        space = nb.nbody_tune_space_default(group_size=[32, 64], ipl=[1, 2],
                                            warps_per_block=[4], list_depth=[128, 256])
        cache = str(tmp_path / "tune.json")
        best, entry, hit = autotune.tuned_config(ctx, "test", [0, n], None, *X, D(amag), space, cache)
        assert not hit and entry["tried"] >= 3
        # valid candidates: group_size <= 32 ipl, ipl slots some tile can use
        assert (best.group_size, best.ipl) in ((32, 1), (32, 2), (64, 2))
        _, entry2, hit2 = autotune.tuned_config(ctx, "test", [0, n], None, *X, D(amag), space, cache)
        assert hit2 and entry2["group_size"] == best.group_size
        # parity with the oracle tree under the tuned configuration
        nb.nbody_build(ctx, *X)
        out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
        nb.nbody_walk(ctx, D(amag), *out)
        g = [o.cpu().numpy().astype(np.float64) for o in out]
        t = oracle.Tree(x, y, z, m, 21, best.leaf_cap)
        ox, oy, oz, _, _ = t.walk(oracle.MAC_GROUP_ACC, 1.0, 1 / 64, 2.0 ** -9, 0.5, best.group_size,
                                  amag.astype(np.float64), want_phi=False)
        assert np.median(oracle.rel_err(*g, ox, oy, oz)) < 5e-6
    finally:
        nb.nbody_destroy(ctx)
