"""nbody_diagnostics_noalloc: the allocation-free variant of the FP64
diagnostics, for callers that cannot call cudaMalloc (device memory already
reserved by another allocator, or no allocation allowed inside a step loop).

It must return what nbody_diagnostics returns, on two calls in a row (its
scratch array is reused between calls and keeps the previous call's
contents).  This file sorts last so that a run stopping at the first failure
has already run every other test; it also passes on its own in a fresh
process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import ics  # noqa: E402
import paper_1811_02761_gb300 as nb  # noqa: E402


def _state(n, seed):
    p = ics.plummer(n, seed)
    g = np.random.default_rng(seed)
    phi = (-1.0 / np.sqrt(1.0 + p["x"] ** 2 + p["y"] ** 2 + p["z"] ** 2)).astype(np.float32)
    cols = [p["x"].astype(np.float64) + 0.5, p["y"].astype(np.float64) - 0.25,
            p["z"].astype(np.float64), p["vx"], p["vy"], p["vz"], p["m"] * g.uniform(0.5, 1.5, n).astype(np.float32),
            phi]
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cols]


def _reference(cols):
    ctx = nb.nbody_create(nb.nbody_config_default())
    try:
        return nb.nbody_diagnostics(ctx, *cols)
    finally:
        nb.nbody_destroy(ctx)


def _close(got, ref):
    # same tolerance as the diagnostics parity test: 1e-12 of each sum's scale
    scale = np.array([abs(ref[0]), abs(ref[1])] + [np.abs(ref[2:5]).max() + 1e-3] * 3 +
                     [np.abs(ref[5:]).max() + 1e-3] * 3)
    return np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-15)


def test_noalloc_diagnostics_matches_existing_entry_point_twice():
    big = _state(200_000, 21)
    small = _state(1_000, 22)
    ref_big, ref_small = _reference(big), _reference(small)
    # two calls in a row: the second sees the scratch left by the first
    got1 = nb.nbody_diagnostics_noalloc(*big)
    got2 = nb.nbody_diagnostics_noalloc(*small)
    assert _close(got1, ref_big), (got1, ref_big)
    assert _close(got2, ref_small), (got2, ref_small)
    # and a device-resident result buffer
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    nb.nbody_diagnostics_noalloc(*big, out=out)
    assert _close(out.cpu().numpy(), ref_big)


def test_noalloc_diagnostics_rejects_host_inputs():
    cols = _state(100, 23)
    host = [c.cpu().numpy() for c in cols]
    with pytest.raises(nb.NbodyError) as e:
        nb.nbody_diagnostics_noalloc(*host)
    assert e.value.status == nb.NBODY_EINVAL


def test_noalloc_diagnostics_rejects_arrays_of_another_gpu():
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    cols = _state(100, 24)
    other = [c.to("cuda:1") for c in cols]
    with torch.cuda.device(0):
        with pytest.raises(nb.NbodyError) as e:
            nb.nbody_diagnostics_noalloc(*other)
    assert e.value.status == nb.NBODY_EINVAL
