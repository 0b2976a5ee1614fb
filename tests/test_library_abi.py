"""The C-ABI library builds, loads and exports every entry point that
include/nbody.h declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

import paper_1811_02761_gb300 as nb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "nbody.h")).read()
    return sorted(set(re.findall(r"^\s*(?:nbody_status|int32_t|void)\s+\*?\s*(nbody_\w+)\s*\(",
                                 src, re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("nbody_build", "nbody_walk", "nbody_direct", "nbody_step", "nbody_create",
              "nbody_destroy", "nbody_build_batched", "nbody_step_batched", "nbody_diagnostics"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    lib = nb.load()
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert set(nb.nbody.EXPORTS) == set(declared_symbols())


def test_abi_version_and_defaults():
    assert nb.nbody_abi_version() == 2
    c = nb.nbody_config_default()
    assert c.G == 1.0 and c.delta_acc == 2.0 ** -9 and c.leaf_cap == 16
    assert c.group_size <= 32 * c.ipl
    assert c.rebuild_interval == 1


@pytest.mark.parametrize("bad", [dict(ipl=5), dict(ipl=0), dict(leaf_cap=0), dict(group_size=8, leaf_cap=16),
                                 dict(group_size=128, ipl=2), dict(list_depth=100),
                                 dict(eps=-1.0), dict(theta=1.5), dict(delta_acc=-1e-3),
                                 dict(warps_per_block=16, list_depth=1024, stack_depth=4096),
                                 dict(rebuild_interval=-1), dict(rebuild_interval=2000)])
def test_create_rejects_bad_config_before_any_device_work(bad):
    with pytest.raises(nb.NbodyError) as e:
        nb.nbody_create(nb.nbody_config_default(**bad))
    assert e.value.status == nb.NBODY_EINVAL


def test_stateless_argument_checks():
    import numpy as np
    x = np.zeros(4, np.float32)
    with pytest.raises(nb.NbodyError) as e:
        nb.nbody_direct(x, x, x, x, 1.0, -1.0, 0, x.copy(), x.copy(), x.copy())
    assert e.value.status == nb.NBODY_EINVAL
    with pytest.raises(nb.NbodyError):
        nb.nbody_direct(x, x, x, np.zeros(3, np.float32), 1.0, 0.1, 0, x, x, x)


def test_binding_rejects_wrong_dtypes():
    import numpy as np
    lib = nb.load()
    assert isinstance(lib, ctypes.CDLL)
    with pytest.raises(nb.NbodyError):
        nb.nbody.nbody_build(None, np.zeros(4, np.float64), *[np.zeros(4, np.float32)] * 3)


def test_rebuild_policy_minimises_the_mean_step_cost():
    """rebuild_interval = 0 (host-only policy): with a walk that slows down
    linearly after each rebuild (cost B + w after a rebuild, R + w + g k after
    k refits) the policy must pick the interval that minimises the mean cost
    per step, about sqrt(2 (B - R) / g); with no slow-down it never rebuilds."""
    B, R, w, g = 3.0, 0.6, 7.0, 0.05

    def cycle(k):
        return [B + w] + [R + w + g * j for j in range(1, k)]

    def mean(k):
        return sum(cycle(k)) / k

    best = min(range(1, 200), key=mean)
    # the policy's first "rebuild now" after steps 0..m-1 of the cycle
    m = next(m for m in range(2, 200) if nb.nbody_rebuild_due(cycle(m)))
    assert abs((m - 1) - best) <= 1, (m, best)
    assert not any(nb.nbody_rebuild_due([B + w] + [R + w] * k) for k in range(1, 100))
    assert not nb.nbody_rebuild_due([5.0]) and not nb.nbody_rebuild_due([])
