"""The build's two sorts against the oracle's stable sort, bit for bit.

The tree build orders particles by Morton key (Sect. 4.1) with a stable
sort.  A build from the caller's order uses the one-sweep LSD radix sort; the
builds inside a step, whose keys are nearly in order already, use the bucket
sort (splitters, scatter, a shared-memory merge sort per bucket).  Both must
give exactly the oracle's stable order, for every input: random keys over
the whole 64-bit range (0 and 2^64 - 1 included), the sizes around the
bucket sort's tile (1984) and shared-memory capacity (2048), random keys
whose uneven buckets exceed the capacity (merged in global memory), heavy and
total ties (the buckets are cut by key and index, so ties spread over them),
reversed and nearly sorted keys, and the galaxy's own keys after a drift in
the order of the build before it.
"""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1811_02761_gb300 as nb  # noqa: E402

METHODS = [nb.SORT_RADIX, nb.SORT_NEAR_ORDER]
U64_MAX = np.iinfo(np.uint64).max


@pytest.fixture(scope="module")
def ctx():
    c = nb.nbody_create(nb.nbody_config_default())
    yield c
    nb.nbody_destroy(c)


def _gpu_sort(ctx, method, k):
    kin = torch.from_numpy(np.ascontiguousarray(k).view(np.int64)).cuda()
    kout = torch.empty_like(kin)
    perm = torch.empty(k.size, dtype=torch.int32, device="cuda")
    nb.nbody_sort_keys(ctx, method, kin, kout, perm)
    assert np.array_equal(kin.cpu().numpy().view(np.uint64), k)  # input left alone
    return kout.cpu().numpy().view(np.uint64), perm.cpu().numpy().astype(np.int64)


def _check(ctx, method, k):
    k = np.ascontiguousarray(k, dtype=np.uint64)
    order = oracle.sort_order(k)
    keys, perm = _gpu_sort(ctx, method, k)
    assert np.array_equal(perm, order)
    assert np.array_equal(keys, k[order])


def _random(g, n):
    return g.integers(0, U64_MAX, n, dtype=np.uint64, endpoint=True)


def _near(g, n, disp=40.0, far=1e-3):
    """Sorted keys displaced by a few dozen places, with a few far movers."""
    base = np.sort(_random(g, n))
    k = base[np.argsort(np.arange(n) + g.normal(0.0, disp, n), kind="stable")].copy()
    i = g.choice(n, max(1, int(n * far)), replace=False)
    k[i] = _random(g, i.size)
    return k


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n", [1, 2, 3, 1983, 1984, 1985, 2047, 2048, 2049, 3969, 4097, 65537])
def test_random_keys_ragged_sizes(ctx, method, n):
    g = np.random.default_rng(n)
    k = _random(g, n)
    if n >= 3:
        k[0], k[n // 2] = U64_MAX, 0
    _check(ctx, method, k)


@pytest.mark.parametrize("method", METHODS)
def test_nearly_sorted_keys(ctx, method):
    _check(ctx, method, _near(np.random.default_rng(1), 1 << 20))


@pytest.mark.parametrize("method", METHODS)
def test_reversed_keys(ctx, method):
    _check(ctx, method, np.sort(_random(np.random.default_rng(2), 1 << 20))[::-1])


@pytest.mark.parametrize("method", METHODS)
def test_heavy_ties(ctx, method):
    """37 distinct keys over 3 10^5 places: buckets of thousands of equal
    keys, the order among them decided by the input index alone."""
    g = np.random.default_rng(3)
    vals = _random(g, 37)
    _check(ctx, method, vals[g.integers(0, 37, 300000)])


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n", [50000, 1 << 21])
def test_all_keys_equal(ctx, method, n):
    """Buckets are cut by (key, index), so 2^21 equal keys still make
    buckets of one tile each instead of one bucket of everything."""
    _check(ctx, method, np.full(n, 0x123456789ABCDEF, dtype=np.uint64))


@pytest.mark.parametrize("method", METHODS)
def test_ties_at_the_largest_key(ctx, method):
    """Keys equal to 2^64 - 1, the value the bucket sort pads a chunk with."""
    g = np.random.default_rng(4)
    k = _near(g, 5000)
    k[g.choice(5000, 700, replace=False)] = U64_MAX
    _check(ctx, method, k)


@pytest.mark.parametrize("method", METHODS)
def test_galaxy_keys_after_a_drift(ctx, method):
    """The case the bucket sort is for: the galaxy's Morton keys at drifted
    positions, in the sorted order of the keys before the drift."""
    p = ics.galaxy(1 << 21, 2)
    x = [p[c].astype(np.float64) for c in ("x64", "y64", "z64")]
    v = [p[c].astype(np.float64) for c in ("vx", "vy", "vz")]
    k0, _ = oracle.keys(*(a.astype(np.float32) for a in x), 21)
    k1, _ = oracle.keys(*((a + 4 * b / 256).astype(np.float32) for a, b in zip(x, v)), 21)
    _check(ctx, method, k1[oracle.sort_order(k0)])


def test_sort_keys_rejects_bad_arguments(ctx):
    k = torch.zeros(16, dtype=torch.int64, device="cuda")
    out = torch.empty_like(k)
    perm = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(nb.NbodyError) as e:
        nb.nbody_sort_keys(ctx, 7, k, out, perm)
    assert e.value.status == nb.NBODY_EINVAL
    with pytest.raises(nb.NbodyError) as e:
        nb.nbody_sort_keys(ctx, nb.SORT_RADIX, k.cpu(), out, perm)  # host keys
    assert e.value.status == nb.NBODY_EINVAL
