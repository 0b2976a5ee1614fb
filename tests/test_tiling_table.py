"""The walk's lane-tiling table (csrc/walk_tiling.cuh, written by
csrc/gen_tiling.py): the committed header is what the generator writes, and
every entry is a valid layout -- at most ipl slots in at most three runs,
each run's splits floor(32 / rows), and the runs' rows and slots covering the
group's particles 0..cnt-1 exactly once -- that no other layout beats under
the generator's cost model (checked by brute force over single runs and
pairs of runs of one slot)."""
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1811_02761_gb300", "csrc")


@pytest.fixture(scope="module")
def gen():
    spec = importlib.util.spec_from_file_location("gen_tiling", os.path.join(CSRC, "gen_tiling.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.fixture(scope="module")
def entries():
    text = open(os.path.join(CSRC, "walk_tiling.cuh")).read()
    rows = re.findall(r"\{([0-9a-fx, ull]+)\}", text)
    return [[int(v.strip().rstrip("ul"), 16) for v in r.split(",")] for r in rows]


def decode(v):
    """The device's reading of an entry: (r, P, s) per run."""
    nr = v & 3
    return [((v >> (2 + 16 * k)) & 15, (v >> (6 + 16 * k)) & 63, (v >> (12 + 16 * k)) & 63)
            for k in range(nr)]


def test_header_matches_generator(gen):
    assert open(os.path.join(CSRC, "walk_tiling.cuh")).read() == gen.header()


def test_every_layout_covers_the_group_once(entries):
    assert len(entries) == 4
    for ipl, row in enumerate(entries, start=1):
        assert len(row) == 129
        assert row[0] == 0
        for cnt in range(1, 129):
            runs = decode(row[cnt])
            if cnt > 32 * ipl:
                assert runs == []
                continue
            assert 1 <= len(runs) <= 3
            assert sum(r for r, _, _ in runs) <= ipl
            seen, base = [], 0
            for r, P, s in runs:
                assert 1 <= r and 1 <= P <= 32 and s == 32 // P
                seen += [base + row_ + P * t for t in range(r) for row_ in range(P)]
                base += r * P
            inside = sorted(i for i in seen if i < cnt)
            assert inside == list(range(cnt)), (ipl, cnt, runs)


def test_layouts_are_optimal_under_the_model(gen, entries):
    def cost(runs):  # runs: (r, P) pairs
        return sum((gen.OVERHEAD + gen.PER_SLOT * r) / (32 // P) for r, P in runs)
    for ipl, row in enumerate(entries, start=1):
        for cnt in range(1, 32 * ipl + 1):
            got = cost([(r, P) for r, P, _ in decode(row[cnt])])
            for r in range(1, ipl + 1):  # one run of r slots
                P = -(-cnt // r)
                if P <= 32:
                    assert got <= cost([(r, P)]) + 1e-9
            if ipl >= 2:  # two runs of one slot
                for P1 in range(1, 33):
                    P2 = cnt - P1
                    if 1 <= P2 <= 32:
                        assert got <= cost([(1, P1), (1, P2)]) + 1e-9
