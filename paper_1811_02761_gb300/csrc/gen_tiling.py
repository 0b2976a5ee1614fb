"""Writes walk_tiling.cuh: how the walk lays a group of cnt particles over the
32 lanes of a warp, for every cnt and every slot count (ipl = 1..4).

A lane holds up to ipl i-particles in slots.  The slots form runs; run k has
r_k slots, P_k rows and s_k = floor(32 / P_k) splits: lane L is row L % P_k
of split L / P_k (idle in run k when L / P_k >= s_k), its t-th slot of the
run holds particle base_k + row + P_k t, and it takes every s_k-th entry pair
of the interaction list.  One flush loop serves a run: per entry pair it
issues two list loads and the loop control (about 5 instructions) plus 14
per slot (12 packed FP32 operations and 2 rsqrt), for list / s_k pairs.  The
table holds, for each cnt, the runs (at most three, at most ipl slots in
all, covering cnt) with the fewest issued instructions per list entry,
sum_k (5 + 14 r_k) / s_k; ties go to fewer slots, then to less FP32 work,
sum_k r_k / s_k.

Encoding of an entry (uint64): bits 0-1 the number of runs; run k in bits
2 + 16 k .. 17 + 16 k as r (4 bits), P (6 bits), s (6 bits).

Run `python gen_tiling.py` in this folder after changing the cost model;
tests/test_tiling_table.py checks that the committed header matches.
"""
import itertools
import os

OVERHEAD, PER_SLOT = 5.0, 14.0
MAX_IPL, MAX_CNT = 4, 128


def splits(P):
    return 32 // P


def cost(runs):
    return (sum((OVERHEAD + PER_SLOT * r) / splits(P) for r, P in runs),
            sum(r for r, _ in runs),
            sum(r / splits(P) for r, P in runs))


def candidates(cnt, ipl):
    """Every run list with at most three runs and ipl slots that covers cnt;
    the last run's rows are the fewest that cover what is left."""
    for nr in (1, 2, 3):
        for rs in itertools.product(range(1, ipl + 1), repeat=nr):
            if sum(rs) > ipl:
                continue
            for Ps in itertools.product(range(1, 33), repeat=nr - 1):
                covered = sum(r * P for r, P in zip(rs, Ps))
                rem = cnt - covered
                if nr > 1 and rem <= 0:
                    continue  # the last run would be empty
                last = -(-max(rem, 1) // rs[-1])
                if last > 32:
                    continue
                yield list(zip(rs, list(Ps) + [last]))


def best(cnt, ipl):
    if cnt < 1 or cnt > 32 * ipl:
        return None
    return min(candidates(cnt, ipl), key=cost)


def encode(runs):
    if runs is None:
        return 0
    v = len(runs)
    for k, (r, P) in enumerate(runs):
        v |= (r | (P << 4) | (splits(P) << 10)) << (2 + 16 * k)
    return v


def table():
    return [[encode(best(cnt, ipl)) for cnt in range(MAX_CNT + 1)] for ipl in range(1, MAX_IPL + 1)]


def header():
    rows = []
    for ipl, entries in enumerate(table(), start=1):
        vals = ", ".join(f"0x{v:013x}ull" for v in entries)
        rows.append(f"    // ipl = {ipl}\n    {{{vals}}}")
    return ("// walk_tiling.cuh -- written by gen_tiling.py (the lane layout of a group\n"
            "// of cnt particles for each slot count; see that script for the cost\n"
            "// model and the encoding).  Do not edit by hand.\n"
            "#pragma once\n#include <cstdint>\n\nnamespace nb {\n\n"
            f"constexpr int kTilingMaxCnt = {MAX_CNT};\n"
            f"__device__ const uint64_t kTiling[{MAX_IPL}][{MAX_CNT + 1}] = {{\n"
            + ",\n".join(rows) + "};\n\n}  // namespace nb\n")


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "walk_tiling.cuh")
    with open(out, "w") as f:
        f.write(header())
    print("wrote", out)
