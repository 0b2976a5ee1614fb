"""Group-by-group comparison of the GPU walk with the FP64 oracle walk.

With the same tree, the same groups, the same a_old and the same reading of
Eq. 2, every group's interaction list has the same length on both sides
unless a MAC decision (d > b_J, or G M b_J^2 <= dacc |a_old| d^4) sits within
FP32 rounding of its threshold: the GPU decides in FP32 with FP32 moments and
group spheres, the oracle in FP64.  These helpers find the groups whose list
lengths differ and check that each one has such a near-threshold node among
the nodes the oracle's traversal of that group visits.
"""
import numpy as np


def group_entries(ninter, order, first):
    """Oracle list length of each group: every member of a group shares one
    list, so it is the interaction count of the group's first member."""
    return np.asarray(ninter)[np.asarray(order)[np.asarray(first, dtype=np.int64)]]


def group_spheres(x, y, z, order, first, count, a_old):
    """FP64 group sphere (bounding-box centre, largest member distance) and the
    smallest |a_old| of the members, as the group-mode MAC reads them."""
    ng = len(first)
    c = np.empty((ng, 3))
    r = np.empty(ng)
    amin = np.empty(ng)
    P = np.stack([x, y, z], 1)
    for g in range(ng):
        idx = order[first[g]:first[g] + count[g]]
        p = P[idx]
        c[g] = 0.5 * (p.min(0) + p.max(0))
        r[g] = np.sqrt(((p - c[g]) ** 2).sum(1)).max()
        amin[g] = a_old[idx].min()
    return c, r, amin


def visited_margin(nodes, c, r, alpha, G):
    """Smallest relative distance to a MAC threshold over the nodes the
    oracle's group walk visits (the root and the children of every opened
    internal node): min over visited J of |d - b_J| / b_J and
    |G M b_J^2 - alpha d^4| / (alpha d^4)."""
    cx, cy, cz, M, b = nodes["cx"], nodes["cy"], nodes["cz"], nodes["M"], nodes["b"]
    child, nchild = nodes["child"], nodes["nchild"]
    front = np.array([0], dtype=np.int64)
    best = np.inf
    while front.size:
        d = np.sqrt((cx[front] - c[0]) ** 2 + (cy[front] - c[1]) ** 2 + (cz[front] - c[2]) ** 2) - r
        bj = b[front]
        lhs = G * M[front] * bj * bj
        rhs = alpha * d ** 4
        with np.errstate(divide="ignore", invalid="ignore"):
            m1 = np.where(bj > 0, np.abs(d - bj) / bj, np.inf)
            m2 = np.where(rhs > 0, np.abs(lhs - rhs) / rhs, np.inf)
        best = min(best, float(np.min(np.minimum(m1, m2))))
        accept = (d > bj) & (lhs <= rhs)
        opened = front[~accept & (nchild[front] > 0)]
        if not opened.size:
            break
        front = np.concatenate([np.arange(child[j], child[j] + nchild[j]) for j in opened])
    return best


def compare_groups(gpu_entries, ora_entries, flipped_budget, explain, margin_tol=1e-5):
    """Groups whose list lengths differ; each must be explained by a visited
    node within margin_tol of a threshold, and there may be at most
    flipped_budget of them.  Returns the flipped group indices and margins."""
    gpu_entries = np.asarray(gpu_entries, dtype=np.int64)
    ora_entries = np.asarray(ora_entries, dtype=np.int64)
    flipped = np.flatnonzero(gpu_entries != ora_entries)
    assert flipped.size <= flipped_budget, (flipped.size, flipped_budget)
    margins = np.array([explain(g) for g in flipped])
    assert np.all(margins < margin_tol), margins
    return flipped, margins
