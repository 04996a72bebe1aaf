"""The link rule of the forest kernel, restated on the CPU and checked against
the oracle's Algorithm 1.

The kernel does not climb: the node over the split between leaves k - 1 and k
covers the leaves between the nearest split on its left with a larger
distance and the nearest split on its right with a distance at least as
large, and its parent is the smaller of those two bounding splits (the right
one when the left is larger, then as child 0; otherwise the left one, as
child 1).  A leaf is the range between its own two splits.  Inside a tile the
two nearest splits are searched among the tile's positions (its interior
splits and the two splits on its edges); a node whose search leaves the tile
and whose parent is not settled by the side it did find goes to a merge pass.
The kernel holds at most 72 such nodes per tile; the bound argued in the
source is 66.

Distances here come from the oracle's keys (Sec. 3.1: the bit length of the
XOR of neighbouring keys, a cell or array boundary counting as larger than
any distance).
"""

import numpy as np
import pytest

from oracle import oracle as o

INF = 64
UNRES_BOUND = 66


def distances(K, cell):
    """delta_j between leaves j and j + 1 (j = 0..n-1); INF across cells and
    after the last leaf."""
    n = cell.size
    d = np.full(n, INF, np.int64)
    for j in range(n - 1):
        if cell[j] == cell[j + 1]:
            d[j] = int(int(K[j]) ^ int(K[j + 1])).bit_length()
    return d


def link_forest(d):
    """Child slots from the nearest-larger-distance rule over the whole array
    (the merge pass's view); returns nodes[n, 2] in the oracle's encoding."""
    n = d.size
    nodes = np.full((n, 2), 0x7FFFFFFF, np.int64)
    dd = lambda j: INF if j < 0 or j >= n else int(d[j])  # noqa: E731

    def set_slot(rec, c, val):
        assert nodes[rec, c] == 0x7FFFFFFF, "a child slot written twice"
        nodes[rec, c] = val

    for leaf in range(n):
        dl, dr = dd(leaf - 1), dd(leaf)
        if dl >= INF:
            set_slot(leaf, 0, ~max(leaf - 1, 0))
        if dl >= INF and dr >= INF:
            set_slot(leaf, 1, ~leaf)
        elif dl > dr:
            set_slot(leaf + 1, 0, ~leaf)
        else:
            set_slot(leaf, 1, ~leaf)
    for k in range(1, n):  # node k: split k - 1, between leaves k - 1 and k
        v = dd(k - 1)
        if v >= INF:
            continue
        jl = k - 2
        while jl >= 0 and dd(jl) <= v:
            jl -= 1
        jr = k
        while dd(jr) < v:
            jr += 1
        dl, dr = dd(jl), dd(jr)
        if dl >= INF and dr >= INF:
            set_slot(jl + 1, 1, k)
        elif dl > dr:
            set_slot(jr + 1, 0, k)
        else:
            set_slot(jl + 1, 1, k)
    assert (nodes != 0x7FFFFFFF).all(), "a child slot was never written"
    return nodes


def unresolved_per_tile(d, tile):
    """Nodes of each tile (positions p in [0, tn) of the tile, the split
    between leaves t0 + p - 1 and t0 + p) whose parent needs distances outside
    the tile: the right search fails, or the left one fails and the right
    bound's distance exceeds the node's."""
    n = d.size
    counts = []
    for t0 in range(0, n, tile):
        t1 = min(t0 + tile, n)
        tn = t1 - t0
        # tile positions 0..tn: the split between leaves t0 + p - 1 and t0 + p
        pos = [INF if (t0 + p - 1 < 0 or t0 + p - 1 >= n) else int(d[t0 + p - 1])
               for p in range(tn + 1)]
        cnt = 0
        for p in range(tn):
            v = pos[p]
            if v >= INF:
                continue
            pl = next((q for q in range(p - 1, -1, -1) if pos[q] > v), -1)
            pr = next((q for q in range(p + 1, tn + 1) if pos[q] >= v), -1)
            if pr < 0 or (pl < 0 and pos[pr] > v):
                cnt += 1
        counts.append(cnt)
    return counts


def random_case(rng, n):
    kind = rng.integers(0, 5)
    if kind == 0:
        w = rng.uniform(0.01, 1.0, n)
    elif kind == 1:
        w = np.exp(rng.normal(0, 3, n))
    elif kind == 2:
        w = rng.integers(1, 5, n).astype(np.float64)
    elif kind == 3:
        w = np.exp(rng.normal(0, 8, n))
    else:
        w = rng.uniform(0.5, 1.0, n)
        w[rng.random(n) < 0.6] = 0.0  # long runs of equal keys
        w[0] = 1.0
    return w.astype(np.float32)


@pytest.mark.parametrize("seed", range(6))
def test_link_rule_equals_algorithm1(seed):
    rng = np.random.default_rng(seed)
    for _ in range(12):
        n = int(rng.integers(1, 600))
        w = random_case(rng, n)
        M = int(1 << rng.integers(0, 9))
        st = o.build(w, M)
        K, cell = o.keys(st.C, M)
        nodes = link_forest(distances(K, cell))
        assert np.array_equal(nodes, st.nodes.astype(np.int64))


@pytest.mark.parametrize("tile", [4, 8, 32, 128])
def test_nodes_left_to_the_merge_pass_per_tile(tile):
    """At most 66 per tile for any tile size, including runs of equal keys
    (distance 0) and cells larger than a tile; with one cell over the whole
    array (M = 1) the count is largest."""
    rng = np.random.default_rng(100 + tile)
    worst = 0
    for _ in range(10):
        n = int(rng.integers(tile, 40 * tile))
        w = random_case(rng, n)
        for M in (1, 4, 64):
            st = o.build(w, M)
            K, cell = o.keys(st.C, M)
            counts = unresolved_per_tile(distances(K, cell), tile)
            worst = max(worst, max(counts))
    assert worst <= UNRES_BOUND
    assert worst > 0
