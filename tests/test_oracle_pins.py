"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is either a value
printed in the paper (tests/golden/), a closed form, an invariant of the
definition, exact rational arithmetic (Python integers / fractions), or an
independent restatement (top-down recursive bisection against the bottom-up
Algorithm 1; a linear scan against std::upper_bound; finite differences
against the analytic gradient).
"""

import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

from conftest import GOLDEN
from oracle import oracle as o

TWO32 = 1 << 32


# ----------------------------------------------------------------------------
# helpers (test-side, independent of the oracle's code)
# ----------------------------------------------------------------------------

def load_forest_example():
    nodes = {}
    with open(os.path.join(GOLDEN, "forest_example.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "weights":
                w = [int(x) for x in tok[1:]]
            elif tok[0] == "cells":
                M = int(tok[1])
            elif tok[0] == "node":
                nodes[int(tok[1])] = (int(tok[2]), int(tok[3]))
            elif tok[0] == "guide":
                guide = [int(x) for x in tok[1:]]
    return w, M, nodes, guide


def bitlen(x):
    return int(x).bit_length()


def topdown_forest(K, cell):
    """Recursive bisection at the highest differing bit (Sec. 3.1: a radix tree
    over base-2 keys); among equal distances (only possible for equal keys)
    the rightmost split is taken.  Independent of Algorithm 1."""
    n = len(cell)
    nodes = {}

    def build(lo, hi):
        if lo == hi:
            return ~lo
        best, kbest = -1, None
        for k in range(lo, hi):
            d = bitlen(int(K[k]) ^ int(K[k + 1]))
            if d >= best:
                best, kbest = d, k
        nid = kbest + 1
        nodes[nid] = (build(lo, kbest), build(kbest + 1, hi))
        return nid

    a = 0
    while a < n:
        b = a
        while b + 1 < n and cell[b + 1] == cell[a]:
            b += 1
        top = build(a, b)
        nodes[a] = (~max(a - 1, 0), top)
        a = b + 1
    return nodes


def random_weights(rng, n, zeros=True, dups=True):
    kind = rng.integers(0, 4)
    if kind == 0:
        w = rng.uniform(0.01, 1.0, n)
    elif kind == 1:
        w = np.exp(rng.normal(0, 3, n))
    elif kind == 2:
        w = rng.integers(1, 5, n).astype(np.float64)  # many equal weights
    else:
        w = np.exp(rng.normal(0, 8, n))                # huge dynamic range
    if zeros and n > 1:
        z = rng.random(n) < 0.2
        w[z] = 0.0
        if w.max() == 0:
            w[rng.integers(0, n)] = 1.0
    return w.astype(np.float32)


def definition_index(C, u):
    """P^{-1}(xi) = i <=> P_{i-1} <= xi < P_i with xi = u / 2^32, P = C / T,
    in exact integers: C_i 2^32 <= u T < C_{i+1} 2^32 (linear scan)."""
    T = int(C[-1])
    for i in range(len(C) - 1):
        if int(C[i]) * TWO32 <= u * T < int(C[i + 1]) * TWO32:
            return i
    raise AssertionError("no interval contains the sample")


def grid_samples(k, extra=()):
    return [j << (32 - k) for j in range(1 << k)] + list(extra)


# ----------------------------------------------------------------------------
# worked example (Fig. 11) and printed densities (Fig. 7)
# ----------------------------------------------------------------------------

def test_worked_forest_fig11_node_for_node():
    w, M, nodes, guide = load_forest_example()
    st = o.build(np.array(w, np.float32), M)
    assert st.T > 0
    for j in range(len(w)):
        assert tuple(st.nodes[j]) == nodes[j], f"node {j}"
    assert st.guide.tolist() == guide


def test_worked_forest_fig11_topdown_agrees():
    w, M, nodes, _ = load_forest_example()
    st = o.build(np.array(w, np.float32), M)
    K, cell = o.keys(st.C, M)
    assert topdown_forest(K, cell) == nodes


def test_float_bit_xor_does_not_reproduce_fig11():
    """Reading of the distance (Sec. 3.1 text vs Fig. 11): XOR of IEEE float
    bits of the normalised CDF would split cell 0 between leaves 0 and 1; the
    figure splits it between leaves 2 and 3, as the fixed-point keys do."""
    w, M, nodes, _ = load_forest_example()
    T = sum(w)
    cdf = np.cumsum([0] + w)[:-1] / T
    bits = np.array(cdf, np.float32).view(np.uint32).astype(np.int64)
    d = [bitlen(bits[k] ^ bits[k + 1]) for k in range(3)]
    assert int(np.argmax(d)) != 2
    assert nodes[0][1] == 3  # the figure's cell-0 tree splits at leaf 3


def load_fig7():
    d = np.loadtxt(os.path.join(GOLDEN, "sine64_fig7.txt"))
    return d


def test_fig7_target_density_is_sine64():
    d = load_fig7()
    p = np.array([(1 - math.cos(2 * math.pi * i / 64)) / 64 for i in range(64)])
    assert np.abs(d[:, 1] - np.round(p, 6)).max() == 0.0


@pytest.mark.parametrize("N,col", [(512, 2), (2048, 3)])
def test_fig7_monotone_counts_reproduced_by_index(N, col):
    """The printed sample densities of the monotonic mapping equal, bin for
    bin, the inverse CDF (P_{i-1} <= xi < P_i) over the float32 running sum of
    the sine-64 density with xi = j / N.  The oracle's index function, given
    that CDF as exact integers, reproduces every count."""
    d = load_fig7()
    p = np.array([(1 - math.cos(2 * math.pi * i / 64)) / 64 for i in range(64)])
    c32 = np.cumsum(p.astype(np.float32), dtype=np.float32)
    C = np.zeros(65, np.uint64)
    for k in range(64):
        C[k + 1] = int(Fraction(float(c32[k])) * (1 << 40))
    k = int(math.log2(N))
    u = np.array(grid_samples(k), np.uint32)
    idx, _ = o.sample(C, u)
    counts = np.bincount(idx, minlength=64)
    fig = np.round(d[:, col] * N).astype(int)
    assert counts.tolist() == fig.tolist()


@pytest.mark.parametrize("N", [512, 2048])
def test_fig7_exact_pipeline_stratified(N):
    """The exact pipeline on the same density keeps every count within one of
    p_i N (as the printed monotone densities do)."""
    d = load_fig7()
    p = np.array([(1 - math.cos(2 * math.pi * i / 64)) / 64 for i in range(64)])
    st = o.build(p.astype(np.float32), 64)
    k = int(math.log2(N))
    idx, _ = o.sample(st.C, np.array(grid_samples(k), np.uint32))
    counts = np.bincount(idx, minlength=64)
    fig = np.round(d[:, 2 if N == 512 else 3] * N).astype(int)
    q = np.diff(st.C.astype(object))
    for i in range(64):
        assert abs(Fraction(int(counts[i])) - Fraction(int(q[i]) * N, st.T)) < 1
        assert abs(int(counts[i]) - int(fig[i])) <= 2
    assert counts.sum() == N


# ----------------------------------------------------------------------------
# quantisation, CDF, keys
# ----------------------------------------------------------------------------

def test_quantisation_properties():
    rng = np.random.default_rng(1)
    for trial in range(40):
        n = int(rng.integers(1, 3000))
        w = random_weights(rng, n)
        if trial % 7 == 0:
            w[0] = np.float32(1e-40)      # subnormal
        S = o.scale(w)
        q = o.quantize(w, S)
        B = 62 - math.ceil(math.log2(n)) if n > 1 else 62
        qmax = int(q.max())
        assert (1 << (B - 1)) <= qmax < (1 << B)
        C = o.cdf(q)
        assert int(C[-1]) == sum(int(x) for x in q) < (1 << 62)
        # truncation error below one unit, exact rationals
        for i in rng.integers(0, n, 20):
            exact = Fraction(float(w[i])) * Fraction(2) ** S
            assert 0 <= exact - int(q[i]) < 1
        # monotone in the weight
        order = np.argsort(w, kind="stable")
        assert np.all(np.diff(q[order].astype(np.float64)) >= 0)
        # a common power of two does not change the integers
        w2 = (w * np.float32(2.0 ** 5)).astype(np.float32)
        assert np.array_equal(o.quantize(w2, o.scale(w2)), q)


def test_scale_rejects_bad_weights():
    for bad in ([1.0, -1.0], [np.nan, 1.0], [np.inf, 1.0], [0.0, 0.0]):
        with pytest.raises(o.OracleError):
            o.scale(np.array(bad, np.float32))


def test_worst_case_total_below_2_62():
    """n weights all just below a power of two: the largest possible total."""
    for n in (1, 2, 3, 1000, 1024, 1025, 1 << 16):
        w = np.full(n, np.nextafter(np.float32(2.0), np.float32(0)), np.float32)
        q = o.quantize(w, o.scale(w))
        assert sum(int(x) for x in q) < (1 << 62)


def test_keys_are_sample_domain_bounds():
    """K_j is the smallest u with floor(u T / 2^32) >= C_j."""
    rng = np.random.default_rng(2)
    for _ in range(30):
        w = random_weights(rng, int(rng.integers(1, 200)))
        st = o.build(w, 16)
        K, cell = o.keys(st.C, 16)
        T = st.T
        assert int(K[0]) == 0 and int(K[-1]) == TWO32
        for j in range(st.n + 1):
            Kj, Cj = int(K[j]), int(st.C[j])
            assert (Kj * T) >> 32 >= Cj
            if Kj > 0:
                assert ((Kj - 1) * T) >> 32 < Cj
        assert np.all(np.diff(K.astype(np.float64)) >= 0)
        assert np.all(cell == (K[:-1].astype(object) * 16 >> 32).astype(np.int64))


# ----------------------------------------------------------------------------
# index and position
# ----------------------------------------------------------------------------

def test_index_equals_definition_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(60):
        n = int(rng.integers(1, 17))
        w = random_weights(rng, n)
        st = o.build(w, 8)
        K, _ = o.keys(st.C, 8)
        us = grid_samples(8, extra=[int(x) for x in K[1:-1] if int(x) < TWO32] +
                          [int(x) - 1 for x in K[1:-1] if 0 < int(x) <= TWO32] +
                          [TWO32 - 1])
        for u in us:
            assert o.index(st.C, u) == definition_index(st.C, u)


def test_position_exact_rational():
    rng = np.random.default_rng(4)
    for _ in range(30):
        w = random_weights(rng, int(rng.integers(1, 100)))
        st = o.build(w, 8)
        T = st.T
        for u in rng.integers(0, TWO32, 50, dtype=np.uint64):
            u = int(u)
            i = o.index(st.C, u)
            exact = Fraction(u * T - int(st.C[i]) * TWO32,
                             (int(st.C[i + 1]) - int(st.C[i])) * TWO32)
            assert 0 <= exact < 1
            got = o.position(st.C, u, i)
            assert abs(Fraction(got) - exact) <= Fraction(1, 1 << 50) * max(exact, Fraction(1, 1 << 60)) + Fraction(1, 1 << 100)


def test_position_single_bin_is_xi():
    for wv in (0.3, 1.0, 7.5e-30, 3.4e38):
        st = o.build(np.array([wv], np.float32), 4)
        for u in (0, 1, 12345, 1 << 31, TWO32 - 1):
            assert o.index(st.C, u) == 0
            assert abs(o.position(st.C, u, 0) - u / TWO32) <= 2.0 ** -52 * (u / TWO32)


def test_stratified_counts_within_one():
    """For u = j 2^{32-k}: count_i = ceil(C_{i+1} 2^k / T) - ceil(C_i 2^k / T),
    so |count_i - p_i 2^k| < 1 strictly and the counts sum to 2^k."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = int(rng.integers(1, 300))
        w = random_weights(rng, n)
        st = o.build(w, 32)
        k = int(rng.integers(4, 13))
        idx, _ = o.sample(st.C, np.array(grid_samples(k), np.uint32))
        counts = np.bincount(idx, minlength=n)
        assert counts.sum() == 1 << k
        q = np.diff(st.C.astype(object))
        for i in range(n):
            assert abs(Fraction(int(counts[i])) - Fraction(int(q[i]) << k, st.T)) < 1


def test_monotone_mapping():
    rng = np.random.default_rng(6)
    w = random_weights(rng, 500)
    st = o.build(w, 64)
    u = np.sort(rng.integers(0, TWO32, 20000, dtype=np.uint64)).astype(np.uint32)
    idx, pos = o.sample(st.C, u)
    assert np.all(np.diff(idx) >= 0)
    same = np.diff(idx) == 0
    assert np.all(np.diff(pos)[same] >= 0)
    assert np.all((pos >= 0) & (pos <= 1))
    # zero-width bins are never selected
    q = np.diff(st.C.astype(np.float64))
    assert np.all(q[idx] > 0)


# ----------------------------------------------------------------------------
# forest (Algorithm 1), guide, Algorithm 2
# ----------------------------------------------------------------------------

def forest_cases(seed, count, nmax=40):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(1, nmax))
        M = int(rng.choice([1, 2, 3, 4, 5, 8, 12, 16, 64]))
        w = random_weights(rng, n)
        yield w, M, o.build(w, M)


def test_forest_equals_topdown_definition():
    for w, M, st in forest_cases(7, 300):
        K, cell = o.keys(st.C, M)
        ref = topdown_forest(K, cell)
        for j in range(st.n):
            assert tuple(st.nodes[j]) == ref[j], (w.tolist(), M, j)


def subtree_range(nodes, ref):
    if ref < 0:
        return ~ref, ~ref
    lo, _ = subtree_range(nodes, int(nodes[ref][0]))
    _, hi = subtree_range(nodes, int(nodes[ref][1]))
    return lo, hi


def test_forest_invariants():
    for w, M, st in forest_cases(8, 200):
        K, cell = o.keys(st.C, M)
        n = st.n
        seen_nodes = []
        leaves = []

        def visit(ref, depth):
            if ref < 0:
                leaves.append(~ref)
                return depth
            seen_nodes.append(ref)
            lo, hi = subtree_range(st.nodes, ref)
            # node `ref` splits between leaves ref-1 and ref, at the highest
            # bit in which the keys of its range differ
            assert lo <= ref - 1 < ref <= hi
            top = bitlen(int(K[lo]) ^ int(K[hi]))
            if top > 0:
                b = top - 1
                assert (int(K[ref - 1]) >> b) & 1 == 0
                assert (int(K[ref]) >> b) & 1 == 1
                assert bitlen(int(K[ref - 1]) ^ int(K[ref])) == top
            return max(visit(int(st.nodes[ref][0]), depth + 1),
                       visit(int(st.nodes[ref][1]), depth + 1))

        a = 0
        while a < n:
            b = a
            while b + 1 < n and cell[b + 1] == cell[a]:
                b += 1
            seen_nodes.append(a)
            assert st.nodes[a][0] == ~max(a - 1, 0)
            leaves.clear()
            visit(int(st.nodes[a][1]), 1)
            assert leaves == list(range(a, b + 1))
            a = b + 1
        assert sorted(seen_nodes) == list(range(n))


def test_algorithm2_equals_inverse_cdf_everywhere():
    for w, M, st in forest_cases(9, 150):
        K, _ = o.keys(st.C, M)
        us = grid_samples(9, extra=[int(x) for x in K[1:-1] if int(x) < TWO32] +
                          [int(x) - 1 for x in K[1:-1] if 0 < int(x) <= TWO32] +
                          [TWO32 - 1])
        for u in us:
            assert o.descend(st.guide, st.nodes, K, M, u) == o.index(st.C, u)


def test_guide_single_interval_brute_force():
    """A cell that exactly one interval of non-zero width overlaps stores ~i;
    every other cell stores its first key's leaf (the root of its tree)."""
    for w, M, st in forest_cases(10, 200):
        K, cell = o.keys(st.C, M)
        for g in range(M):
            s0 = -(-(g << 32) // M)
            s1 = -(-((g + 1) << 32) // M)
            over = [i for i in range(st.n)
                    if int(K[i]) < int(K[i + 1]) and int(K[i]) < s1 and int(K[i + 1]) > s0]
            if len(over) == 1:
                assert st.guide[g] == ~over[0]
            else:
                first = [j for j in range(st.n) if cell[j] == g]
                assert st.guide[g] == first[0]


def topdown_visits(K, cell, M, u):
    """Node visits of Algorithm 2 for sample u, from the top-down definition
    of the cell's tree: none when one interval covers the sample's cell (no key
    in it, or all its keys at the cell's start), else the cell's root (whose
    left child is the interval before the cell's first key) and one inner node
    per bisection that isolates the sample's interval."""
    g = (u * M) >> 32
    idx = [j for j in range(len(cell)) if int(cell[j]) == g]
    start = -((-g * TWO32) // M)  # smallest u of cell g
    if not idx or all(int(K[j]) == start for j in idx):
        return 0
    a, b = idx[0], idx[-1]
    if u < int(K[a]):
        return 1
    lo, hi, visits = a, b, 1
    while lo < hi:
        best, kb = -1, None
        for k in range(lo, hi):
            d = bitlen(int(K[k]) ^ int(K[k + 1]))
            if d >= best:
                best, kb = d, k
        visits += 1
        if u < int(K[kb + 1]):
            hi = kb
        else:
            lo = kb + 1
    return visits


def test_descent_steps_equal_topdown_depth():
    """The load counts behind Table 1: visits of Algorithm 2 on the oracle's
    structure equal the depth of the sample's interval in the top-down tree of
    its cell (0 for a covered cell, 1 for the interval left of the cell's first
    key), at every key, key - 1 and grid point."""
    for w, M, st in forest_cases(17, 150):
        K, cell = o.keys(st.C, M)
        us = set(grid_samples(6))
        for k in K[:-1] if len(K) > len(cell) else K:
            for d in (-1, 0, 1):
                if 0 <= int(k) + d < TWO32:
                    us.add(int(k) + d)
        for u in sorted(us):
            assert o.descend_steps(st.guide, st.nodes, K, M, u) == topdown_visits(K, cell, M, u), \
                (w.tolist(), M, u)


def test_descent_depth_bound_power_of_two_cells():
    """With 2^m cells, in-cell keys differ only in their low 32-m bits, so a
    reachable path visits at most 1 + (32 - m) nodes."""
    rng = np.random.default_rng(11)
    for _ in range(30):
        n = int(rng.integers(2, 400))
        m = int(rng.integers(0, 9))
        w = random_weights(rng, n)
        st = o.build(w, 1 << m)
        K, _ = o.keys(st.C, 1 << m)
        for u in rng.integers(0, TWO32, 300, dtype=np.uint64):
            assert o.descend_steps(st.guide, st.nodes, K, 1 << m, int(u)) <= 1 + (32 - m)


# ----------------------------------------------------------------------------
# 4-ary records (two binary levels collapsed)
# ----------------------------------------------------------------------------

def test_quad_descent_equals_inverse_cdf_everywhere():
    """The 4-ary descent finds the interval of the definition P_{i-1} <= xi < P_i
    at every grid point and at every key and key - 1 (deep single-cell trees
    included: M = 1)."""
    for w, M, st in forest_cases(21, 150, nmax=120):
        K, _ = o.keys(st.C, M)
        split, child = o.quad(st.nodes)
        us = grid_samples(8, extra=[int(x) for x in K[1:-1] if int(x) < TWO32] +
                          [int(x) - 1 for x in K[1:-1] if 0 < int(x) <= TWO32] +
                          [TWO32 - 1])
        for u in us:
            i, _ = o.descend_quad(st.guide, st.nodes, split, child, K, M, u)
            assert i == o.index(st.C, u), (w.tolist(), M, u)


def test_quad_records_halve_the_binary_visits():
    """Below the root decision, a path of v - 1 binary node visits reads
    ceil((v - 1) / 2) 4-ary records (v = visits of Algorithm 2, root included)."""
    rng = np.random.default_rng(22)
    for w, M, st in forest_cases(22, 120, nmax=300):
        K, _ = o.keys(st.C, M)
        split, child = o.quad(st.nodes)
        for u in rng.integers(0, TWO32, 200, dtype=np.uint64):
            v = o.descend_steps(st.guide, st.nodes, K, M, int(u))
            _, r = o.descend_quad(st.guide, st.nodes, split, child, K, M, int(u))
            assert r == (0 if v == 0 else v // 2), (v, r)


def test_quad_record_splits_in_key_order():
    """The three splits of a record are the left child, the node and the right
    child (or the node itself for a leaf side): keys ascend, and a leaf side
    names its leaf twice."""
    for w, M, st in forest_cases(23, 100, nmax=200):
        K, _ = o.keys(st.C, M)
        split, child = o.quad(st.nodes)
        for j in range(st.n):
            a, b = st.nodes[j]
            assert split[j, 1] == j
            assert K[split[j, 0]] <= K[j] <= K[split[j, 2]]
            if a < 0:
                assert split[j, 0] == j and child[j, 0] == child[j, 1] == a
            else:
                assert split[j, 0] == a and tuple(child[j, :2]) == tuple(st.nodes[a])
            if b < 0:
                assert split[j, 2] == j and child[j, 2] == child[j, 3] == b
            else:
                assert split[j, 2] == b and tuple(child[j, 2:]) == tuple(st.nodes[b])


# ----------------------------------------------------------------------------
# batched and 2-D
# ----------------------------------------------------------------------------

def test_env_map_marginal_is_row_totals_and_stratified():
    rng = np.random.default_rng(12)
    H, W = 16, 32
    lum = np.exp(rng.normal(0, 1, (H, W))).astype(np.float32)
    rows, marg = o.build_env(lum, 16, 32)
    S = o.scale(lum.reshape(-1), n_group=H * W)
    tot = [sum(int(x) for x in o.quantize(lum[r], S)) for r in range(H)]
    assert [int(x) for x in np.diff(marg.C.astype(object))] == tot
    assert marg.T == sum(tot) < (1 << 62)
    # stratified 2-D grid: each row hit within one of its probability
    k1, k2 = 6, 5
    u1 = np.repeat(np.array(grid_samples(k1), np.uint32), 1 << k2)
    u2 = np.tile(np.array(grid_samples(k2), np.uint32), 1 << k1)
    r, c, pr, pc = o.sample_env(rows, marg, u1, u2)
    cnt = np.bincount(r, minlength=H)
    for i in range(H):
        assert abs(Fraction(int(cnt[i]), 1 << k2) - Fraction(tot[i] << k1, marg.T)) < 1
    assert np.all((pc >= 0) & (pc <= 1)) and np.all((pr >= 0) & (pr <= 1))


def test_env_sampling_equals_definition_brute_force():
    """Component-wise 2-D sampling (Sec. 5) against its definition in Python
    integers: the shared scale from the largest exponent of the whole map, the
    row as the largest index whose marginal prefix sum is at most
    floor(u1 T / 2^32), the column likewise in that row with u2 and the row's
    total, and both positions as exact rationals."""
    rng = np.random.default_rng(21)
    H, W = 5, 7
    lum = np.exp(rng.normal(0, 1.5, (H, W))).astype(np.float32)
    lum[1, 3] = 0.0  # a zero-width bin inside a row
    lum[3, 0] = 0.0  # and one at a row's start
    rows, marg = o.build_env(lum, 2, 3)
    B = 62 - math.ceil(math.log2(H * W))
    e_max = max(math.frexp(float(x))[1] - 1 for x in lum.reshape(-1) if x > 0)
    S = B - 1 - e_max
    q = [[math.floor(Fraction(float(x)) * 2 ** S) for x in lum[r]] for r in range(H)]
    R = [sum(row) for row in q]
    T = sum(R)
    u1 = rng.integers(0, TWO32, 3000, dtype=np.uint64).astype(np.uint32)
    u2 = rng.integers(0, TWO32, 3000, dtype=np.uint64).astype(np.uint32)
    u1[:4] = [0, TWO32 - 1, 0, TWO32 - 1]
    u2[:4] = [0, 0, TWO32 - 1, TWO32 - 1]
    r, c, pr, pc = o.sample_env(rows, marg, u1, u2)
    for k in range(u1.size):
        a, b = int(u1[k]), int(u2[k])
        t1 = (a * T) >> 32
        rr = max(i for i in range(H) if sum(R[:i]) <= t1)
        assert r[k] == rr
        t2 = (b * R[rr]) >> 32
        cc = max(j for j in range(W) if sum(q[rr][:j]) <= t2)
        assert c[k] == cc
        xr = Fraction(a * T - sum(R[:rr]) * TWO32, R[rr] * TWO32)
        xc = Fraction(b * R[rr] - sum(q[rr][:cc]) * TWO32, q[rr][cc] * TWO32)
        assert 0 <= xr < 1 and 0 <= xc < 1
        assert abs(pr[k] - float(xr)) <= 1e-15 and abs(pc[k] - float(xc)) <= 1e-15


def test_batched_equals_independent_builds():
    rng = np.random.default_rng(13)
    sizes = [1, 7, 64, 300]
    w = np.concatenate([random_weights(rng, s) for s in sizes])
    off = np.concatenate([[0], np.cumsum(sizes)])
    Ms = [2, 8, 16, 64]
    outs = o.build_batched(w, off, Ms)
    for d, st in enumerate(outs):
        ref = o.build(w[off[d]:off[d + 1]], Ms[d])
        assert np.array_equal(st.C, ref.C)
        assert np.array_equal(st.nodes, ref.nodes)
        assert np.array_equal(st.guide, ref.guide)


# ----------------------------------------------------------------------------
# gradient
# ----------------------------------------------------------------------------

def relaxed_forward(w64, u, idx):
    """x = (xi W - C_i) / w_i with real weights (test-side numpy restatement)."""
    C = np.concatenate([[0.0], np.cumsum(w64)])
    xi = u.astype(np.float64) / 2.0 ** 32
    return (xi * C[-1] - C[idx]) / w64[idx]


def exact_quantized(w, S):
    """floor(w 2^S) 2^-S as an exact rational, from the float's own value."""
    v = Fraction(float(w)) * Fraction(2) ** S
    return Fraction(math.floor(v)) / Fraction(2) ** S


def test_quantized_weights_exact_rational():
    rng = np.random.default_rng(17)
    for _ in range(20):
        n = int(rng.integers(1, 300))
        w = random_weights(rng, n)
        S = o.scale(w)
        wq = o.quantized_weights(w, S)
        for k in range(n):
            assert Fraction(float(wq[k])) == exact_quantized(w[k], S)


def test_relaxation_at_quantised_weights_is_the_computed_forward():
    """The gradient's reading: the function differentiated is the relaxation
    at w' = floor(w 2^S) 2^-S, which equals the exact position the pipeline
    computes; at the unquantised weights it does not (here a weight whose
    low bits fall below the grid 2^-S of a distribution with a large
    weight)."""
    rng = np.random.default_rng(14)
    w = np.exp(rng.normal(0, 1, 200)).astype(np.float32)
    st = o.build(w, 64)
    u = rng.integers(0, TWO32, 2000, dtype=np.uint64).astype(np.uint32)
    idx, pos = o.sample(st.C, u)
    wq = o.quantized_weights(w, st.S)
    assert np.abs(relaxed_forward(wq, u, idx) - pos).max() < 1e-12
    x2 = o.relaxed_position(wq, u, idx)
    assert np.abs(x2 - relaxed_forward(wq, u, idx)).max() < 1e-12
    # n = 2 in a group of 2^30 weights (B = 32), w = (1, 1.75 2^-30): S = 31,
    # q = (2^31, floor(3.5) = 3), T = 2^31 + 3; the top samples land in bin 1
    w2 = np.array([1.0, 1.75 * 2.0 ** -30], np.float32)
    st2 = o.build(w2, 4, n_group=1 << 30)
    assert st2.S == 31 and int(st2.C[2] - st2.C[1]) == 3
    u2 = np.array([TWO32 - 1, TWO32 - 3], np.uint32)
    i2, p2 = o.sample(st2.C, u2)
    assert (i2 == 1).all()
    wq2 = o.quantized_weights(w2, st2.S)
    # the exact position, in rationals, equals the relaxation at w'
    Tq = int(st2.C[2])
    for k in range(2):
        exact = Fraction(int(u2[k]) * Tq - int(st2.C[1]) * TWO32, 3 * TWO32)
        assert abs(float(exact) - p2[k]) < 1e-15
    assert np.abs(relaxed_forward(wq2, u2, i2) - p2).max() < 1e-6
    assert np.abs(relaxed_forward(w2.astype(np.float64), u2, i2) - p2).max() > 0.05


def fd_gradient(w64, u, idx, g, h_rel=1e-3):
    """Central differences of the relaxed forward, weight by weight."""
    fd = np.zeros(w64.size)
    for k in range(w64.size):
        h = h_rel * w64[k]
        wp, wm = w64.copy(), w64.copy()
        wp[k] += h
        wm[k] -= h
        fd[k] = np.dot(g.astype(np.float64),
                       (relaxed_forward(wp, u, idx) - relaxed_forward(wm, u, idx)) / (2 * h))
    return fd


def test_gradient_central_differences():
    """Element by element against central differences of the relaxation at
    the quantised weights, on samples away from the bin edges."""
    rng = np.random.default_rng(15)
    n = 24
    w = np.exp(rng.normal(0, 1, n)).astype(np.float32)
    st = o.build(w, 16)
    u = rng.integers(0, TWO32, 400, dtype=np.uint64).astype(np.uint32)
    idx, pos = o.sample(st.C, u)
    keep = (pos > 0.01) & (pos < 0.99)
    u, idx = u[keep], idx[keep]
    g = rng.normal(0, 1, u.size).astype(np.float32)
    grad = o.grad(w, u, idx, g)
    fd = fd_gradient(o.quantized_weights(w, st.S), u, idx, g)
    assert np.all(np.abs(grad - fd) <= 1e-5 * (np.abs(fd) + np.abs(fd).max() * 1e-3))


def test_gradient_is_taken_at_the_quantised_weights():
    """A group of 2^54 weights (B = 8: about 7 significant bits per weight
    survive the quantisation): the gradient agrees with the differences of the
    relaxation at w' and not with those at the unquantised weights, so
    dividing by w instead of w' fails."""
    rng = np.random.default_rng(18)
    n, ng = 40, 1 << 54
    w = np.exp(rng.normal(0, 1, n)).astype(np.float32)
    st = o.build(w, 16, n_group=ng)
    wq = o.quantized_weights(w, st.S)
    assert (wq > 0).all()
    assert np.abs(wq / w - 1.0).max() > 1e-3
    u = rng.integers(0, TWO32, 4000, dtype=np.uint64).astype(np.uint32)
    idx, pos = o.sample(st.C, u)
    keep = (pos > 0.01) & (pos < 0.99)
    u, idx = u[keep], idx[keep]
    g = rng.normal(0, 1, u.size).astype(np.float32)
    grad = o.grad(w, u, idx, g, n_group=ng)
    fd_q = fd_gradient(wq, u, idx, g)
    fd_w = fd_gradient(w.astype(np.float64), u, idx, g)
    assert np.all(np.abs(grad - fd_q) <= 1e-5 * (np.abs(fd_q) + np.abs(fd_q).max() * 1e-3))
    assert np.abs(grad - fd_w).max() > 1e-3 * np.abs(fd_w).max()


def test_gradient_single_bin_is_zero():
    w = np.array([2.5], np.float32)
    u = np.array([0, 5, 1 << 31, TWO32 - 1], np.uint32)
    g = np.array([1.0, -2.0, 0.5, 3.0], np.float32)
    assert np.abs(o.grad(w, u, np.zeros(4, np.int32), g)).max() < 1e-15


def test_gradient_two_bins_closed_form():
    """Two bins, one sample in bin 1: x = (xi (w0 + w1) - w0) / w1, so
    dx/dw0 = (xi - 1) / w1 and dx/dw1 = (xi - x) / w1 (1 and 3 lie on the
    quantisation grid, so w' = w)."""
    w = np.array([1.0, 3.0], np.float32)
    u = np.array([3 << 30], np.uint32)   # xi = 0.75 -> bin 1 (P_1 = 0.25)
    xi = 0.75
    x = (xi * 4.0 - 1.0) / 3.0
    grad = o.grad(w, u, np.array([1], np.int32), np.array([1.0], np.float32))
    assert abs(grad[0] - (xi - 1) / 3.0) < 1e-15
    assert abs(grad[1] - (xi - x) / 3.0) < 1e-15


def relaxed_forward_2d(lum64, u1, u2, r, c):
    """Relaxed 2-D forward (test-side): row position through the row sums,
    column position through the row's weights."""
    R = lum64.sum(axis=1)
    Cm = np.concatenate([[0.0], np.cumsum(R)])
    xi1 = u1.astype(np.float64) / 2.0 ** 32
    xi2 = u2.astype(np.float64) / 2.0 ** 32
    y = (xi1 * Cm[-1] - Cm[r]) / R[r]
    Crow = np.concatenate([np.zeros((lum64.shape[0], 1)), np.cumsum(lum64, axis=1)], axis=1)
    x = (xi2 * R[r] - Crow[r, c]) / lum64[r, c]
    return y, x


def test_env_gradient_central_differences():
    """2-D: element by element against central differences of the relaxation
    at the quantised map (shared scale), whose row sums are the marginal's
    exact row totals; the relaxation there equals the exact positions."""
    rng = np.random.default_rng(16)
    H, Wd = 5, 7
    lum = np.exp(rng.normal(0, 1, (H, Wd))).astype(np.float32)
    rows, marg = o.build_env(lum, 8, 8)
    u1 = rng.integers(0, TWO32, 600, dtype=np.uint64).astype(np.uint32)
    u2 = rng.integers(0, TWO32, 600, dtype=np.uint64).astype(np.uint32)
    r, c, pr, pc = o.sample_env(rows, marg, u1, u2)
    keep = (pr > 0.01) & (pr < 0.99) & (pc > 0.01) & (pc < 0.99)
    u1, u2, r, c = u1[keep], u2[keep], r[keep], c[keep]
    pr, pc = pr[keep], pc[keep]
    gy = rng.normal(0, 1, u1.size).astype(np.float32)
    gx = rng.normal(0, 1, u1.size).astype(np.float32)
    grad = o.grad_env(lum, u1, u2, r, c, gy, gx)
    lq = o.quantized_weights(lum.reshape(-1), marg.S).reshape(H, Wd)
    y0, x0 = relaxed_forward_2d(lq, u1, u2, r, c)
    assert np.abs(y0 - pr).max() < 1e-12 and np.abs(x0 - pc).max() < 1e-12
    fd = np.zeros((H, Wd))
    for k in range(H):
        for j in range(Wd):
            h = 1e-3 * lq[k, j]
            lp, lm = lq.copy(), lq.copy()
            lp[k, j] += h
            lm[k, j] -= h
            yp, xp = relaxed_forward_2d(lp, u1, u2, r, c)
            ym, xm = relaxed_forward_2d(lm, u1, u2, r, c)
            fd[k, j] = (np.dot(gy.astype(np.float64), yp - ym) +
                        np.dot(gx.astype(np.float64), xp - xm)) / (2 * h)
    assert np.all(np.abs(grad - fd) <= 1e-5 * (np.abs(fd) + np.abs(fd).max() * 1e-3))
