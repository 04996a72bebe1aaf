"""Parity of the CUDA path (through the C interface) with the CPU oracle.

Bit-exact: the integer CDF, the forest's child references, the guide table and
the sampled bin indices.  Floating point: the in-bin positions within 4 ulp of
the oracle's fp64 value rounded to float32 (the three roundings of the float32
quotient bound the error by 3 ulp plus the reference's half ulp).
"""

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1901_05423_gb300 import api
from paper_1901_05423_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
MAX_ULP = 4


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_05423_gb300 import _native
    _native.load()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def ulp_dist(pos_gpu, pos_ref64):
    a = np.ascontiguousarray(pos_gpu, dtype=np.float32).view(np.int32).astype(np.int64)
    b = np.asarray(pos_ref64, dtype=np.float64).astype(np.float32).view(np.int32).astype(np.int64)
    return np.abs(a - b)


def host_structure(f):
    """The forest's device arrays copied to the host once: CDF, children,
    guide table, guide records."""
    return (f.cdf().cpu().numpy().view(np.uint64), f.children().cpu().numpy(),
            f.guide.cpu().numpy(), f.guide_records().cpu().numpy())


def check_structure(f, ref, elem_off=0, guide_off=0, n=None, cells=None, host=None):
    host = host_structure(f) if host is None else host
    n = ref.n if n is None else n
    cells = ref.M if cells is None else cells
    C = host[0][elem_off:elem_off + n]
    ch = host[1][elem_off:elem_off + n]
    g = host[2][guide_off:guide_off + cells]
    assert np.array_equal(C, ref.C[:-1]), "CDF"
    bad = np.nonzero((ch != ref.nodes).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} node records differ, first {bad[:5]}"
    badg = np.nonzero(g != ref.guide)[0]
    assert badg.size == 0, f"{badg.size} guide cells differ, first {badg[:5]}"
    # guide records: a copy of each root's record with the bounds C_{j0-1} and
    # C_{j1+1} of the cell's outer intervals; {C_i, ~i, ~i, C_i, C_{i+1}} for a
    # cell that one interval i covers
    rec = host[3][guide_off:guide_off + cells]
    rec_c = rec[:, 0].view(np.uint64)
    rec_ch = rec[:, 1:2].copy().view(np.int32)
    rec_lo = rec[:, 2].view(np.uint64)
    rec_hi = rec[:, 3].view(np.uint64)
    _, cell = orc.keys(ref.C, cells)
    g_idx = np.arange(cells)
    root = ref.guide >= 0
    j0 = np.where(root, ref.guide, 0)
    j1 = np.searchsorted(cell, g_idx, side="right") - 1  # last leaf whose key lies in g
    i = np.where(root, 0, ~ref.guide)
    exp_c = np.where(root, ref.C[j0], ref.C[i])
    exp_c0 = np.where(root, ref.nodes[j0, 0], ref.guide)
    exp_c1 = np.where(root, ref.nodes[j0, 1], ref.guide)
    exp_lo = np.where(root, ref.C[np.maximum(j0 - 1, 0)], ref.C[i])
    exp_hi = np.where(root, ref.C[np.clip(j1 + 1, 0, n)], ref.C[i + 1])
    assert np.array_equal(rec_c, exp_c), "guide record CDF"
    assert np.array_equal(rec_ch[:, 0], exp_c0) and np.array_equal(rec_ch[:, 1], exp_c1), \
        "guide record children"
    assert np.array_equal(rec_lo, exp_lo), "guide record lower bound"
    assert np.array_equal(rec_hi, exp_hi), "guide record upper bound"


def oracle_builds(ws, ms, threads=None):
    """orc.build of every distribution (a thread pool over the independent
    builds; the oracle's calls release the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(threads or orc.host_threads()) as ex:
        return list(ex.map(lambda a: orc.build(a[0], 1 << int(a[1])), zip(ws, ms)))


def oracle_tagged(refs, u, dist):
    """Index and position of every tagged sample through the oracle of its
    distribution (samples grouped by distribution, a thread pool over the
    distributions)."""
    from concurrent.futures import ThreadPoolExecutor
    order = np.argsort(dist, kind="stable")
    bounds = np.searchsorted(dist[order], np.arange(len(refs) + 1))
    ridx = np.empty(u.size, np.int32)
    rpos = np.empty(u.size, np.float64)

    def run(d):
        sel = order[bounds[d]:bounds[d + 1]]
        if sel.size:
            i, p = orc.sample(refs[d].C, u[sel])
            ridx[sel] = i
            rpos[sel] = p

    with ThreadPoolExecutor(orc.host_threads()) as ex:
        list(ex.map(run, range(len(refs))))
    return ridx, rpos


def check_samples(idx, pos, ridx, rpos):
    idx = idx.cpu().numpy() if torch.is_tensor(idx) else idx
    pos = pos.cpu().numpy() if torch.is_tensor(pos) else pos
    bad = np.nonzero(idx != ridx)[0]
    assert bad.size == 0, f"{bad.size} indices differ, first at {bad[:5]}"
    d = ulp_dist(pos, rpos)
    assert d.max() <= MAX_ULP, f"position off by {d.max()} ulp"
    return int(d.max())


def build_and_check(w, m):
    f = api.rtf_build(to_dev(w), m)
    torch.cuda.synchronize()
    f.check_status()
    ref = orc.build(w, 1 << m)
    check_structure(f, ref)
    return f, ref


# ---------------------------------------------------------------------------
# single distribution
# ---------------------------------------------------------------------------

def test_config_small_uniform_radical_inverse():
    """n = 1024 uniform(0.01, 1) weights, 2^8 cells, 2^20 radical-inverse samples."""
    w = W.uniform_weights(1024, seed=0)
    f, ref = build_and_check(w, 8)
    u = W.radical_inverse_u32(1 << 20)
    idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV))
    ridx, rpos = orc.sample(ref.C, u)
    check_samples(idx, pos, ridx, rpos)


def weight_cases():
    rng = np.random.default_rng(123)
    sizes = [1, 2, 3, 4, 5, 31, 32, 33, 1023, 2047, 2048, 2049, 4095, 4096, 4097,
             3 * 2048 + 17, 20000]
    kinds = ["uniform", "lognormal2", "equal", "zeros", "spike", "range", "subnormal", "dups"]
    cases = []
    for n in sizes:
        for kind in kinds:
            if kind == "uniform":
                w = rng.uniform(0.01, 1, n)
            elif kind == "lognormal2":
                w = np.exp(rng.normal(0, 2, n))
            elif kind == "equal":
                w = np.full(n, 0.37)
            elif kind == "zeros":
                w = rng.uniform(0, 1, n) * (rng.random(n) < 0.3)
                if not w.any():
                    w[n // 2] = 1.0
            elif kind == "spike":
                w = np.full(n, 1e-3)
                w[rng.integers(0, n)] = 1e6
            elif kind == "range":
                w = np.exp(rng.normal(0, 12, n))
            elif kind == "subnormal":
                w = np.full(n, 1e-40)
                w[::7] = 3e-39
            else:
                w = np.repeat(rng.uniform(0.01, 1, (n + 7) // 8), 8)[:n] * (rng.random(n) < 0.8)
                if not w.any():
                    w[0] = 1.0
            cases.append((n, kind, w.astype(np.float32)))
    return cases


@pytest.mark.parametrize("m", [0, 1, 4, 9, 14])
def test_random_sizes_and_weight_kinds(m):
    rng = np.random.default_rng(m)
    for n, kind, w in weight_cases():
        f = api.rtf_build(to_dev(w), m)
        u = rng.integers(0, 1 << 32, 4096, dtype=np.uint64).astype(np.uint32)
        u[:3] = [0, 1, 0xFFFFFFFF]
        idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV))
        torch.cuda.synchronize()
        f.check_status()
        ref = orc.build(w, 1 << m)
        try:
            check_structure(f, ref)
            ridx, rpos = orc.sample(ref.C, u)
            check_samples(idx, pos, ridx, rpos)
        except AssertionError as e:
            raise AssertionError(f"n={n} kind={kind} m={m}: {e}")


def test_worked_example_fig11_cells_power_of_two():
    """The weights of the worked forest with 16 cells (the GPU supports 2^m)."""
    w = np.array([5, 1, 3, 2, 6, 6, 7, 6, 28, 2, 14, 33], np.float32)
    build_and_check(w, 4)


def test_rebuild_reuses_workspace():
    """Repeated builds through one cached workspace give identical structures."""
    w = W.lognormal_weights(50000, seed=3, sigma=2.0)
    f1, ref = build_and_check(w, 12)
    snap = f1.nodes.clone()
    for _ in range(3):
        f2 = api.rtf_build(to_dev(w), 12)
        torch.cuda.synchronize()
        f2.check_status()
        assert torch.equal(f2.nodes, snap)


def test_workspace_reused_across_sizes():
    """A workspace that served a larger batched build (whose regions lie
    elsewhere) serves smaller and differently shaped builds correctly."""
    wb, offb = W.ragged_batch(600, seed=9)
    sizes = np.diff(offb)
    ms = np.clip(np.round(np.log2(sizes)).astype(int), 3, 16)
    f = api.rtf_build_batched(to_dev(wb), sizes, ms)
    torch.cuda.synchronize()
    f.check_status()
    for n, m, seed in ((300000, 14, 1), (4097, 5, 2), (1 << 20, 18, 3)):
        w = W.lognormal_weights(n, seed=seed, sigma=2.0)
        build_and_check(w, m)


def test_status_bits_for_bad_weights():
    for bad, bit in (([1.0, -1.0, 2.0], api.STATUS_BAD_WEIGHT),
                     ([1.0, np.nan, 2.0], api.STATUS_BAD_WEIGHT),
                     ([np.inf, 1.0, 1.0], api.STATUS_BAD_WEIGHT),
                     ([0.0, 0.0, 0.0], api.STATUS_ZERO_TOTAL)):
        f = api.rtf_build(to_dev(np.array(bad, np.float32)), 2)
        torch.cuda.synchronize()
        assert int(f.status.item()) & bit
    # a good build afterwards is clean again
    build_and_check(np.array([1.0, 2.0, 3.0], np.float32), 2)


def test_monotone_on_sorted_samples():
    w = W.lognormal_weights(100000, seed=4, sigma=2.0)
    f = api.rtf_build(to_dev(w), 14)
    u = W.sorted_radical_inverse_u32(1 << 22)
    idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV))
    idx = idx.cpu().numpy()
    pos = pos.cpu().numpy()
    assert np.all(np.diff(idx) >= 0)
    same = np.diff(idx) == 0
    assert np.all(np.diff(pos)[same] >= 0)


# ---------------------------------------------------------------------------
# full size: n = 2^24 lognormal(0, 2), 2^20 cells
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big():
    w = W.lognormal_weights(1 << 24, seed=0, sigma=2.0)
    f = api.rtf_build(to_dev(w), 20)
    torch.cuda.synchronize()
    f.check_status()
    ref = orc.build(w, 1 << 20)
    return w, f, ref


def test_full_size_structure_bit_exact(big):
    w, f, ref = big
    check_structure(f, ref)


@pytest.mark.parametrize("m", [0, 2, 5])
def test_cells_spanning_groups_of_tiles(m):
    """Cells of 2^16 to 2^22 leaves span up to 32 groups of 64 tiles: the merge
    pass's searches leave their group (the warp-wide group search) for the
    tops of those cells, on both sides; the structure bit for bit.  A batch of
    the same weights cut into two distributions takes the segmented path."""
    n = (1 << 22) + 4097
    w = W.lognormal_weights(n, seed=40 + m, sigma=2.0)
    f = api.rtf_build(to_dev(w), m)
    torch.cuda.synchronize()
    f.check_status()
    check_structure(f, orc.build(w, 1 << m))
    cut = (1 << 21) + 1000
    fb = api.rtf_build_batched(to_dev(w), [cut, n - cut], [m, m])
    torch.cuda.synchronize()
    fb.check_status()
    host = host_structure(fb)
    check_structure(fb, orc.build(w[:cut], 1 << m), host=host)
    check_structure(fb, orc.build(w[cut:], 1 << m), elem_off=cut, guide_off=1 << m, host=host)


def test_full_size_samples(big):
    """Both sample sets at full size through the same launch configuration as
    the benchmark; the oracle checks every 64th sample of each."""
    w, f, ref = big
    n_s = 1 << 28
    # the benchmark maps the sorted set with the coherence hint (runs of
    # consecutive samples per thread)
    for name, u, mode in (("iid", W.iid_u32(n_s, seed=1), api.SAMPLE_1D),
                          ("sorted", W.sorted_radical_inverse_u32(n_s),
                           api.SAMPLE_1D | api.SAMPLE_COHERENT)):
        ud = api.u32_tensor(u, DEV)
        idx, pos = api.rtf_sample(f, ud, mode=mode)
        torch.cuda.synchronize()
        if mode & api.SAMPLE_COHERENT:
            # every sample, against the per-sample descent
            i2, p2 = api.rtf_sample(f, ud)
            assert torch.equal(idx, i2) and torch.equal(pos.view(torch.int32), p2.view(torch.int32))
            del i2, p2
        sel = np.arange(0, n_s, 64)
        sel = np.concatenate([sel, np.arange(n_s - 4096, n_s)])
        ridx, rpos = orc.sample(ref.C, u[sel])
        check_samples(idx[torch.from_numpy(sel).to(DEV)], pos[torch.from_numpy(sel).to(DEV)],
                      ridx, rpos)
        del ud, idx, pos


# ---------------------------------------------------------------------------
# batched
# ---------------------------------------------------------------------------

def batched_check(w, offsets, ms, samples_per=512, seed=0):
    """Every distribution's structure against the oracle's, and tagged samples
    (samples_per per distribution, up to 64 distributions' worth)."""
    sizes = np.diff(offsets)
    f = api.rtf_build_batched(to_dev(w), sizes, ms)
    torch.cuda.synchronize()
    f.check_status()
    goff = f.guide_offsets
    rng = np.random.default_rng(seed)
    D = len(sizes)
    dist = rng.integers(0, D, samples_per * min(D, 64), dtype=np.int64).astype(np.int32)
    u = rng.integers(0, 1 << 32, dist.size, dtype=np.uint64).astype(np.uint32)
    idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV), dist_id=to_dev(dist))
    refs = oracle_builds([w[offsets[d]:offsets[d + 1]] for d in range(D)], ms)
    host = host_structure(f)
    for d in range(D):
        check_structure(f, refs[d], elem_off=int(offsets[d]), guide_off=int(goff[d]), host=host)
    ridx, rpos = oracle_tagged(refs, u, dist)
    check_samples(idx, pos, ridx, rpos)
    return f


def test_batched_small_ragged():
    rng = np.random.default_rng(5)
    sizes = np.concatenate([[1, 2, 3, 2048, 2049, 1, 1], rng.integers(1, 5000, 300)])
    w = np.concatenate([W.lognormal_weights(int(s), seed=int(i), sigma=1.5)
                        for i, s in enumerate(sizes)])
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    ms = np.clip(np.ceil(np.log2(np.maximum(sizes, 1))).astype(int) - 1, 0, 16)
    batched_check(w, offsets, ms)


def test_batched_tile_aligned_boundaries():
    """Distribution boundaries on tile edges (2048 weights) and next to them,
    distributions of exactly one or several tiles, hundreds of one-to-three
    weight distributions inside one tile, leading and trailing zero weights:
    the cases of the single-distribution paths of the batched scale, tile-sum
    and forest passes (a head only at t0, an end only at t1) and of the table
    of each tile's first distribution; every structure against the oracle."""
    rng = np.random.default_rng(11)
    sizes = [2048, 2048, 4096, 1, 2047, 2049, 6144, 3, 2045, 4096 + 2048]
    sizes += list(rng.integers(1, 4, 400))
    cum = int(np.sum(sizes))
    sizes.append(2048 - cum % 2048 + 2048)  # realign the next boundary on a tile edge
    sizes += [2048, 1, 1, 2046, 8192, 2049, 2047]
    sizes = np.array(sizes, np.int64)
    parts = []
    for i, n in enumerate(sizes):
        x = W.lognormal_weights(int(n), seed=200 + i, sigma=1.5)
        if n > 8 and i % 3 == 0:
            x[:2] = 0.0  # leading zero-width bins
        if n > 8 and i % 3 == 1:
            x[-3:] = 0.0  # trailing zero-width bins (keys equal to 2^32)
        parts.append(x)
    w = np.concatenate(parts).astype(np.float32)
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    assert (offsets % 2048 == 0).sum() >= 8
    ms = np.clip(np.round(np.log2(sizes)).astype(int) + rng.integers(-2, 3, sizes.size), 0, 14)
    batched_check(w, offsets, ms)


def test_batched_ragged_full_config():
    """The ragged workload in full: 16384 distributions, sizes log-uniform in
    [8, 65536], lognormal(0, 1.5), the autotuned guide bits the benchmark
    uses, 2^27 samples with uniform distribution ids.  Every distribution's
    structure and every sample against the oracle; then the batched build and
    the tagged sampling captured in one CUDA graph and replayed twice give the
    same bits."""
    from paper_1901_05423_gb300 import autotune
    w, offsets = W.ragged_batch(16384, seed=0)
    sizes = np.diff(offsets)
    ms = autotune.guide_bits_for(sizes, autotune.tune(DEV))
    D = sizes.size
    wd = to_dev(w)
    f = api.rtf_build_batched(wd, sizes, ms)
    ns = 1 << 27
    u = W.iid_u32(ns, seed=1)
    dist = W.dist_ids(ns, D, seed=2)
    ud, dd = api.u32_tensor(u, DEV), to_dev(dist)
    idx, pos = api.rtf_sample(f, ud, dist_id=dd)
    torch.cuda.synchronize()
    f.check_status()
    goff = f.guide_offsets
    refs = oracle_builds([w[offsets[d]:offsets[d + 1]] for d in range(D)], ms)
    host = host_structure(f)
    for d in range(D):
        check_structure(f, refs[d], elem_off=int(offsets[d]), guide_off=int(goff[d]), host=host)
    ridx, rpos = oracle_tagged(refs, u, dist)
    check_samples(idx, pos, ridx, rpos)
    del ridx, rpos
    # graph capture of build + tagged sampling, replayed
    f.nodes.zero_()
    f.guide.zero_()
    idx2, pos2 = torch.zeros_like(idx), torch.zeros_like(pos)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            api.rtf_build_batched(wd, sizes, ms, forest=f, plan_dev=f._plan_dev)
            api.rtf_sample(f, ud, dist_id=dd, idx_out=idx2, pos_out=pos2)
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        f.check_status()
        h2 = host_structure(f)
        assert all(np.array_equal(a, b) for a, b in zip(host, h2))
        assert torch.equal(idx, idx2)
        assert torch.equal(pos.view(torch.int32), pos2.view(torch.int32))
        idx2.zero_()
        pos2.zero_()
        f.nodes.zero_()


# ---------------------------------------------------------------------------
# 2-D environment map (marginal + conditionals in one batched build)
# ---------------------------------------------------------------------------

def env_check(H, Wd, m_row, m_col, n_s, seed=0, stride=1):
    """The marginal's and every row's structure against the oracle's, and the
    sample pairs (every `stride`-th, plus the last 4096) against the oracle's
    component-wise sampling."""
    lum = W.env_map(H, Wd, seed=seed)
    sizes = [Wd] * H + [H]
    ms = [m_col] * H + [m_row]
    f = api.rtf_build_batched(to_dev(lum.reshape(-1)), sizes, ms, marginal=True)
    torch.cuda.synchronize()
    f.check_status()
    rows, marg = orc.build_env(lum, 1 << m_row, 1 << m_col)
    host = host_structure(f)
    check_structure(f, marg, elem_off=H * Wd, guide_off=H << m_col, host=host)
    for r in range(H):
        check_structure(f, rows[r], elem_off=r * Wd, guide_off=r << m_col, host=host)
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 1 << 32, 2 * n_s, dtype=np.uint64).astype(np.uint32)
    idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV), mode=api.SAMPLE_2D)
    idx = idx.cpu().numpy()
    pos = pos.cpu().numpy()
    sel = np.unique(np.concatenate([np.arange(0, n_s, stride),
                                    np.arange(max(0, n_s - 4096), n_s)]))
    r, c, pr, pc = orc.sample_env(rows, marg, u[2 * sel], u[2 * sel + 1])
    check_samples(idx[sel, 0], pos[sel, 0], r, pr)
    check_samples(idx[sel, 1], pos[sel, 1], c, pc)
    return f, lum


def test_env_map_small():
    env_check(64, 128, 6, 7, 1 << 16)
    env_check(48, 96, 5, 6, (1 << 12) + 3, seed=3)  # pairs left over after groups of four


def test_env_map_full_config():
    """4096 x 2048 luminance with hot spots; marginal over 2048 rows and 2048
    conditionals built in one batched launch sequence: every row and the
    marginal bit for bit; every 16th of the 2^26 sample pairs and the last
    4096 against the oracle."""
    env_check(2048, 4096, 12, 12, 1 << 26, stride=16)


# ---------------------------------------------------------------------------
# graph capture
# ---------------------------------------------------------------------------

def test_graph_replay_is_deterministic():
    w = W.lognormal_weights(300000, seed=7, sigma=2.0)
    wd = to_dev(w)
    u = api.u32_tensor(W.iid_u32(1 << 20, seed=8), DEV)
    f = api.rtf_build(wd, 14)
    idx, pos = api.rtf_sample(f, u)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            api.rtf_build(wd, 14, forest=f)
            api.rtf_sample(f, u, idx_out=idx, pos_out=pos)
    torch.cuda.synchronize()
    outs = []
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        f.check_status()
        outs.append((f.nodes.clone(), idx.clone(), pos.clone()))
    assert all(torch.equal(a, b) for a, b in zip(outs[0], outs[1]))
    ref = orc.build(w, 1 << 14)
    check_structure(f, ref)


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_misaligned_weights(shift):
    """Weights that start 4, 8 or 12 bytes past a 16-byte boundary (the bulk
    copy covers the aligned middle of each tile, plain loads the edges)."""
    n = 3 * 2048 + 77
    w = W.lognormal_weights(n + 8, seed=40 + shift, sigma=2.0)
    full = to_dev(w)
    view = full[shift:shift + n]
    assert view.data_ptr() % 16 == 4 * shift
    f = api.rtf_build(view, 9)
    torch.cuda.synchronize()
    f.check_status()
    check_structure(f, orc.build(w[shift:shift + n], 1 << 9))
    sizes = [5, 2048, 700, n - 2753]
    fb = api.rtf_build_batched(view, sizes, [2, 8, 7, 9])
    torch.cuda.synchronize()
    fb.check_status()
    off = fb.offsets
    for d in range(len(sizes)):
        ref = orc.build(w[shift + off[d]:shift + off[d + 1]], 1 << [2, 8, 7, 9][d])
        check_structure(fb, ref, elem_off=int(off[d]), guide_off=int(fb.guide_offsets[d]))


# ---------------------------------------------------------------------------
# cutpoint method + binary search on the same structure (RTF_SAMPLE_BSEARCH)
# ---------------------------------------------------------------------------

BS = api.SAMPLE_BSEARCH


@pytest.mark.parametrize("m", [0, 3, 10, 11, 14])
def test_bsearch_matches_oracle_all_weight_kinds(m):
    """Shared-memory guide (m <= 10) and global guide (m >= 11) variants."""
    rng = np.random.default_rng(100 + m)
    for n, kind, w in weight_cases():
        f = api.rtf_build(to_dev(w), m)
        u = rng.integers(0, 1 << 32, 4096, dtype=np.uint64).astype(np.uint32)
        u[:3] = [0, 1, 0xFFFFFFFF]
        idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV), mode=api.SAMPLE_1D | BS)
        torch.cuda.synchronize()
        f.check_status()
        ref = orc.build(w, 1 << m)
        ridx, rpos = orc.sample(ref.C, u)
        try:
            check_samples(idx, pos, ridx, rpos)
        except AssertionError as e:
            raise AssertionError(f"n={n} kind={kind} m={m}: {e}")


def test_bsearch_equals_forest_at_full_size(big):
    """Bit-identical bins and positions of the two methods, 2^24 samples of
    each set at n = 2^24."""
    w, f, ref = big
    for u in (W.iid_u32(1 << 24, seed=3), W.sorted_radical_inverse_u32(1 << 28)[::16]):
        ud = api.u32_tensor(u, DEV)
        i1, p1 = api.rtf_sample(f, ud)
        i2, p2 = api.rtf_sample(f, ud, mode=api.SAMPLE_1D | BS)
        assert torch.equal(i1, i2)
        assert torch.equal(p1.view(torch.int32), p2.view(torch.int32))
        assert int(i1.min()) >= 0


def test_bsearch_tagged_and_2d():
    rng = np.random.default_rng(11)
    sizes = np.concatenate([[1, 2, 2049], rng.integers(1, 3000, 100)])
    w = np.concatenate([W.lognormal_weights(int(s), seed=int(i), sigma=1.5)
                        for i, s in enumerate(sizes)])
    ms = np.clip(np.ceil(np.log2(np.maximum(sizes, 1))).astype(int), 0, 12)
    f = api.rtf_build_batched(to_dev(w), sizes, ms)
    dist = rng.integers(0, len(sizes), 1 << 16).astype(np.int32)
    u = rng.integers(0, 1 << 32, dist.size, dtype=np.uint64).astype(np.uint32)
    ud, dd = api.u32_tensor(u, DEV), to_dev(dist)
    i1, p1 = api.rtf_sample(f, ud, dist_id=dd)
    i2, p2 = api.rtf_sample(f, ud, dist_id=dd, mode=api.SAMPLE_1D | BS)
    assert torch.equal(i1, i2) and torch.equal(p1.view(torch.int32), p2.view(torch.int32))
    H, Wd = 48, 80
    lum = W.env_map(H, Wd, seed=12)
    fe = api.rtf_build_batched(to_dev(lum.reshape(-1)), [Wd] * H + [H], [6] * H + [5],
                               marginal=True)
    u2 = rng.integers(0, 1 << 32, 2 * (1 << 15), dtype=np.uint64).astype(np.uint32)
    u2d = api.u32_tensor(u2, DEV)
    j1, q1 = api.rtf_sample(fe, u2d, mode=api.SAMPLE_2D)
    j2, q2 = api.rtf_sample(fe, u2d, mode=api.SAMPLE_2D | BS)
    assert torch.equal(j1, j2) and torch.equal(q1.view(torch.int32), q2.view(torch.int32))
    rows, marg = orc.build_env(lum, 1 << 5, 1 << 6)
    r, c, _, _ = orc.sample_env(rows, marg, u2[0::2], u2[1::2])
    jj = j2.cpu().numpy()
    assert np.array_equal(jj[:, 0], r) and np.array_equal(jj[:, 1], c)


# ---------------------------------------------------------------------------
# load counts per sample (the statistics of Table 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m", [0, 4, 10])
def test_forest_load_counts_equal_oracle_descent(m):
    """Radix forest: one guide record plus the nodes below the root, i.e. the
    oracle's descent from the guide entry (at least 1)."""
    for n, kind, w in weight_cases()[::3]:
        f = api.rtf_build(to_dev(w), m)
        ref = orc.build(w, 1 << m)
        K, _ = orc.keys(ref.C, 1 << m)
        u = W.iid_u32(2048, seed=n)
        loads = api.rtf_sample_loads(f, api.u32_tensor(u, DEV)).cpu().numpy()
        steps = np.array([orc.descend_steps(ref.guide, ref.nodes, K, 1 << m, int(x)) for x in u])
        assert np.array_equal(loads, np.maximum(steps, 1)), f"n={n} kind={kind}"


def test_bsearch_load_counts_bounded():
    """Binary search: guide record(s) plus at most ceil(log2(bracket + 1))
    probes; exactly 1 in a cell that one interval covers."""
    w = W.lognormal_weights(50000, seed=9, sigma=2.0)
    m = 12
    f = api.rtf_build(to_dev(w), m)
    ref = orc.build(w, 1 << m)
    u = W.iid_u32(1 << 14, seed=10)
    loads = api.rtf_sample_loads(f, api.u32_tensor(u, DEV), mode=api.SAMPLE_1D | BS).cpu().numpy()
    g = (u.astype(np.uint64) >> np.uint64(32 - m)).astype(np.int64)
    lo = np.where(ref.guide >= 0, np.maximum(ref.guide - 1, 0), ~ref.guide)
    nxt = np.concatenate([lo[1:], [ref.n - 1]])
    covered = ref.guide < 0
    span = np.where(covered, 0, nxt - lo)[g]
    bound = np.where(covered[g], 1, 2 + np.ceil(np.log2(span + 1)).astype(np.int64))
    assert (loads >= 1).all() and (loads <= bound).all()
    assert (loads[covered[g]] == 1).all()


# ---------------------------------------------------------------------------
# host-streamed sampling (rtf_sample_pipelined)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("coherent", [False, True])
@pytest.mark.parametrize("chunk", [4, 4096, 1 << 20])
def test_pipelined_equals_device_sampling(chunk, coherent):
    """Host samples in, device and host results out, chunked with overlap; a
    count that is not a multiple of the chunk; i.i.d. samples, and sorted
    samples with the coherence hint (the coherent sampler per chunk)."""
    w = W.lognormal_weights(100000, seed=70, sigma=2.0)
    f = api.rtf_build(to_dev(w), 14)
    n_s = 50001 if chunk > 4 else 999
    u = W.iid_u32(n_s, seed=71)
    mode = api.SAMPLE_1D
    if coherent:
        u = np.sort(u)
        mode |= api.SAMPLE_COHERENT
    u_host = torch.from_numpy(u.view(np.int32)).pin_memory()
    u_dev = torch.empty(n_s, dtype=torch.int32, device=DEV)
    idx_dev = torch.empty(n_s, dtype=torch.int32, device=DEV)
    pos_dev = torch.empty(n_s, dtype=torch.float32, device=DEV)
    idx_host = torch.empty(n_s, dtype=torch.int32).pin_memory()
    pos_host = torch.empty(n_s, dtype=torch.float32).pin_memory()
    api.rtf_sample_pipelined(f, u_host, u_dev, idx_dev, pos_dev, idx_host, pos_host, chunk=chunk,
                             mode=mode)
    torch.cuda.synchronize()
    ridx, rpos = orc.sample(orc.build(w, 1 << 14).C, u)
    check_samples(idx_host.numpy(), pos_host.numpy(), ridx, rpos)
    check_samples(idx_dev, pos_dev, ridx, rpos)
    assert np.array_equal(u_dev.cpu().numpy().view(np.uint32), u)


def test_pipelined_tagged_and_2d():
    rng = np.random.default_rng(72)
    sizes = rng.integers(1, 3000, 50)
    w = np.concatenate([W.lognormal_weights(int(s), seed=int(i), sigma=1.5)
                        for i, s in enumerate(sizes)])
    f = api.rtf_build_batched(to_dev(w), sizes, np.full(len(sizes), 9))
    n_s = 1 << 16
    dist = rng.integers(0, len(sizes), n_s).astype(np.int32)
    u = W.iid_u32(n_s, seed=73)
    ref_idx, ref_pos = api.rtf_sample(f, api.u32_tensor(u, DEV), dist_id=to_dev(dist))
    u_dev = torch.empty(n_s, dtype=torch.int32, device=DEV)
    d_dev = torch.empty(n_s, dtype=torch.int32, device=DEV)
    idx_dev = torch.empty(n_s, dtype=torch.int32, device=DEV)
    pos_dev = torch.empty(n_s, dtype=torch.float32, device=DEV)
    idx_host = torch.empty(n_s, dtype=torch.int32).pin_memory()
    pos_host = torch.empty(n_s, dtype=torch.float32).pin_memory()
    api.rtf_sample_pipelined(f, torch.from_numpy(u.view(np.int32)).pin_memory(), u_dev, idx_dev,
                             pos_dev, idx_host, pos_host,
                             dist_id_host=torch.from_numpy(dist).pin_memory(), dist_id_dev=d_dev,
                             chunk=8192)
    torch.cuda.synchronize()
    assert torch.equal(idx_host, ref_idx.cpu()) and torch.equal(pos_host, ref_pos.cpu())
    H, Wd = 40, 64
    lum = W.env_map(H, Wd, seed=74)
    fe = api.rtf_build_batched(to_dev(lum.reshape(-1)), [Wd] * H + [H], [6] * H + [5],
                               marginal=True)
    u2 = W.iid_u32(2 * 30000, seed=75)
    r_idx, r_pos = api.rtf_sample(fe, api.u32_tensor(u2, DEV), mode=api.SAMPLE_2D)
    u2_dev = torch.empty(2 * 30000, dtype=torch.int32, device=DEV)
    i2 = torch.empty((30000, 2), dtype=torch.int32, device=DEV)
    p2 = torch.empty((30000, 2), dtype=torch.float32, device=DEV)
    i2h = torch.empty((30000, 2), dtype=torch.int32).pin_memory()
    p2h = torch.empty((30000, 2), dtype=torch.float32).pin_memory()
    api.rtf_sample_pipelined(fe, torch.from_numpy(u2.view(np.int32)).pin_memory(), u2_dev, i2, p2,
                             i2h, p2h, mode=api.SAMPLE_2D, chunk=4096)
    torch.cuda.synchronize()
    assert torch.equal(i2h, r_idx.cpu()) and torch.equal(p2h, r_pos.cpu())


def test_pipelined_graph_capture():
    """The fork and join onto the copy streams is captured as graph edges;
    replays with new host samples give their results."""
    w = W.lognormal_weights(20000, seed=76, sigma=1.0)
    f = api.rtf_build(to_dev(w), 12)
    ref = orc.build(w, 1 << 12)
    n_s = 1 << 15
    u_host = torch.empty(n_s, dtype=torch.int32).pin_memory()
    u_dev = torch.empty(n_s, dtype=torch.int32, device=DEV)
    idx_dev = torch.empty(n_s, dtype=torch.int32, device=DEV)
    pos_dev = torch.empty(n_s, dtype=torch.float32, device=DEV)
    idx_host = torch.empty(n_s, dtype=torch.int32).pin_memory()
    pos_host = torch.empty(n_s, dtype=torch.float32).pin_memory()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        api.rtf_sample_pipelined(f, u_host, u_dev, idx_dev, pos_dev, idx_host, pos_host,
                                 chunk=8192)
    for seed in (77, 78):
        u = W.iid_u32(n_s, seed=seed)
        u_host.copy_(torch.from_numpy(u.view(np.int32)))
        g.replay()
        torch.cuda.synchronize()
        ridx, rpos = orc.sample(ref.C, u)
        check_samples(idx_host.numpy(), pos_host.numpy(), ridx, rpos)


def test_pipelined_done_event_overlaps_next_call():
    """With done events the stream does not wait for the copies back; after
    waiting for the events both calls' host outputs are complete."""
    w = W.lognormal_weights(30000, seed=80, sigma=2.0)
    f = api.rtf_build(to_dev(w), 13)
    ref = orc.build(w, 1 << 13)
    n_s = 40000
    outs = []
    for seed in (81, 82):
        u = W.iid_u32(n_s, seed=seed)
        bufs = dict(u_host=torch.from_numpy(u.view(np.int32)).pin_memory(),
                    u_dev=torch.empty(n_s, dtype=torch.int32, device=DEV),
                    idx_dev=torch.empty(n_s, dtype=torch.int32, device=DEV),
                    pos_dev=torch.empty(n_s, dtype=torch.float32, device=DEV),
                    idx_host=torch.empty(n_s, dtype=torch.int32).pin_memory(),
                    pos_host=torch.empty(n_s, dtype=torch.float32).pin_memory())
        ev = torch.cuda.Event()
        api.rtf_sample_pipelined(f, chunk=4096, done_event=ev, **bufs)
        outs.append((u, bufs, ev))
    cur = torch.cuda.current_stream()
    for u, bufs, ev in outs:
        cur.wait_event(ev)
    cur.synchronize()
    for u, bufs, ev in outs:
        ridx, rpos = orc.sample(ref.C, u)
        check_samples(bufs["idx_host"].numpy(), bufs["pos_host"].numpy(), ridx, rpos)


def test_coherent_hint_changes_nothing_but_the_grid(big):
    """RTF_SAMPLE_COHERENT only selects the launch shape: identical results on
    scattered and on sorted samples, both methods."""
    w, f, ref = big
    for u in (W.iid_u32(1 << 22, seed=90), W.sorted_radical_inverse_u32(1 << 26)[::16]):
        ud = api.u32_tensor(u, DEV)
        for method in (0, api.SAMPLE_BSEARCH):
            i1, p1 = api.rtf_sample(f, ud, mode=api.SAMPLE_1D | method)
            i2, p2 = api.rtf_sample(f, ud, mode=api.SAMPLE_1D | method | api.SAMPLE_COHERENT)
            assert torch.equal(i1, i2) and torch.equal(p1.view(torch.int32), p2.view(torch.int32))


@pytest.mark.parametrize("m", [0, 4, 14])
def test_coherent_runs_match_oracle_all_weight_kinds(m):
    """The coherent sampler (RTF_SAMPLE_COHERENT): a sample in the previous
    sample's bin, a step forward over zero-width bins, a step backward and a
    jump all give the oracle's bin and position.  Counts leave a ragged tail
    (not a multiple of the 256-sample batch of a warp)."""
    rng = np.random.default_rng(50 + m)
    for n, kind, w in weight_cases():
        f = api.rtf_build(to_dev(w), m)
        ref = orc.build(w, 1 << m)
        base = np.sort(rng.integers(0, 1 << 32, 4096 + 13, dtype=np.uint64)).astype(np.uint32)
        dense = np.sort(rng.integers(0, 1 << 32, 64, dtype=np.uint64)).astype(np.uint32)
        dense = (dense[:, None] + np.arange(0, 4096, 16, dtype=np.uint32)).ravel()  # tight runs
        orders = (base, base[::-1].copy(), np.repeat(base[:1000], 3),
                  np.concatenate([base[:2000], base[100:1700]]), np.sort(dense))
        for u in orders:
            u = u.copy()
            u[:2] = [0, 1]
            u[-1] = 0xFFFFFFFF
            idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV),
                                      mode=api.SAMPLE_1D | api.SAMPLE_COHERENT)
            torch.cuda.synchronize()
            f.check_status()
            ridx, rpos = orc.sample(ref.C, u)
            try:
                check_samples(idx, pos, ridx, rpos)
            except AssertionError as e:
                raise AssertionError(f"n={n} kind={kind} m={m} count={u.size}: {e}")


def test_coherent_runs_tiny_counts():
    """Fewer samples than one run, exactly one run, one run and a tail."""
    w = W.lognormal_weights(5000, seed=8, sigma=2.0)
    f = api.rtf_build(to_dev(w), 10)
    ref = orc.build(w, 1 << 10)
    for count in (1, 3, 15, 16, 17, 31, 33):
        u = np.sort(W.iid_u32(count, seed=count))
        idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV), mode=api.SAMPLE_1D | api.SAMPLE_COHERENT)
        ridx, rpos = orc.sample(ref.C, u)
        check_samples(idx, pos, ridx, rpos)


@pytest.mark.parametrize("kind", ["lognormal2", "zeros", "dups"])
def test_coherent_window_orders_many_batches(kind):
    """The coherent sampler over many batches per warp (its window carried from
    batch to batch): sorted, descending, sorted runs of random lengths, sorted
    with outliers, sorted and so sparse that the window slides far, one value
    repeated.  Every sample equals the per-sample descent's."""
    rng = np.random.default_rng({"lognormal2": 61, "zeros": 62, "dups": 63}[kind])
    n = 1 << 20
    if kind == "lognormal2":
        w = np.exp(rng.normal(0, 2, n))
    elif kind == "zeros":
        w = rng.uniform(0, 1, n) * (rng.random(n) < 0.3)
    else:
        w = np.repeat(rng.uniform(0.01, 1, n // 8), 8) * (rng.random(n) < 0.8)
    f = api.rtf_build(to_dev(w.astype(np.float32)), 16)
    ns = 1 << 23
    base = np.sort(rng.integers(0, 1 << 32, ns, dtype=np.uint64)).astype(np.uint32)
    cuts = np.sort(rng.choice(np.arange(1, ns), 63, replace=False))
    saw = np.concatenate([np.sort(c) for c in np.split(rng.integers(0, 1 << 32, ns, dtype=np.uint64)
                                                       .astype(np.uint32), cuts)])
    outl = base.copy()
    outl[::1000] = rng.integers(0, 1 << 32, outl[::1000].size, dtype=np.uint64).astype(np.uint32)
    sparse = (np.arange(ns, dtype=np.uint64) * 509).astype(np.uint32)  # wraps: sorted pieces
    same = np.full(ns, 0x9E3779B9, np.uint32)
    for name, u in (("sorted", base), ("descending", base[::-1].copy()), ("sawtooth", saw),
                    ("outliers", outl), ("sparse", sparse), ("same", same)):
        ud = api.u32_tensor(u, DEV)
        i1, p1 = api.rtf_sample(f, ud, mode=api.SAMPLE_1D | api.SAMPLE_COHERENT)
        i2, p2 = api.rtf_sample(f, ud)
        torch.cuda.synchronize()
        f.check_status()
        assert torch.equal(i1, i2), f"{kind}/{name}: indices"
        assert torch.equal(p1.view(torch.int32), p2.view(torch.int32)), f"{kind}/{name}: positions"
        assert int(i1.min()) >= 0


# ---------------------------------------------------------------------------
# failure path of the bounded waits (no fault: a flag that nothing sets)
# ---------------------------------------------------------------------------

def test_bounded_wait_gives_up_and_the_context_stays_usable():
    import time
    t0 = time.time()
    st = api.check_bounded_wait(DEV)
    dt = time.time() - t0
    assert st & api.STATUS_TIMEOUT, st
    assert dt < 60, f"the wait took {dt:.1f} s"
    # the same context builds and samples correctly afterwards
    w = W.lognormal_weights(5000, seed=81, sigma=2.0)
    f, ref = build_and_check(w, 9)
    u = W.iid_u32(1 << 14, seed=82)
    idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV))
    ridx, rpos = orc.sample(ref.C, u)
    check_samples(idx, pos, ridx, rpos)


# ---------------------------------------------------------------------------
# sizes past 32-bit indexing, and guide tables much larger than n
# ---------------------------------------------------------------------------

def test_sample_counts_past_2_31():
    """2^31 + 1029 samples in one call (i.i.d. and, ascending, through the
    coherent sampler): the kernels' 64-bit sample indexing and their tails;
    the oracle checks the first and last 1024 samples and 2048 in between."""
    w = W.lognormal_weights(1 << 20, seed=91, sigma=2.0)
    f = api.rtf_build(to_dev(w), 16)
    ref = orc.build(w, 1 << 16)
    ns = (1 << 31) + 1029
    gen = torch.Generator(device=DEV).manual_seed(92)
    sel = np.concatenate([np.arange(1024), ns - 1024 + np.arange(1024),
                          np.random.default_rng(93).integers(1024, ns - 1024, 2048)])
    sel_t = torch.from_numpy(sel).to(DEV)
    for name in ("iid", "ascending"):
        if name == "iid":
            u = torch.randint(-(1 << 31), 1 << 31, (ns,), dtype=torch.int32, device=DEV,
                              generator=gen)
            mode = api.SAMPLE_1D
        else:
            u = torch.arange(ns, dtype=torch.int64, device=DEV).to(torch.int32)  # 0, 1, 2, ...
            mode = api.SAMPLE_1D | api.SAMPLE_COHERENT
        idx, pos = api.rtf_sample(f, u, mode=mode)
        torch.cuda.synchronize()
        f.check_status()
        us = u[sel_t].cpu().numpy().view(np.uint32)
        ridx, rpos = orc.sample(ref.C, us)
        check_samples(idx[sel_t], pos[sel_t], ridx, rpos)
        del u, idx, pos
        torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [1, 777, 40000])
def test_guide_tables_much_larger_than_n(n):
    """2^22 cells over few weights: long runs of cells without keys take the
    interval of the last key before them (the carry-forward over many tiles)."""
    w = W.lognormal_weights(n, seed=94 + n, sigma=3.0)
    f, ref = build_and_check(w, 22)
    u = W.iid_u32(1 << 16, seed=95)
    idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV))
    ridx, rpos = orc.sample(ref.C, u)
    check_samples(idx, pos, ridx, rpos)


def test_maximum_guide_bits():
    """m = 30, the largest table the interface accepts (2^30 cells of 4 u-units:
    36 GB of guide entries and records) over 40000 lognormal(0, 3) weights:
    samples through the whole path against the oracle's inverse CDF, and
    sampled guide entries against their definition: negative exactly when one
    interval covers the cell (the same bin at its first and last u), and then
    that interval."""
    n, m = 40000, 30
    w = W.lognormal_weights(n, seed=98, sigma=3.0)
    f = api.rtf_build(to_dev(w), m)
    torch.cuda.synchronize()
    f.check_status()
    C = orc.cdf(orc.quantize(w, orc.scale(w)))
    u = W.iid_u32(1 << 18, seed=99)
    u[:2] = [0, 0xFFFFFFFF]
    idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV))
    ridx, rpos = orc.sample(C, u)
    check_samples(idx, pos, ridx, rpos)
    rng = np.random.default_rng(100)
    cells = np.concatenate([np.arange(64), (1 << m) - 64 + np.arange(64),
                            rng.integers(0, 1 << m, 1 << 16)]).astype(np.int64)
    got = f.guide[torch.from_numpy(cells).to(DEV)].cpu().numpy()
    first, _ = orc.sample(C, (cells << (32 - m)).astype(np.uint32))
    last, _ = orc.sample(C, ((cells << (32 - m)) + (1 << (32 - m)) - 1).astype(np.uint32))
    covered = first == last
    assert np.array_equal(got < 0, covered)
    assert np.array_equal(~got[covered], first[covered])
    del f
    torch.cuda.empty_cache()


def test_build_past_4gb_of_records():
    """n = 2^29 + 3 weights, 2^24 cells (8 GB of node records, 512 MB of
    guide records): the CDF at sampled elements, T, and 2^16 sampled indices
    and positions against the oracle's exact CDF."""
    n = (1 << 29) + 3
    rng = np.random.default_rng(96)
    w = np.exp(rng.standard_normal(n, dtype=np.float32) * np.float32(2.0)).astype(np.float32)
    f = api.rtf_build(to_dev(w), 24)
    torch.cuda.synchronize()
    f.check_status()
    C = orc.cdf(orc.quantize(w, orc.scale(w)))
    sel = np.concatenate([np.arange(2048), n - 2048 + np.arange(2048),
                          rng.integers(2048, n - 2048, 4096)])
    got = f.cdf()[torch.from_numpy(sel).to(DEV)].cpu().numpy().view(np.uint64)
    assert np.array_equal(got, C[sel]), "CDF"
    assert int(f.dist_table()[0, 3].item()) & ((1 << 64) - 1) == int(C[-1]), "T"
    u = W.iid_u32(1 << 16, seed=97)
    u[:2] = [0, 0xFFFFFFFF]
    idx, pos = api.rtf_sample(f, api.u32_tensor(u, DEV))
    ridx, rpos = orc.sample(C, u)
    check_samples(idx, pos, ridx, rpos)
    del f
    torch.cuda.empty_cache()
