"""The guide-size autotuner: a small tuning run yields guide bits near
log2(n) for every bucket, and the per-distribution lookup is consistent."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_small_tuning_run(tmp_path, monkeypatch):
    from paper_1901_05423_gb300 import autotune
    monkeypatch.setenv("RTF_CACHE_DIR", str(tmp_path))
    table = autotune.tune("cuda:0", buckets=range(3, 9), total=1 << 16, reps=1)
    assert sorted(table) == list(range(3, 9))
    for b, m in table.items():
        assert b - 2 <= m <= b + 2
    again = autotune.tune("cuda:0", buckets=range(3, 9), total=1 << 16, reps=1)
    assert again == table  # served from the cache file
    ms = autotune.guide_bits_for(np.array([8, 9, 100, 256, 10 ** 6]), table)
    assert ms.dtype == np.int32 and ms[0] == table[3] and ms[-1] == table[8]


def test_launch_shape_changes_no_result_and_is_tuned(tmp_path, monkeypatch):
    """Every launch shape gives the same bits (tagged samples over a ragged
    batch, and scattered samples over one structure larger than L2); the
    launch-shape autotuner picks one of its candidates, sets it and caches it."""
    from paper_1901_05423_gb300 import api, autotune
    from paper_1901_05423_gb300 import workloads as W
    monkeypatch.setenv("RTF_CACHE_DIR", str(tmp_path))
    dev = torch.device("cuda:0")
    try:
        w_h, off = W.ragged_batch(512, seed=5)
        sizes = np.diff(off)
        f = api.rtf_build_batched(torch.from_numpy(w_h).to(dev), sizes,
                                  np.clip(np.round(np.log2(sizes)).astype(int), 3, 16))
        u = api.u32_tensor(W.iid_u32(1 << 20, seed=6), dev)
        d = torch.from_numpy(W.dist_ids(1 << 20, len(sizes), seed=7)).to(dev)
        i0, p0 = api.rtf_sample(f, u, dist_id=d)
        for c in (1, 2, 5, 16):
            api.set_launch_shape(tagged=c)
            i1, p1 = api.rtf_sample(f, u, dist_id=d)
            assert torch.equal(i0, i1) and torch.equal(p0.view(torch.int32), p1.view(torch.int32))
        kind, best, times = autotune.tune_launch_shape(f, u, d, candidates=(2, 8), reps=1,
                                                       key="ragged512")
        assert kind == "tagged" and best in (2, 8) and sorted(times) == [2, 8]
        assert api.get_launch_shape()["tagged"] == best
        api.reset_launch_shape()
        kind2, best2, times2 = autotune.tune_launch_shape(f, u, d, candidates=(2, 8), reps=1,
                                                         key="ragged512")
        assert (kind2, best2, times2) == ("tagged", best, {})  # from the cache
        assert api.get_launch_shape()["tagged"] == best

        wb = W.lognormal_weights(1 << 23, seed=8, sigma=2.0)  # 128 MB of node records
        fb = api.rtf_build(torch.from_numpy(wb).to(dev), 20)
        ub = api.u32_tensor(W.iid_u32(1 << 22, seed=9), dev)
        i0, p0 = api.rtf_sample(fb, ub)
        for c in (1, 3, 8):
            api.set_launch_shape(single_large=c)
            i1, p1 = api.rtf_sample(fb, ub)
            assert torch.equal(i0, i1) and torch.equal(p0.view(torch.int32), p1.view(torch.int32))
        kind, best, _ = autotune.tune_launch_shape(fb, ub, candidates=(3, 8), reps=1)
        assert kind == "single_large" and api.get_launch_shape()["single_large"] == best
        fb.check_status()
        f.check_status()
    finally:
        api.reset_launch_shape()


def test_env_guide_bits_tuner(tmp_path, monkeypatch):
    """The 2-D map tuner times its candidates around (log2 cols, log2 rows),
    returns the fastest and caches it; the map built with its choice equals
    the oracle's structure (rows and marginal)."""
    from oracle import oracle as orc
    from paper_1901_05423_gb300 import api, autotune
    from paper_1901_05423_gb300 import workloads as W
    monkeypatch.setenv("RTF_CACHE_DIR", str(tmp_path))
    dev = torch.device("cuda:0")
    H, Wd = 64, 256
    lum_h = W.env_map(H, Wd, seed=7)
    lum = torch.from_numpy(lum_h.reshape(-1)).to(dev)
    mr, mm, times = autotune.tune_env_bits(lum, H, Wd, 1 << 20, probe_pairs=1 << 16, reps=1)
    assert (mr, mm) == min(times, key=times.get)
    assert all(6 <= a <= 10 and 5 <= b <= 7 for a, b in times)
    assert autotune.tune_env_bits(lum, H, Wd, 1 << 20)[:2] == (mr, mm)  # cached
    f = api.rtf_build_batched(lum, [Wd] * H + [H], [mr] * H + [mm], marginal=True)
    torch.cuda.synchronize()
    f.check_status()
    rows, marg = orc.build_env(lum_h, 1 << mm, 1 << mr)  # marginal's cells first
    ch = f.children().cpu().numpy()
    C = f.cdf().cpu().numpy().view(np.uint64)
    g = f.guide.cpu().numpy()
    for r in (0, H // 2, H - 1):
        assert np.array_equal(C[r * Wd:(r + 1) * Wd], rows[r].C[:-1])
        assert np.array_equal(ch[r * Wd:(r + 1) * Wd], rows[r].nodes)
        assert np.array_equal(g[r << mr:(r + 1) << mr], rows[r].guide)
    assert np.array_equal(ch[H * Wd:], marg.nodes)
    assert np.array_equal(g[H << mr:], marg.guide)
