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
