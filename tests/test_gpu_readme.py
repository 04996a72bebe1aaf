"""The usage example of README.md runs as written and gives valid results."""

import os
import re

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_readme_example_runs():
    with open(os.path.join(ROOT, "README.md")) as f:
        text = f.read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert len(blocks) == 1
    ns = {}
    exec(compile(blocks[0], "README.md", "exec"), ns)
    torch.cuda.synchronize()
    idx, pos, w = ns["idx"], ns["pos"], ns["w"]
    assert idx.shape == pos.shape == ns["u"].shape
    assert int(idx.min()) >= 0 and int(idx.max()) < w.numel()
    assert float(pos.min()) >= 0.0 and float(pos.max()) < 1.0
    assert torch.isfinite(ns["grad_w"]).all() and torch.isfinite(ns["wg"].grad).all()
    sizes, dist, idx_b = ns["sizes"], ns["dist"], ns["idx_b"]
    lim = torch.tensor(sizes, device=idx_b.device)[dist.long()]
    assert bool(((idx_b >= 0) & (idx_b < lim)).all())
    rc, xy = ns["rc"], ns["xy"]
    assert rc.shape == xy.shape == (4096, 2)
    assert bool(((rc[:, 0] >= 0) & (rc[:, 0] < ns["H"]) & (rc[:, 1] >= 0) & (rc[:, 1] < ns["W"])).all())
    assert bool(((xy >= 0) & (xy < 1)).all())
    for f in (ns["forest"], ns["fb"], ns["fm"]):
        f.check_status()
