"""The allocation-free build (rtf_build_static) against rtf_build.

rtf_build_static serves callers that cannot allocate device memory: it keeps
its scratch in a fixed array inside the library.  Called twice in a row
through the C interface, on different weights of the same size, it must give
the same forest, guide table and samples as rtf_build with a caller
workspace; sizes beyond its limit are refused.
This file is collected last so that a failure here leaves every other test
already run.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_1901_05423_gb300 import _native, api
from paper_1901_05423_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
EWORKSPACE = 2


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def static_build(lib, w, n, m, stream):
    f = api.Forest(1, 0, n, 1 << m, m, DEV)
    cf = f.c_struct()
    rc = lib.rtf_build_static(ctypes.c_void_p(w.data_ptr()), n, m, ctypes.byref(cf), stream)
    assert rc == 0
    return f


def test_static_build_matches_workspace_build_twice_in_a_row():
    """Per size, two calls in a row on different weights of the same n and m
    (so that flags or prefixes left in the shared array by the first call
    would show in the second), each against rtf_build with a workspace."""
    lib = _native.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    cases = [(1 << 20, 16, 0, 2.0), (3 * 2048 + 5, 9, 1, 1.0)]
    for n, m, seed, sigma in cases:
        for k, (sd, sg) in enumerate(((seed, sigma), (seed + 100, 1.5 * sigma))):
            w = torch.from_numpy(W.lognormal_weights(n, seed=sd, sigma=sg)).to(DEV)
            ref = api.rtf_build(w, m)
            f = static_build(lib, w, n, m, stream)
            torch.cuda.synchronize()
            ref.check_status()
            f.check_status()
            assert torch.equal(f.nodes, ref.nodes), (n, k)
            assert torch.equal(f.guide, ref.guide), (n, k)
            assert torch.equal(f.guide_recs, ref.guide_recs), (n, k)
            assert torch.equal(f.dists, ref.dists), (n, k)
            u = api.u32_tensor(W.iid_u32(1 << 18, seed=sd + 7), DEV)
            i0, p0 = api.rtf_sample(ref, u)
            i1, p1 = api.rtf_sample(f, u)
            assert torch.equal(i0, i1)
            assert torch.equal(p0, p1)


def test_static_build_refuses_sizes_beyond_its_array():
    lib = _native.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    n = (1 << 20) + 1
    w = torch.ones(n, dtype=torch.float32, device=DEV)
    f = api.Forest(1, 0, n, 1 << 10, 10, DEV)
    cf = f.c_struct()
    assert lib.rtf_build_static(ctypes.c_void_p(w.data_ptr()), n, 10, ctypes.byref(cf),
                                stream) == EWORKSPACE
    f2 = api.Forest(1, 0, 1000, 1 << 17, 17, DEV)
    cf2 = f2.c_struct()
    assert lib.rtf_build_static(ctypes.c_void_p(w.data_ptr()), 1000, 17, ctypes.byref(cf2),
                                stream) == EWORKSPACE
