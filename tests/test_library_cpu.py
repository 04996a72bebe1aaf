"""CPU-side checks of the C interface: the library builds for sm_103a, loads,
exports every function include/rtf.h declares, mirrors its structs, and rejects
bad arguments before any GPU work.  No compute call is made here."""

import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "rtf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rtf_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1901_05423_gb300 import _native
    return _native.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rtf_build", "rtf_build_batched", "rtf_sample", "rtf_sample_backward"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1901_05423_gb300 import _native
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _native.EXPORTS, f"binding lacks {name}"
    assert lib.rtf_version().startswith(b"rtf")


def test_struct_layout_matches_header():
    from paper_1901_05423_gb300 import _native
    assert ctypes.sizeof(_native.RtfForestC) == 72
    # rtf_quad_rec: three u64 splits and four int16 references, 32 bytes
    text_q = open(HEADER).read()
    assert "uint64_t cdf[3];" in text_q and "int16_t ref[4];" in text_q
    # rtf_node is 16 bytes (u64 + 2 x i32) and rtf_dist 64 bytes
    text = open(HEADER).read()
    assert "uint64_t cdf;" in text and "int32_t child[2];" in text


def test_workspace_sizes(lib):
    a = lib.rtf_build_workspace_size(1 << 24, 1, 1 << 20)
    b = lib.rtf_build_workspace_size(1 << 10, 1, 1 << 8)
    assert a > b > 0
    assert a % 256 == 0
    # the distance byte per element dominates; the list of long runs of empty
    # guide cells takes 16 B per 17 cells
    n, G = 1 << 24, 1 << 20
    assert n + G // 2 <= a <= n + G + n // 4
    assert lib.rtf_build_workspace_size(0, 1, 1) == 0
    # two fp32 sums per bin
    assert lib.rtf_backward_workspace_size(1 << 20, 1) >= 8 * (1 << 20)


def test_bad_arguments_rejected_without_gpu_work(lib):
    from paper_1901_05423_gb300 import _native
    EINVAL = 1
    f = _native.RtfForestC()
    assert lib.rtf_build(None, 10, 4, ctypes.byref(f), None, 0, None) == EINVAL
    f = _native.RtfForestC(num_dists=1, flags=0, num_elems=10, num_cells=16, max_m=4,
                           nodes=16, guide=16, dists=64, status=4, guide_recs=32)
    # misaligned weights / bad m / inconsistent sizes never reach the GPU
    assert lib.rtf_build(ctypes.c_void_p(2), 10, 4, ctypes.byref(f), ctypes.c_void_p(256),
                         1 << 20, None) == EINVAL
    assert lib.rtf_build(ctypes.c_void_p(16), 10, 31, ctypes.byref(f), ctypes.c_void_p(256),
                         1 << 20, None) == EINVAL
    assert lib.rtf_build(ctypes.c_void_p(16), 11, 4, ctypes.byref(f), ctypes.c_void_p(256),
                         1 << 20, None) == EINVAL
    assert lib.rtf_build(ctypes.c_void_p(16), 10, 4, ctypes.byref(f), ctypes.c_void_p(256),
                         16, None) == 2  # workspace too small
    assert lib.rtf_sample(ctypes.byref(f), ctypes.c_void_p(16), None, -1, 0, ctypes.c_void_p(16),
                          ctypes.c_void_p(16), None) == EINVAL
    assert lib.rtf_sample(ctypes.byref(f), ctypes.c_void_p(16), None, 5, 1, ctypes.c_void_p(16),
                          ctypes.c_void_p(16), None) == EINVAL  # 2-D needs a marginal
    for mode in (2, 0x400, 0x101, 0x301, 0x80):  # unknown mode or flag; 2-D + bsearch needs a marginal
        assert lib.rtf_sample(ctypes.byref(f), ctypes.c_void_p(16), None, 5, mode,
                              ctypes.c_void_p(16), ctypes.c_void_p(16), None) == EINVAL
    assert lib.rtf_sample(ctypes.byref(f), ctypes.c_void_p(16), None, 0, 0, None, None,
                          None) == 0  # nothing to do
    P0 = ctypes.c_void_p
    assert lib.rtf_backward_begin(ctypes.byref(f), P0(8), 1 << 30, None) == EINVAL  # ws alignment
    assert lib.rtf_backward_begin(ctypes.byref(f), P0(256), 16, None) == 2  # workspace too small
    assert lib.rtf_backward_accumulate(ctypes.byref(f), None, None, None, None, 5, 0, P0(256),
                                       1 << 30, None) == EINVAL  # count > 0 needs inputs
    assert lib.rtf_backward_accumulate(ctypes.byref(f), None, P0(16), P0(16), P0(16), 5, 1,
                                       P0(256), 1 << 30, None) == EINVAL  # 2-D needs a marginal
    assert lib.rtf_backward_finish(ctypes.byref(f), None, 0, P0(16), P0(256), 1 << 30,
                                   None) == EINVAL  # weights needed
    assert lib.rtf_build_quad(ctypes.byref(f), P0(16), None) == EINVAL  # records 32-byte aligned
    assert lib.rtf_build_quad(ctypes.byref(f), None, None) == EINVAL
    for mode in (0x100, 0x101, 2, 0x400):  # no binary search through 4-ary records; unknown flags
        assert lib.rtf_sample_quad(ctypes.byref(f), P0(32), P0(16), None, 8, mode, P0(16), P0(16),
                                   None, None) == EINVAL
    assert lib.rtf_sample_quad(ctypes.byref(f), P0(32), P0(16), None, 8, 0, P0(16), P0(16),
                               P0(4), None) == EINVAL  # load counts 8-byte aligned
    assert lib.rtf_sample_quad(ctypes.byref(f), P0(32), None, None, 8, 0, P0(16), P0(16),
                               None, None) == EINVAL  # samples needed
    assert lib.rtf_sample_quad(ctypes.byref(f), P0(32), None, None, 0, 0, None, None,
                               None, None) == 0  # nothing to do
    assert lib.rtf_check_bounded_wait(None, P0(16), None) == EINVAL
    assert lib.rtf_check_bounded_wait(P0(16), P0(12), None) == EINVAL  # scratch 8-byte aligned
    P = ctypes.c_void_p
    for chunk in (0, 3, 6):  # chunks are positive multiples of 4
        assert lib.rtf_sample_pipelined(ctypes.byref(f), None, P(16), None, None, 8, 0, P(16),
                                        P(16), None, None, chunk, None, None) == EINVAL
    assert lib.rtf_sample_pipelined(ctypes.byref(f), None, P(16), P(16), None, 8, 0, P(16),
                                    P(16), None, None, 4, None, None) == EINVAL  # ids need a device buffer
    assert lib.rtf_sample_pipelined(ctypes.byref(f), None, P(8), None, None, 8, 0, P(16),
                                    P(16), None, None, 4, None, None) == EINVAL  # misaligned
    assert lib.rtf_sample_pipelined(ctypes.byref(f), None, None, None, None, 0, 0, None,
                                    None, None, None, 4, None, None) == 0  # nothing to do


def test_plan_batched_host_logic():
    from paper_1901_05423_gb300 import api
    off, goff, m = api.plan_batched([3, 1, 5], [2, 0, 4])
    assert off.tolist() == [0, 3, 4, 9]
    assert goff.tolist() == [0, 4, 5, 21]
    with pytest.raises(api.RtfError):
        api.plan_batched([0, 2], [1, 1])
    with pytest.raises(api.RtfError):
        api.plan_batched([4, 4, 3], [1, 1, 1], marginal=True)  # marginal needs 2 weights
    off, goff, m = api.plan_batched([4, 4, 2], [1, 1, 1], marginal=True)
    assert off[-1] == 10


def test_workload_generators_shapes():
    from paper_1901_05423_gb300 import workloads as W
    u = W.radical_inverse_u32(1 << 12)
    assert u.dtype == np.uint32 and len(set(u.tolist())) == 1 << 12
    assert np.array_equal(np.sort(u), W.sorted_radical_inverse_u32(1 << 12))
    w, off = W.ragged_batch(64, seed=0)
    sizes = np.diff(off)
    assert sizes.min() >= 8 and sizes.max() <= 65536 and w.size == off[-1]
    lum = W.env_map(32, 64, seed=0)
    assert lum.shape == (32, 64) and lum.dtype == np.float32 and lum.min() > 0


def test_guide_bits_lookup_without_gpu():
    from paper_1901_05423_gb300 import autotune
    table = {3: 2, 4: 4, 5: 5, 6: 7}
    ms = autotune.guide_bits_for([1, 8, 11, 16, 40, 64, 10 ** 6], table)
    assert ms.tolist() == [2, 2, 2, 4, 5, 7, 7]


def test_load_statistics_columns():
    from paper_1901_05423_gb300.api import load_statistics
    a = np.ones(64, np.int32)
    a[5] = 7
    a[40] = 3
    st = load_statistics(a)
    assert st["maximum"] == 7
    assert abs(st["average"] - (62 + 7 + 3) / 64) < 1e-12
    assert st["average32"] == (7 + 3) / 2
    with pytest.raises(ValueError):
        load_statistics(np.array([1, -1]))


def test_launch_shape_host_logic(lib):
    """rtf_set_launch_shape / rtf_get_launch_shape: values in [0, 64], 0 for the
    built-in choice, NULL restores all; no GPU work."""
    from paper_1901_05423_gb300 import _native
    EINVAL = 1
    s = _native.RtfLaunchShapeC()
    try:
        assert lib.rtf_set_launch_shape(None) == 0
        assert lib.rtf_get_launch_shape(ctypes.byref(s)) == 0
        builtin = (s.single_large, s.single, s.tagged, s.pairs)
        assert builtin == (3, 8, 8, 8)
        assert lib.rtf_set_launch_shape(ctypes.byref(_native.RtfLaunchShapeC(5, 0, 12, 0))) == 0
        lib.rtf_get_launch_shape(ctypes.byref(s))
        assert (s.single_large, s.single, s.tagged, s.pairs) == (5, 8, 12, 8)
        for bad in ((65, 0, 0, 0), (0, -1, 0, 0), (0, 0, 0, 1000)):
            assert lib.rtf_set_launch_shape(ctypes.byref(_native.RtfLaunchShapeC(*bad))) == EINVAL
        lib.rtf_get_launch_shape(ctypes.byref(s))
        assert (s.single_large, s.tagged) == (5, 12)  # a rejected call changes nothing
        assert lib.rtf_get_launch_shape(None) == EINVAL
    finally:
        lib.rtf_set_launch_shape(None)
    lib.rtf_get_launch_shape(ctypes.byref(s))
    assert (s.single_large, s.single, s.tagged, s.pairs) == builtin
