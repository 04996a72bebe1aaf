"""4-ary records (two binary levels collapsed, the section on k-ary trees):
the records against the oracle's collapse, and sampling through them against
the oracle and bit for bit against the binary sampler.  Load counts equal one
guide record plus the oracle's number of 4-ary records."""

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1901_05423_gb300 import api
from paper_1901_05423_gb300 import workloads as W
from test_gpu_parity import DEV, check_samples, to_dev, weight_cases

pytestmark = pytest.mark.gpu

TWO32 = 1 << 32


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def decode(quad, n):
    """GPU records -> (splits uint64 [n, 3], far bool [n], refs int64 [n, 4] as
    node ids >= 0 or ~bin)."""
    q = quad.cpu().numpy()
    cdf = q[:, :3].view(np.uint64).copy()
    far = (cdf[:, 1] >> np.uint64(63)) == 1
    cdf[:, 1] &= np.uint64((1 << 63) - 1)
    codes = q[:, 3].copy().view(np.int16).reshape(n, 4).astype(np.int64)
    j = np.arange(n, dtype=np.int64)[:, None]
    k = j + (codes >> 1)
    refs = np.where(codes & 1, ~k, k)
    return cdf, far, refs


def check_records(f, quad, ref):
    n = ref.n
    cdf, far, refs = decode(quad, n)
    split, child = orc.quad(ref.nodes)
    assert np.array_equal(cdf, ref.C[split]), "4-ary record splits"
    near = ~far
    bad = np.nonzero((refs[near] != child[near]).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} 4-ary records differ, first {np.nonzero(near)[0][bad[:5]]}"
    # a record is far exactly when one of its references is more than 2^14 away
    tgt = np.where(child < 0, ~child, child).astype(np.int64)
    dist = tgt - np.arange(n, dtype=np.int64)[:, None]
    too_far = ((dist < -16384) | (dist > 16383)).any(axis=1)
    assert np.array_equal(far, too_far), "far flags"
    return far


@pytest.mark.parametrize("m", [0, 4, 9, 14])
def test_quad_records_and_samples_all_weight_kinds(m):
    rng = np.random.default_rng(300 + m)
    for n, kind, w in weight_cases():
        f = api.rtf_build(to_dev(w), m)
        quad = api.rtf_build_quad(f)
        u = rng.integers(0, TWO32, 4096 + 3, dtype=np.uint64).astype(np.uint32)
        u[:3] = [0, 1, 0xFFFFFFFF]
        ud = api.u32_tensor(u, DEV)
        loads = torch.empty(u.size, dtype=torch.int32, device=DEV)
        idx, pos = api.rtf_sample_quad(f, quad, ud, loads_out=loads)
        i2, p2 = api.rtf_sample(f, ud)
        torch.cuda.synchronize()
        f.check_status()
        ref = orc.build(w, 1 << m)
        try:
            far = check_records(f, quad, ref)
            ridx, rpos = orc.sample(ref.C, u)
            check_samples(idx, pos, ridx, rpos)
            assert torch.equal(idx, i2) and torch.equal(pos.view(torch.int32), p2.view(torch.int32))
            if not far.any():
                K, _ = orc.keys(ref.C, 1 << m)
                split, child = orc.quad(ref.nodes)
                lg = loads.cpu().numpy()
                for s in range(0, u.size, 97):
                    _, r = orc.descend_quad(ref.guide, ref.nodes, split, child, K, 1 << m, int(u[s]))
                    assert lg[s] == 1 + r, (s, lg[s], r)
        except AssertionError as e:
            raise AssertionError(f"n={n} kind={kind} m={m}: {e}")


def test_quad_far_records_single_cell():
    """One cell over 40000 bins: references more than 2^14 away are far, and
    the descent takes binary steps through them."""
    w = W.lognormal_weights(40000, seed=31, sigma=2.0)
    f = api.rtf_build(to_dev(w), 0)
    quad = api.rtf_build_quad(f)
    torch.cuda.synchronize()
    ref = orc.build(w, 1)
    far = check_records(f, quad, ref)
    assert far.any() and not far.all()
    u = np.concatenate([W.iid_u32(1 << 16, seed=32), np.sort(W.iid_u32(4099, seed=33))])
    ud = api.u32_tensor(u, DEV)
    idx, pos = api.rtf_sample_quad(f, quad, ud)
    ridx, rpos = orc.sample(ref.C, u)
    check_samples(idx, pos, ridx, rpos)


def test_quad_tagged_and_2d():
    wb, offb = W.ragged_batch(300, seed=34)
    sizes = np.diff(offb)
    ms = np.clip(np.round(np.log2(sizes)).astype(int) - 2, 0, 16)
    f = api.rtf_build_batched(to_dev(wb), sizes, ms)
    quad = api.rtf_build_quad(f)
    u = W.iid_u32(1 << 18, seed=35)
    d = np.random.default_rng(36).integers(0, sizes.size, u.size).astype(np.int32)
    ud, dd = api.u32_tensor(u, DEV), to_dev(d)
    loads = torch.empty(u.size, dtype=torch.int32, device=DEV)
    idx, pos = api.rtf_sample_quad(f, quad, ud, dist_id=dd, loads_out=loads)
    i2, p2 = api.rtf_sample(f, ud, dist_id=dd)
    torch.cuda.synchronize()
    f.check_status()
    assert torch.equal(idx, i2) and torch.equal(pos.view(torch.int32), p2.view(torch.int32))
    assert int(loads.min()) >= 1
    # records of every distribution against the oracle
    qn = quad.cpu()
    for dist in range(0, sizes.size, 37):
        lo, hi = int(offb[dist]), int(offb[dist + 1])
        ref = orc.build(wb[lo:hi], 1 << int(ms[dist]))
        check_records(None, qn[lo:hi], ref)

    lum = W.env_map(96, 160, seed=37)
    f2 = api.rtf_build_batched(to_dev(lum.reshape(-1)), [160] * 96 + [96], [6] * 96 + [5],
                               marginal=True)
    quad2 = api.rtf_build_quad(f2)
    u2 = W.iid_u32(2 * (1 << 16), seed=38)
    u2d = api.u32_tensor(u2, DEV)
    idx, pos = api.rtf_sample_quad(f2, quad2, u2d, mode=api.SAMPLE_2D)
    i2, p2 = api.rtf_sample(f2, u2d, mode=api.SAMPLE_2D)
    torch.cuda.synchronize()
    f2.check_status()
    assert torch.equal(idx, i2) and torch.equal(pos.view(torch.int32), p2.view(torch.int32))


def test_quad_full_size_equals_binary():
    """n = 2^24 lognormal(0, 2), 2^20 cells: records, then 2^24 i.i.d. and 2^24
    sorted samples identical to the binary sampler's."""
    w = W.lognormal_weights(1 << 24, seed=0, sigma=2.0)
    f = api.rtf_build(to_dev(w), 20)
    quad = api.rtf_build_quad(f)
    torch.cuda.synchronize()
    f.check_status()
    ref = orc.build(w, 1 << 20)
    far = check_records(f, quad, ref)
    assert not far.any()
    for u, mode in ((W.iid_u32(1 << 24, seed=39), api.SAMPLE_1D),
                    (W.sorted_radical_inverse_u32(1 << 28)[::16], api.SAMPLE_1D | api.SAMPLE_COHERENT)):
        ud = api.u32_tensor(u, DEV)
        idx, pos = api.rtf_sample_quad(f, quad, ud, mode=mode)
        i2, p2 = api.rtf_sample(f, ud)
        assert torch.equal(idx, i2) and torch.equal(pos.view(torch.int32), p2.view(torch.int32))


def test_quad_coherent_hint_and_2d_load_counts():
    """The coherence hint only widens the 4-ary sampler's grid (same bits);
    in 2-D the load counts come as (row, column) pairs, each at least the
    guide record, and equal the 1-D counts of the marginal and of each row."""
    w = W.lognormal_weights(300000, seed=41, sigma=2.0)
    f = api.rtf_build(to_dev(w), 16)
    quad = api.rtf_build_quad(f)
    u = np.sort(W.iid_u32(1 << 20, seed=42))
    ud = api.u32_tensor(u, DEV)
    i1, p1 = api.rtf_sample_quad(f, quad, ud)
    i2, p2 = api.rtf_sample_quad(f, quad, ud, mode=api.SAMPLE_1D | api.SAMPLE_COHERENT)
    assert torch.equal(i1, i2) and torch.equal(p1.view(torch.int32), p2.view(torch.int32))

    H, Wd = 64, 96
    lum = W.env_map(H, Wd, seed=43)
    f2 = api.rtf_build_batched(to_dev(lum.reshape(-1)), [Wd] * H + [H], [5] * H + [4], marginal=True)
    q2 = api.rtf_build_quad(f2)
    ns = 4099
    uu = W.iid_u32(2 * ns, seed=44)
    loads = torch.empty((ns, 2), dtype=torch.int32, device=DEV)
    idx, pos = api.rtf_sample_quad(f2, q2, api.u32_tensor(uu, DEV), mode=api.SAMPLE_2D,
                                   loads_out=loads)
    torch.cuda.synchronize()
    f2.check_status()
    i_ref, p_ref = api.rtf_sample(f2, api.u32_tensor(uu, DEV), mode=api.SAMPLE_2D)
    assert torch.equal(idx, i_ref) and torch.equal(pos.view(torch.int32), p_ref.view(torch.int32))
    lg = loads.cpu().numpy()
    assert (lg >= 1).all()
    # the row counts equal those of a 1-D descent through the marginal alone
    rows = np.full(ns, H, np.int32)  # the marginal is the last distribution
    lrow = torch.empty(ns, dtype=torch.int32, device=DEV)
    api.rtf_sample_quad(f2, q2, api.u32_tensor(uu[0::2].copy(), DEV), dist_id=to_dev(rows),
                        loads_out=lrow)
    assert np.array_equal(lrow.cpu().numpy(), lg[:, 0])
