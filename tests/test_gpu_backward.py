"""Gradient of the in-bin positions on the GPU against the oracle's fp64
chain-rule gradient and against central differences of the GPU forward itself.

Both sides differentiate the forward that is computed, x = (xi T - C_i) / q_i,
with the floor of the quantisation passed straight through: the relaxation at
the quantised weights w' = floor(w 2^S) 2^-S.

Tolerance, element by element: |g - g_ref| <= 1e-4 (|g_ref| + 1e-3 max|g_ref|).
The 1e-4 is the relative gradient error the path is held to; the absolute
floor 1e-7 max|g_ref| covers the float32 rounding of the partial sums that
enter one element (the per-bin sums, the tile's suffix sums and the final
G - S_k - X_k / w'_k are float32; each rounding is 2^-24 of a sum no larger
than the largest element in these workloads).  The relative error in the
2-norm is checked against 1e-4 as well."""

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1901_05423_gb300 import api
from paper_1901_05423_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def check_grad(gw, gref, rel=TOL, floor=1e-3):
    """Element-wise mixed bound and the 2-norm bound; returns the worst ratio
    of an element's error to its bound."""
    gw = np.asarray(gw, np.float64).reshape(-1)
    gref = np.asarray(gref, np.float64).reshape(-1)
    assert np.isfinite(gw).all()
    err = np.abs(gw - gref)
    bound = rel * (np.abs(gref) + floor * np.abs(gref).max())
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, (f"{bad.size} of {gref.size} gradient elements off; worst "
                           f"{(err / bound).max():.3g} x the bound, first at {bad[:5]}")
    assert rel_err(gw, gref) <= rel
    return float((err / bound).max())


def run_1d(n, n_s, m, seed, sigma=1.0):
    w = W.lognormal_weights(n, seed=seed, sigma=sigma)
    u = W.iid_u32(n_s, seed=seed + 1)
    g = W.normal_f32(n_s, seed=seed + 2)
    wd = to_dev(w)
    f = api.rtf_build(wd, m)
    ud = api.u32_tensor(u, DEV)
    idx, pos = api.rtf_sample(f, ud)
    gw = api.rtf_sample_backward(f, wd, ud, None, idx, pos, to_dev(g))
    torch.cuda.synchronize()
    f.check_status()
    ref = orc.build(w, 1 << m)
    ridx, _ = orc.sample(ref.C, u)
    assert np.array_equal(idx.cpu().numpy(), ridx)
    gref = orc.grad(w, u, ridx, g)
    return gw.cpu().numpy(), gref


def test_backward_small():
    gw, gref = run_1d(1000, 100000, 8, seed=0)
    check_grad(gw, gref)


def test_backward_few_samples_per_bin():
    """Far fewer samples than bins: most bins get no sample."""
    gw, gref = run_1d(1 << 16, 5000, 12, seed=5)
    check_grad(gw, gref)


def test_backward_ragged_tail():
    """n not a multiple of the 2048-element tiles of the suffix scan."""
    gw, gref = run_1d(3 * 8192 + 1234, 1 << 18, 12, seed=6)
    check_grad(gw, gref)


def test_backward_single_bin_is_zero():
    w = np.array([3.0], np.float32)
    u = W.iid_u32(4096, seed=1)
    g = W.normal_f32(4096, seed=2)
    wd = to_dev(w)
    f = api.rtf_build(wd, 2)
    ud = api.u32_tensor(u, DEV)
    idx, pos = api.rtf_sample(f, ud)
    gw = api.rtf_sample_backward(f, wd, ud, None, idx, pos, to_dev(g))
    # xi W - 0 over W: the weight cancels exactly in the relaxed position
    assert abs(float(gw.item())) <= 1e-5 * float(np.abs(g).sum())


def test_backward_without_samples_is_zero():
    """No samples: every per-bin sum is zero and so is every element of the
    gradient (output buffers pre-filled with NaN), for 1-D, 2-D and an
    accumulator that received no batch; sampling no samples is a no-op."""
    w = W.lognormal_weights(3000, seed=40, sigma=1.0)
    wd = to_dev(w)
    f = api.rtf_build(wd, 8)
    eu = api.u32_tensor(np.zeros(0, np.uint32), DEV)
    idx, pos = api.rtf_sample(f, eu)
    assert idx.numel() == 0 and pos.numel() == 0
    ef = torch.empty(0, dtype=torch.float32, device=DEV)
    gw = torch.full_like(wd, float("nan"))
    api.rtf_sample_backward(f, wd, eu, None, idx, pos, ef, grad_w=gw)
    acc = api.GradientAccumulator(f).begin()
    gw2 = acc.finish(wd, torch.full_like(wd, float("nan")))
    H, Wd = 8, 16
    lum = to_dev(W.env_map(H, Wd, seed=41).reshape(-1))
    fe = api.rtf_build_batched(lum, [Wd] * H + [H], [4] * (H + 1), marginal=True)
    e2 = torch.empty((0, 2), dtype=torch.int32, device=DEV)
    gw3 = torch.full_like(lum, float("nan"))
    api.rtf_sample_backward(fe, lum, eu, None, e2, e2.float(), e2.float(), mode=api.SAMPLE_2D,
                            grad_w=gw3)
    torch.cuda.synchronize()
    f.check_status()
    fe.check_status()
    for g in (gw, gw2, gw3):
        assert torch.equal(g, torch.zeros_like(g))


def test_backward_config_full():
    """n = 2^20 lognormal(0, 1), 2^24 uniform samples, dL/dx ~ N(0, 1)."""
    gw, gref = run_1d(1 << 20, 1 << 24, 18, seed=10)
    check_grad(gw, gref)


def oracle_grad_sorted(w, m, u, g, idx_gpu):
    """The oracle's gradient for many samples: the same samples taken in
    ascending order (the gradient is a sum over the samples; sorted, the
    oracle's searches stay in cache), indices checked against the GPU's."""
    n_s = u.size
    key = (u.astype(np.uint64) << np.uint64(32)) | np.arange(n_s, dtype=np.uint64)
    key.sort()
    order = (key & np.uint64(0xFFFFFFFF)).astype(np.int64)
    del key
    us, gs = u[order], g[order]
    ref = orc.build(w, 1 << m)
    ridx, _ = orc.sample(ref.C, us, threads=orc.host_threads())
    assert np.array_equal(idx_gpu[order], ridx)
    return orc.grad_q(ref.C, ref.S, us, ridx, gs)


def test_backward_two_pass_scatter():
    """2^26 samples into 2^24 lognormal(0, 2) bins (the benchmark's weights):
    the per-bin sums (128 MiB) exceed 3/4 of the L2 with 4 samples per bin, so
    the scatter adds them in two passes over the halves of the bins."""
    n, n_s, m = 1 << 24, 1 << 26, 20
    w = W.lognormal_weights(n, seed=30, sigma=2.0)
    u = W.iid_u32(n_s, seed=31)
    g = W.normal_f32(n_s, seed=32)
    wd = to_dev(w)
    f = api.rtf_build(wd, m)
    ud = api.u32_tensor(u, DEV)
    idx, pos = api.rtf_sample(f, ud)
    gw = api.rtf_sample_backward(f, wd, ud, None, idx, pos, to_dev(g))
    torch.cuda.synchronize()
    f.check_status()
    gref = oracle_grad_sorted(w, m, u, g, idx.cpu().numpy())
    check_grad(gw.cpu().numpy(), gref)


def test_backward_bench_workload():
    """The benchmark's backward, input for input: n = 2^24 lognormal(0, 2)
    weights (seed 0), 2^20 cells, the 2^28 i.i.d. samples (seed 1) and
    dL/dx ~ N(0, 1) (seed 2), in the launch configuration the benchmark times
    (one call, two scatter passes)."""
    n, n_s, m = 1 << 24, 1 << 28, 20
    w = W.lognormal_weights(n, seed=0, sigma=2.0)
    u = W.iid_u32(n_s, seed=1)
    g = W.normal_f32(n_s, seed=2)
    wd = to_dev(w)
    f = api.rtf_build(wd, m)
    ud = api.u32_tensor(u, DEV)
    idx, pos = api.rtf_sample(f, ud)
    gd = to_dev(g)
    gw = api.rtf_sample_backward(f, wd, ud, None, idx, pos, gd)
    torch.cuda.synchronize()
    f.check_status()
    idx_h = idx.cpu().numpy()
    gw_h = gw.cpu().numpy()
    del ud, idx, pos, gd, gw
    gref = oracle_grad_sorted(w, m, u, g, idx_h)
    check_grad(gw_h, gref)


def test_backward_sorted_samples_merge_runs():
    """Sorted samples put long runs of equal bins inside a warp."""
    n, n_s, m = 5000, 1 << 20, 10
    w = W.lognormal_weights(n, seed=20, sigma=1.0)
    u = W.sorted_radical_inverse_u32(n_s)
    g = W.normal_f32(n_s, seed=21)
    wd = to_dev(w)
    f = api.rtf_build(wd, m)
    ud = api.u32_tensor(u, DEV)
    idx, pos = api.rtf_sample(f, ud)
    gw = api.rtf_sample_backward(f, wd, ud, None, idx, pos, to_dev(g))
    ref = orc.build(w, 1 << m)
    ridx, _ = orc.sample(ref.C, u)
    gref = orc.grad(w, u, ridx, g)
    check_grad(gw.cpu().numpy(), gref)


def test_backward_tagged_batch():
    sizes = [1, 17, 300, 4096, 2049]
    ms = [0, 3, 6, 10, 9]
    w = np.concatenate([W.lognormal_weights(s, seed=30 + i, sigma=1.0) for i, s in enumerate(sizes)])
    n_s = 1 << 18
    rng = np.random.default_rng(31)
    dist = rng.integers(0, len(sizes), n_s).astype(np.int32)
    u = W.iid_u32(n_s, seed=32)
    g = W.normal_f32(n_s, seed=33)
    wd = to_dev(w)
    f = api.rtf_build_batched(wd, sizes, ms)
    ud = api.u32_tensor(u, DEV)
    dd = to_dev(dist)
    idx, pos = api.rtf_sample(f, ud, dist_id=dd)
    gw = api.rtf_sample_backward(f, wd, ud, dd, idx, pos, to_dev(g)).cpu().numpy()
    off = f.offsets
    gref = np.zeros(w.size)
    for d in range(len(sizes)):
        sel = dist == d
        ref = orc.build(w[off[d]:off[d + 1]], 1 << ms[d])
        ridx, _ = orc.sample(ref.C, u[sel])
        gref[off[d]:off[d + 1]] = orc.grad(w[off[d]:off[d + 1]], u[sel], ridx, g[sel])
    check_grad(gw, gref)


@pytest.mark.parametrize("H,Wd,n_s", [(32, 64, 1 << 16), (512, 1024, 1 << 22)])
def test_backward_env_map(H, Wd, n_s):
    lum = W.env_map(H, Wd, seed=40)
    m_row, m_col = 9, 10
    sizes = [Wd] * H + [H]
    ms = [m_col] * H + [m_row]
    wd = to_dev(lum.reshape(-1))
    f = api.rtf_build_batched(wd, sizes, ms, marginal=True)
    rng = np.random.default_rng(41)
    u = rng.integers(0, 1 << 32, 2 * n_s, dtype=np.uint64).astype(np.uint32)
    g = W.normal_f32(2 * n_s, seed=42)
    ud = api.u32_tensor(u, DEV)
    idx, pos = api.rtf_sample(f, ud, mode=api.SAMPLE_2D)
    gw = api.rtf_sample_backward(f, wd, ud, None, idx, pos, to_dev(g), mode=api.SAMPLE_2D)
    torch.cuda.synchronize()
    f.check_status()
    rows, marg = orc.build_env(lum, 1 << m_row, 1 << m_col)
    r, c, _, _ = orc.sample_env(rows, marg, u[0::2], u[1::2])
    ii = idx.cpu().numpy()
    assert np.array_equal(ii[:, 0], r) and np.array_equal(ii[:, 1], c)
    gref = orc.grad_env(lum, u[0::2], u[1::2], r, c, g[0::2], g[1::2]).reshape(-1)
    check_grad(gw.cpu().numpy(), gref)


def test_backward_matches_gpu_forward_differences():
    """Central differences of the GPU forward (positions in float32) for
    weights whose integer q is >= 2^30, on samples whose bin does not change."""
    n, n_s, m = 64, 1 << 16, 6
    w = W.lognormal_weights(n, seed=50, sigma=0.5)
    u = W.iid_u32(n_s, seed=51)
    g = W.normal_f32(n_s, seed=52)
    wd = to_dev(w)
    ud = api.u32_tensor(u, DEV)
    f = api.rtf_build(wd, m)
    idx, pos = api.rtf_sample(f, ud)
    gw = api.rtf_sample_backward(f, wd, ud, None, idx, pos, to_dev(g)).cpu().numpy()
    i0 = idx.cpu().numpy()
    for k in (3, 17, 40):
        h = np.float32(1e-2) * w[k]
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fp = api.rtf_build(to_dev(wp), m)
        ip, pp = api.rtf_sample(fp, ud)
        ip, pp = ip.cpu().numpy(), pp.cpu().numpy().astype(np.float64)
        fm = api.rtf_build(to_dev(wm), m)
        im, pm = api.rtf_sample(fm, ud)
        im, pm = im.cpu().numpy(), pm.cpu().numpy().astype(np.float64)
        keep = (ip == i0) & (im == i0)
        hk = float(wp[k]) - float(wm[k])
        fd = np.dot(g[keep].astype(np.float64), pp[keep] - pm[keep]) / hk
        # the analytic gradient restricted to the same samples
        ref = orc.build(w, 1 << m)
        ridx, _ = orc.sample(ref.C, u[keep])
        gk = orc.grad(w, u[keep], ridx, g[keep])[k]
        assert abs(fd - gk) <= 2e-3 * (abs(gk) + np.abs(g[keep]).sum() * 1e-4)
    assert np.isfinite(gw).all()


def test_autograd_function_matches_oracle():
    from paper_1901_05423_gb300.autograd import sample_positions
    n, n_s, m = 3000, 1 << 16, 11
    w_h = W.lognormal_weights(n, seed=60, sigma=1.0)
    u_h = W.iid_u32(n_s, seed=61)
    c_h = W.normal_f32(n_s, seed=62)
    w = to_dev(w_h).requires_grad_(True)
    pos, idx = sample_positions(w, api.u32_tensor(u_h, DEV), m)
    loss = (pos * to_dev(c_h)).sum()
    loss.backward()
    ref = orc.build(w_h, 1 << m)
    ridx, _ = orc.sample(ref.C, u_h)
    assert np.array_equal(idx.cpu().numpy(), ridx)
    gref = orc.grad(w_h, u_h, ridx, c_h)
    check_grad(w.grad.cpu().numpy(), gref)


def test_autograd_function_2d_matches_oracle():
    from paper_1901_05423_gb300.autograd import sample_positions_2d
    H, Wd, n_s = 24, 40, 1 << 15
    lum_h = W.env_map(H, Wd, seed=63)
    rng = np.random.default_rng(64)
    u_h = rng.integers(0, 1 << 32, 2 * n_s, dtype=np.uint64).astype(np.uint32)
    c_h = W.normal_f32(2 * n_s, seed=65).reshape(n_s, 2)
    lum = to_dev(lum_h).requires_grad_(True)
    pos, idx = sample_positions_2d(lum, api.u32_tensor(u_h, DEV), 6, 7)
    (pos * to_dev(c_h)).sum().backward()
    rows, marg = orc.build_env(lum_h, 1 << 6, 1 << 7)
    r, c, _, _ = orc.sample_env(rows, marg, u_h[0::2], u_h[1::2])
    gref = orc.grad_env(lum_h, u_h[0::2], u_h[1::2], r, c, c_h[:, 0].copy(), c_h[:, 1].copy())
    check_grad(lum.grad.cpu().numpy(), gref)


def test_accumulated_backward_equals_one_call():
    """begin / accumulate over uneven chunks / finish gives the one-call
    gradient up to float summation order, and the oracle's within 1e-4."""
    n, n_s, m = 50000, 300001, 13
    w = W.lognormal_weights(n, seed=100, sigma=1.5)
    u = W.iid_u32(n_s, seed=101)
    g = W.normal_f32(n_s, seed=102)
    wd, ud, gd = to_dev(w), api.u32_tensor(u, DEV), to_dev(g)
    f = api.rtf_build(wd, m)
    idx, pos = api.rtf_sample(f, ud)
    one = api.rtf_sample_backward(f, wd, ud, None, idx, pos, gd).cpu().numpy()
    acc = api.GradientAccumulator(f).begin()
    cuts = [0, 7, 100000, 100004, 250000, n_s]
    for a, b in zip(cuts[:-1], cuts[1:]):
        acc.accumulate(idx[a:b], pos[a:b], gd[a:b])
    split = acc.finish(wd).cpu().numpy()
    assert rel_err(split, one.astype(np.float64)) <= 1e-5
    ref = orc.build(w, 1 << m)
    ridx, _ = orc.sample(ref.C, u)
    check_grad(split, orc.grad(w, u, ridx, g))


def test_accumulated_backward_2d_and_on_a_second_stream():
    """2-D accumulation, with the accumulate calls on a side stream ordered by
    events after the samples they read."""
    H, Wd, n_s = 64, 96, 1 << 16
    lum = W.env_map(H, Wd, seed=110)
    wd = to_dev(lum.reshape(-1))
    f = api.rtf_build_batched(wd, [Wd] * H + [H], [7] * H + [6], marginal=True)
    rng = np.random.default_rng(111)
    u = rng.integers(0, 1 << 32, 2 * n_s, dtype=np.uint64).astype(np.uint32)
    g = W.normal_f32(2 * n_s, seed=112)
    ud, gd = api.u32_tensor(u, DEV), to_dev(g)
    idx = torch.empty((n_s, 2), dtype=torch.int32, device=DEV)
    pos = torch.empty((n_s, 2), dtype=torch.float32, device=DEV)
    side = torch.cuda.Stream()
    acc = api.GradientAccumulator(f, mode=api.SAMPLE_2D)
    ev0 = torch.cuda.Event()
    ev0.record()
    side.wait_event(ev0)
    with torch.cuda.stream(side):
        acc.begin()
    half = n_s // 2
    for a, b in ((0, half), (half, n_s)):
        api.rtf_sample(f, ud[2 * a:2 * b], mode=api.SAMPLE_2D, idx_out=idx[a:b], pos_out=pos[a:b])
        ev = torch.cuda.Event()
        ev.record()
        side.wait_event(ev)
        with torch.cuda.stream(side):
            acc.accumulate(idx[a:b], pos[a:b], gd[2 * a:2 * b])
    torch.cuda.current_stream().wait_stream(side)
    split = acc.finish(wd).cpu().numpy()
    one = api.rtf_sample_backward(f, wd, ud, None, idx, pos, gd, mode=api.SAMPLE_2D).cpu().numpy()
    assert rel_err(split, one.astype(np.float64)) <= 1e-5
