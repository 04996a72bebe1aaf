"""Seeded synthetic inputs for the radix-tree-forest sampler.

This module only draws random numbers and arranges them; it holds none of the
method's arithmetic, so both the CUDA path and the CPU oracle may take their
inputs from it.  The paper's own workloads (an HDR environment photograph and
the data behind its Table 1) are not available; the generators below stand in
for them with the shapes and value distributions stated in each docstring.

All generators use ``numpy.random.default_rng(seed)`` and return host numpy
arrays.  Weights are float32, samples uint32.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "radical_inverse_u32", "sorted_radical_inverse_u32", "iid_u32",
    "uniform_weights", "lognormal_weights", "env_map", "ragged_batch",
    "normal_f32", "table1_weights", "TABLE1_KINDS",
]


def radical_inverse_u32(count: int) -> np.ndarray:
    """Base-2 radical inverse of 0..count-1 as 32-bit fixed point (the bits of
    j mirrored about the binary point), in generation order."""
    j = np.arange(count, dtype=np.uint32)
    r = j.copy()
    r = ((r >> np.uint32(1)) & np.uint32(0x55555555)) | ((r & np.uint32(0x55555555)) << np.uint32(1))
    r = ((r >> np.uint32(2)) & np.uint32(0x33333333)) | ((r & np.uint32(0x33333333)) << np.uint32(2))
    r = ((r >> np.uint32(4)) & np.uint32(0x0F0F0F0F)) | ((r & np.uint32(0x0F0F0F0F)) << np.uint32(4))
    r = ((r >> np.uint32(8)) & np.uint32(0x00FF00FF)) | ((r & np.uint32(0x00FF00FF)) << np.uint32(8))
    r = (r >> np.uint32(16)) | (r << np.uint32(16))
    return r


def sorted_radical_inverse_u32(count: int) -> np.ndarray:
    """The radical-inverse set of a power-of-two size, sorted: j * 2^32/count."""
    assert count & (count - 1) == 0 and 0 < count <= 1 << 32
    step = (1 << 32) // count
    return (np.arange(count, dtype=np.uint64) * np.uint64(step)).astype(np.uint32)


def iid_u32(count: int, seed: int) -> np.ndarray:
    """Independent uniform 32-bit samples in random order."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1 << 32, size=count, dtype=np.uint32)


def uniform_weights(n: int, seed: int, lo: float = 0.01, hi: float = 1.0) -> np.ndarray:
    """n weights i.i.d. uniform(lo, hi), float32."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n).astype(np.float32)


def lognormal_weights(n: int, seed: int, sigma: float, mu: float = 0.0) -> np.ndarray:
    """n weights exp(N(mu, sigma^2)), float32."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.normal(mu, sigma, n)).astype(np.float32)


def normal_f32(count: int, seed: int) -> np.ndarray:
    """count values N(0, 1), float32 (incoming gradients)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(count, dtype=np.float32)


def env_map(rows: int, cols: int, seed: int, spots: int = 3,
            spot_sigma: float = 4.0, spot_peak: float = 1e5) -> np.ndarray:
    """Synthetic HDR environment luminance, float32[rows, cols].

    L(r, c) = (1.5 + sin(3x) cos(2y)) * exp(N(0, 1)) + sum of `spots` Gaussian
    hot spots (sigma `spot_sigma` pixels, peak `spot_peak`), with
    x = 2 pi (c + 1/2) / cols and y = pi (r + 1/2) / rows.  The spot centres are
    uniform over the map.
    """
    rng = np.random.default_rng(seed)
    x = 2.0 * np.pi * (np.arange(cols) + 0.5) / cols
    y = np.pi * (np.arange(rows) + 0.5) / rows
    base = 1.5 + np.sin(3.0 * x)[None, :] * np.cos(2.0 * y)[:, None]
    lum = base * np.exp(rng.normal(0.0, 1.0, (rows, cols)))
    cr = rng.uniform(0, rows, spots)
    cc = rng.uniform(0, cols, spots)
    rr = np.arange(rows)[:, None] + 0.5
    ccol = np.arange(cols)[None, :] + 0.5
    for k in range(spots):
        d2 = (rr - cr[k]) ** 2 + (ccol - cc[k]) ** 2
        lum = lum + spot_peak * np.exp(-d2 / (2.0 * spot_sigma ** 2))
    return lum.astype(np.float32)


def ragged_batch(num: int, seed: int, nmin: int = 8, nmax: int = 65536,
                 sigma: float = 1.5):
    """`num` distributions with sizes floor(exp(U(ln nmin, ln (nmax+1)))) and
    weights exp(N(0, sigma^2)).  Returns (weights float32[sum n], offsets
    int64[num + 1])."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(nmin), np.log(nmax + 1), num))).astype(np.int64)
    sizes = np.clip(sizes, nmin, nmax)
    offsets = np.zeros(num + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    w = np.exp(rng.normal(0.0, sigma, int(offsets[-1]))).astype(np.float32)
    return w, offsets


def dist_ids(count: int, num: int, seed: int) -> np.ndarray:
    """count distribution ids uniform on 0..num-1, int32."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, num, size=count, dtype=np.int32)


TABLE1_KINDS = ("i^20", "(i mod 32 + 1)^25", "(i mod 64 + 1)^35", "4 spikes")


def table1_weights(kind: str, n: int = 1024, seed: int = 0) -> np.ndarray:
    """The four density shapes of the paper's Table 1 (Fig. 13), scaled so the
    largest weight is 1 (evaluated in float64, then rounded to float32, so the
    smallest powers underflow to zero as they would in any float32 input):

    ``i^20``, ``(i mod 32 + 1)^25``, ``(i mod 64 + 1)^35`` for i = 0..n-1, and
    ``4 spikes``: the paper shows but does not define it; here four Gaussian
    bumps of width n/256 at uniform random positions with heights 1, 1/2,
    1/4, 1/8 over a floor of 1e-3.
    """
    i = np.arange(n, dtype=np.float64)
    if kind == "i^20":
        w = (i / (n - 1)) ** 20
    elif kind == "(i mod 32 + 1)^25":
        w = ((i % 32 + 1) / 32.0) ** 25
    elif kind == "(i mod 64 + 1)^35":
        w = ((i % 64 + 1) / 64.0) ** 35
    elif kind == "4 spikes":
        rng = np.random.default_rng(seed)
        c = rng.uniform(0, n, 4)
        s = n / 256.0
        w = np.full(n, 1e-3)
        for k in range(4):
            w += 0.5 ** k * np.exp(-0.5 * ((i - c[k]) / s) ** 2)
    else:
        raise ValueError(f"unknown kind {kind!r}")
    return w.astype(np.float32)

