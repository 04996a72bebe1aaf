"""Autotuner of the guide size for ragged batches and of the samplers'
launch shape.

The paper leaves the guide table size to the application: as large as memory
allows, or proportional to the size of the distribution (Sec. 3).  For a
batch of many distributions of different sizes the choice per size class is
measured here on the GPU: for every power-of-two size bucket a batch of
synthetic lognormal distributions of that size is built and sampled (one
tagged sample per weight, the ratio of the ragged workload) for each candidate
number of guide bits m around log2(n), and the m with the smallest build +
sampling time wins.

The launch shape (resident blocks per SM of each kind of sampling launch,
``rtf_set_launch_shape``) is tuned on the caller's own structure and samples:
each candidate is timed on them and the fastest is set.  It matters most where
the structure does not fit L2 and the samples are scattered: fewer resident
descents then keep more of the structure in L2.

Results are cached per GPU model in JSON files (``$RTF_CACHE_DIR`` or
``~/.cache/rtf``).
"""

from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import api
from . import workloads as W

DEFAULT_OFFSETS = (-2, -1, 0, 1, 2)


def _cache_path(device: torch.device, what: str = "guide_bits") -> str:
    root = os.environ.get("RTF_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "rtf")
    name = torch.cuda.get_device_name(device).replace(" ", "_")
    return os.path.join(root, f"{what}_{name}.json")


def _time_bucket(n: int, m: int, device, total: int, reps: int, seed: int) -> float:
    D = max(1, total // n)
    sizes = [n] * D
    w = torch.from_numpy(W.lognormal_weights(n * D, seed=seed, sigma=1.5)).to(device)
    ns = n * D
    u = api.u32_tensor(W.iid_u32(ns, seed=seed + 1), device)
    dist = torch.from_numpy(W.dist_ids(ns, D, seed=seed + 2)).to(device)
    idx = torch.empty(ns, dtype=torch.int32, device=device)
    pos = torch.empty(ns, dtype=torch.float32, device=device)
    f = api.rtf_build_batched(w, sizes, [m] * D)
    api.rtf_sample(f, u, dist_id=dist, idx_out=idx, pos_out=pos)
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        api.rtf_build_batched(w, sizes, [m] * D, forest=f, plan_dev=f._plan_dev)
        api.rtf_sample(f, u, dist_id=dist, idx_out=idx, pos_out=pos)
    e1.record()
    torch.cuda.synchronize(device)
    f.check_status()
    return e0.elapsed_time(e1) / reps


def tune(device=None, buckets=range(3, 17), offsets=DEFAULT_OFFSETS, total: int = 1 << 22,
         reps: int = 3, use_cache: bool = True) -> dict:
    """Guide bits per size bucket: {bucket: m} with bucket = round(log2 n)."""
    device = torch.device(device or "cuda:0")
    path = _cache_path(device)
    if use_cache and os.path.exists(path):
        with open(path) as fh:
            table = {int(k): int(v) for k, v in json.load(fh).items()}
        if all(b in table for b in buckets):
            return table
    table = {}
    for b in buckets:
        n = 1 << b
        best = None
        for off in offsets:
            m = min(max(b + off, 0), 24)
            t = _time_bucket(n, m, device, total, reps, seed=b)
            if best is None or t < best[0]:
                best = (t, m)
        table[b] = best[1]
    if use_cache:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as fh:
            json.dump({str(k): v for k, v in table.items()}, fh)
    return table


def guide_bits_for(sizes, table: dict) -> np.ndarray:
    """m per distribution from a tuned table (nearest bucket, clamped)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    b = np.clip(np.round(np.log2(np.maximum(sizes, 1))).astype(int), min(table), max(table))
    lut = np.array([table.get(int(k), int(k)) for k in range(0, max(table) + 1)])
    return lut[b].astype(np.int32)


DEFAULT_SHAPES = (2, 3, 4, 6, 8, 12, 16)


def _launch_kind(forest, u, dist_id, mode) -> str:
    if (mode & 0xFF) == api.SAMPLE_2D:
        return "pairs"
    if dist_id is not None:
        return "tagged"
    records = forest.num_elems * api.NODE_BYTES + forest.num_cells * api.GUIDE_REC_BYTES
    l2 = torch.cuda.get_device_properties(u.device).L2_cache_size
    return "single_large" if records > l2 else "single"


def tune_launch_shape(forest, u: torch.Tensor, dist_id: torch.Tensor | None = None,
                      mode: int = api.SAMPLE_1D, candidates=DEFAULT_SHAPES, reps: int = 3,
                      key: str | None = None, use_cache: bool = True) -> tuple[str, int, dict]:
    """Time rtf_sample on (forest, u, dist_id, mode) with each candidate number
    of blocks per SM for the kind of launch it makes, set the fastest and
    return (kind, blocks per SM, {candidate: ms}).  With `key`, the choice is
    cached under it (per GPU model) and reused without timing."""
    if mode & api.SAMPLE_COHERENT:
        raise api.RtfError("the coherent sampler runs one wave of resident blocks; nothing to tune")
    kind = _launch_kind(forest, u, dist_id, mode)
    path = _cache_path(u.device, "launch_shape")
    cache = {}
    if use_cache and key is not None and os.path.exists(path):
        with open(path) as fh:
            cache = json.load(fh)
        if f"{kind}/{key}" in cache:
            best = int(cache[f"{kind}/{key}"])
            api.set_launch_shape(**{kind: best})
            return kind, best, {}
    two_d = (mode & 0xFF) == api.SAMPLE_2D
    count = u.numel() // (2 if two_d else 1)
    shape = (count, 2) if two_d else (count,)
    idx = torch.empty(shape, dtype=torch.int32, device=u.device)
    pos = torch.empty(shape, dtype=torch.float32, device=u.device)
    times = {}
    for c in candidates:
        api.set_launch_shape(**{kind: int(c)})
        api.rtf_sample(forest, u, dist_id=dist_id, mode=mode, idx_out=idx, pos_out=pos)
        torch.cuda.synchronize(u.device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            api.rtf_sample(forest, u, dist_id=dist_id, mode=mode, idx_out=idx, pos_out=pos)
        e1.record()
        torch.cuda.synchronize(u.device)
        times[int(c)] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    api.set_launch_shape(**{kind: best})
    if use_cache and key is not None:
        cache[f"{kind}/{key}"] = best
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as fh:
            json.dump(cache, fh)
    return kind, best, times


def tune_env_bits(lum: torch.Tensor, rows: int, cols: int, pairs_per_build: int,
                  row_offsets=(-2, -1, 0, 1, 2), marg_offsets=(-1, 0, 1),
                  probe_pairs: int = 1 << 24, reps: int = 3, seed: int = 0,
                  use_cache: bool = True) -> tuple[int, int, dict]:
    """Guide bits of a 2-D map (Sec. 5: one table per row and one over the
    rows): for each candidate (m_row, m_marginal) around (log2 cols,
    log2 rows), the batched build and `probe_pairs` 2-D samples are timed on
    the caller's map `lum` (device float32[rows * cols]); the pair with the
    smallest build + pairs_per_build samples wins.  Larger tables cost build
    time and memory and save node loads (a cell that one interval covers needs
    none).  Returns (m_row, m_marginal, {(m_row, m_marginal): ms}); the choice
    is cached per GPU model, map shape and pairs_per_build."""
    device = lum.device
    path = _cache_path(device, "env_bits")
    key = f"{rows}x{cols}/{pairs_per_build}"
    cache = {}
    if use_cache and os.path.exists(path):
        with open(path) as fh:
            cache = json.load(fh)
        if key in cache:
            mr, mm = cache[key]
            return int(mr), int(mm), {}
    sizes = [cols] * rows + [rows]
    br = int(round(np.log2(max(cols, 1))))
    bm = int(round(np.log2(max(rows, 1))))
    u = api.u32_tensor(W.iid_u32(2 * probe_pairs, seed=seed), device)
    idx = torch.empty((probe_pairs, 2), dtype=torch.int32, device=device)
    pos = torch.empty((probe_pairs, 2), dtype=torch.float32, device=device)
    times = {}
    for orow in row_offsets:
        for om in marg_offsets:
            mr, mm = min(max(br + orow, 0), 20), min(max(bm + om, 0), 20)
            ms = [mr] * rows + [mm]
            f = api.rtf_build_batched(lum, sizes, ms, marginal=True)
            api.rtf_sample(f, u, mode=api.SAMPLE_2D, idx_out=idx, pos_out=pos)
            torch.cuda.synchronize(device)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            for _ in range(reps):
                api.rtf_build_batched(lum, sizes, ms, marginal=True, forest=f, plan_dev=f._plan_dev)
            e[1].record()
            for _ in range(reps):
                api.rtf_sample(f, u, mode=api.SAMPLE_2D, idx_out=idx, pos_out=pos)
            e[2].record()
            torch.cuda.synchronize(device)
            f.check_status()
            tb = e[0].elapsed_time(e[1]) / reps
            ts = e[1].elapsed_time(e[2]) / reps
            times[(mr, mm)] = tb + ts * pairs_per_build / probe_pairs
            del f
    mr, mm = min(times, key=times.get)
    if use_cache:
        cache[key] = [mr, mm]
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as fh:
            json.dump(cache, fh)
    return mr, mm, times
