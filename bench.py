"""Benchmark of the radix-tree-forest sampling path on one GB300.

One step = the whole path on the n = 2^24 workload:
  build (validation + scale, exact integer CDF, keys, forest, guide) of
  2^24 lognormal(0, 2) weights with 2^20 guide cells,
  sampling of 2^28 i.i.d. uniform uint32 samples and of the 2^28 sorted
  radical-inverse samples (index + float32 in-bin position),
  backward of the i.i.d. positions (dL/dx ~ N(0, 1)) to dL/dw.
value = samples mapped per second over the whole step (2 x 2^28 samples per
step; the build and the backward are inside the timed region).  Every input is
larger than L2, so no L2 flush is needed between steps.

`--impl reference` times the CPU oracle on a bounded sample of the same
workload instead (the paper has no reference implementation to run).
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "samples/s & build elem/s at n=2^24 (bit-exact); batched vs looped; % HBM peak"
N_W = 1 << 24
M_BITS = 20
N_S = 1 << 28
# kernels of this library per step: build 6 (init_dists, scale, tile_sum,
# forest_lean, forest_merge, fill), sampling 2, backward 4 (scatter in two
# passes over the halves of the 2^24 bins, bin_total, suffix)
LAUNCHES_PER_STEP = 12
# with --streams 3 the i.i.d. set is sampled in ACC_CHUNKS chunks and each
# chunk's terms added by one scatter pass (2^25 samples: under 4 per bin)
LAUNCHES_PER_STEP_ACC = 6 + 1 + 8 + 8 + 2


# DRAM bytes per unit measured by ncu at full size (dram__bytes_read.sum +
# dram__bytes_write.sum per launch / units per launch;
# profiles/launches_bench_n24.md), with the SHA-256 prefixes of the kernel
# sources they were captured from.  An entry whose sources have changed since
# is reported as null until the capture is repeated.
TRAFFIC_CAPTURES = {
    "sample_iid": {
        "bytes_per_unit": (37.960e9 + 2.144e9) / (1 << 28),
        "sources": {"paper_1901_05423_gb300/csrc/sample.cu": "cadb9701cb6d872d",
                    "paper_1901_05423_gb300/csrc/sample_common.cuh": "7836d4584a4ff2cf"},
    },
}


def _sha16(rel: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def traffic_per_unit(kernel: str):
    """(bytes per unit, "current" | "stale" | "none") of an ncu capture."""
    cap = TRAFFIC_CAPTURES.get(kernel)
    if cap is None:
        return None, "none"
    if any(_sha16(f) != h for f, h in cap["sources"].items()):
        return None, "stale"
    return cap["bytes_per_unit"], "current"


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """Per-step time of the job: the slowest rank's (each rank runs a full
    replica of the workload on its own GPU)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: int, ms: float) -> float:
    """Units of all ranks per second (weak scaling: every rank maps its own
    2 x 2^28 samples)."""
    return world * units_per_rank / (ms * 1e-3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def wait_ready(self, timeout=5.0):
        """Block until nvidia-smi printed its first sample (it takes a while
        to start), so that the samples cover the timed region."""
        t_end = time.monotonic() + timeout
        while self.proc is not None and not self.lines and time.monotonic() < t_end:
            time.sleep(0.01)

    def mark(self, which):
        setattr(self, which, time.monotonic())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t_start", None), getattr(self, "t_end", None)
        for t, ln in self.lines:
            # a sample printed at t describes the interval just before it
            if t0 is not None and not (t0 < t <= t1 + 0.05):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(sorted_dense=False):
    from paper_1901_05423_gb300 import workloads as W
    w = W.lognormal_weights(N_W, seed=0, sigma=2.0)
    u_iid = W.iid_u32(N_S, seed=1)
    # sorted_dense: the first N_S samples of the 2^28-sample sorted set (its
    # density, 16 u-units apart, over part of [0, 1)) instead of N_S samples
    # spread over all of [0, 1); a profiling aid for small N_S
    u_sorted = ((np.arange(N_S, dtype=np.uint64) * np.uint64(16)).astype(np.uint32) if sorted_dense
                else W.sorted_radical_inverse_u32(N_S))
    gx = W.normal_f32(N_S, seed=2)
    return w, u_iid, u_sorted, gx


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------

def time_oracle(w, u_iid, u_sorted, gx, sample_count=1 << 21, threads=1):
    """The oracle on a bounded sample of one step: the build of n = 2^24
    (sequential by definition), index + position of `sample_count` samples of
    each set (on `threads` host threads, the samples cut into contiguous
    chunks) and the gradient of `sample_count` samples (sequential); scaled
    linearly to 2^28 samples per set."""
    from oracle import oracle as orc
    t_all = time.perf_counter()
    t0 = time.perf_counter()
    st = orc.build(w, 1 << M_BITS)
    t_build = time.perf_counter() - t0
    ui = u_iid[:sample_count]
    us = u_sorted[::max(1, N_S // sample_count)][:sample_count]
    t0 = time.perf_counter()
    idx_i, _ = orc.sample(st.C, ui, threads=threads)
    orc.sample(st.C, us, threads=threads)
    t_sample = time.perf_counter() - t0
    t0 = time.perf_counter()
    orc.grad_q(st.C, st.S, ui, idx_i, gx[:sample_count])
    t_grad = time.perf_counter() - t0
    measured = time.perf_counter() - t_all
    scale = N_S / sample_count
    step = t_build + t_sample * scale + t_grad * scale
    lg = N_S.bit_length() - 1
    return {
        "step_s": step,
        "measured_s": measured,
        "scale": scale,
        "value": 2 * N_S / step,
        "build_elem_per_s": N_W / t_build,
        "sample_per_s": 2 * sample_count / t_sample,
        "sample": (f"oracle build of n=2^24 (timed once, 1 core), index+position on {sample_count} "
                   f"i.i.d. + {sample_count} sorted samples on {threads} host thread(s), the "
                   f"gradient on {sample_count} samples (1 core); sampling and gradient scaled "
                   f"linearly by {scale:g} to 2^{lg} samples per set"),
    }


def cpu_baseline(w, u_iid, u_sorted, gx, sample_count=1 << 21):
    """The oracle on one host core and on all of them (sampling threaded)."""
    from oracle import oracle as orc
    cores = orc.host_threads()
    one = time_oracle(w, u_iid, u_sorted, gx, sample_count, threads=1)
    allc = time_oracle(w, u_iid, u_sorted, gx, sample_count, threads=cores)
    return {"value": allc["value"], "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": allc["sample"], "host_cores": os.cpu_count(),
            "value_1core": one["value"], "sample_1core": one["sample"],
            "sample_per_s": allc["sample_per_s"], "sample_per_s_1core": one["sample_per_s"],
            "build_elem_per_s": one["build_elem_per_s"]}


def workload_config(world: int, streams: int, sorted_dense: bool = False) -> dict:
    lg = N_S.bit_length() - 1
    return {"workload": f"n=2^24 lognormal(0,2) weights, 2^20 guide cells, "
                        f"2^{lg} iid + 2^{lg} sorted radical-inverse samples"
                        + (" (the first of the 2^28 set)" if sorted_dense else "")
                        + ", backward on the iid set",
            "l2": "inputs larger than L2", "parallelism": f"replicas{world}",
            "streams": {1: "1", 2: "2: sorted set concurrent with the i.i.d. set and "
                                    "the backward",
                        3: "3: sorted set concurrent; backward accumulated per chunk of "
                           "the i.i.d. set while later chunks are mapped"}[streams]}


def reference_arm(args):
    """The oracle timed on the host cores (rank 0 only).  Each step is the
    build plus a bounded sample of 2^19 samples per set (sampling on all host
    cores); `ms_per_step` is that measured step, `value` the throughput of the
    full step extrapolated from it (scale factor in `extrapolation`)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as orc
    w, u_iid, u_sorted, gx = make_inputs()
    cores = orc.host_threads()
    measured, full = [], []
    res = None
    for it in range(args.warmup + args.steps):
        res = time_oracle(w, u_iid, u_sorted, gx, sample_count=1 << 19, threads=cores)
        if it >= args.warmup:
            measured.append(res["measured_s"])
            full.append(res["step_s"])
    step = float(np.mean(full))
    value = 2 * N_S / step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(measured)) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(args.gpus, args.streams),
        "extrapolation": {"timed_samples_per_set": 1 << 19, "scale": res["scale"],
                          "full_step_ms": step * 1e3,
                          "value_basis": "samples of the full step (2 x 2^28) per second of "
                                         "the extrapolated full step"},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": res["sample"], "host_cores": os.cpu_count()},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def gpu_arm(args):
    import torch
    from paper_1901_05423_gb300 import api

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w, u_iid, u_sorted, gx = make_inputs(sorted_dense=args.sorted_dense)
    wd = torch.from_numpy(w).to(dev)
    ui = api.u32_tensor(u_iid, dev)
    us = api.u32_tensor(u_sorted, dev)
    gd = torch.from_numpy(gx).to(dev)
    idx_i = torch.empty(N_S, dtype=torch.int32, device=dev)
    pos_i = torch.empty(N_S, dtype=torch.float32, device=dev)
    idx_s = torch.empty_like(idx_i)
    pos_s = torch.empty_like(pos_i)
    grad_w = torch.empty_like(wd)
    f = api.rtf_build(wd, M_BITS)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    names = ["build", "sample_iid", "sample_sorted", "backward"]
    # the sorted set is passed with the coherence hint (a sorted sequence in order)
    SORTED_MODE = api.SAMPLE_1D | api.SAMPLE_COHERENT

    # With --streams 2 the sorted set is sampled on a second stream, at the
    # same time as the i.i.d. set and its backward: the two sides stress
    # different parts of the chip (DRAM lines and L2 updates on one, issue
    # slots on the other).
    # With --streams 3 the backward of the i.i.d. set also overlaps its
    # sampling: the set is mapped in ACC_CHUNKS chunks and each chunk's terms
    # are added to the per-bin sums on a third stream as soon as the chunk is
    # mapped (rtf_backward_accumulate); the gradient is finished once all are in.
    side = torch.cuda.Stream(dev) if args.streams >= 2 else stream
    acc_stream = torch.cuda.Stream(dev) if args.streams == 3 else None
    accum = api.GradientAccumulator(f) if args.streams == 3 else None
    ACC_CHUNKS = 8
    ev_built = torch.cuda.Event()
    ev_chunk = [torch.cuda.Event() for _ in range(ACC_CHUNKS)]

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        api.rtf_build(wd, M_BITS, forest=f)
        if ev is not None:
            ev[1].record(stream)
        if accum is not None:
            ev_built.record(stream)
            side.wait_event(ev_built)
            acc_stream.wait_event(ev_built)
            with torch.cuda.stream(side):
                if ev is not None:
                    ev[5].record(side)
                api.rtf_sample(f, us, mode=SORTED_MODE, idx_out=idx_s, pos_out=pos_s)
                if ev is not None:
                    ev[6].record(side)
            with torch.cuda.stream(acc_stream):
                accum.begin()
            cs = N_S // ACC_CHUNKS
            for k in range(ACC_CHUNKS):
                sl = slice(k * cs, (k + 1) * cs)
                api.rtf_sample(f, ui[sl], idx_out=idx_i[sl], pos_out=pos_i[sl])
                ev_chunk[k].record(stream)
                acc_stream.wait_event(ev_chunk[k])
                with torch.cuda.stream(acc_stream):
                    accum.accumulate(idx_i[sl], pos_i[sl], gd[sl])
            if ev is not None:
                ev[2].record(stream)
                ev[3].record(stream)
            stream.wait_stream(acc_stream)
            accum.finish(wd, grad_w=grad_w)
            if ev is not None:
                ev[4].record(stream)
            stream.wait_stream(side)
            return
        if side is not stream:
            ev_built.record(stream)
            side.wait_event(ev_built)
            with torch.cuda.stream(side):
                if ev is not None:
                    ev[5].record(side)
                api.rtf_sample(f, us, mode=SORTED_MODE, idx_out=idx_s, pos_out=pos_s)
                if ev is not None:
                    ev[6].record(side)
        api.rtf_sample(f, ui, idx_out=idx_i, pos_out=pos_i)
        if ev is not None:
            ev[2].record(stream)
        if side is stream:
            api.rtf_sample(f, us, mode=SORTED_MODE, idx_out=idx_s, pos_out=pos_s)
        if ev is not None:
            ev[3].record(stream)
        api.rtf_sample_backward(f, wd, ui, None, idx_i, pos_i, gd, grad_w=grad_w)
        if ev is not None:
            ev[4].record(stream)
        if side is not stream:
            stream.wait_stream(side)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    f.check_status()

    part = {k: [] for k in names}
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        clk.wait_ready()
        clk.mark("t_start")
        start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        end.record(stream)
        torch.cuda.synchronize()
        clk.mark("t_end")
    if dist:
        dist.barrier()
    total_ms = start.elapsed_time(end)
    for k in range(args.steps):
        e = evs[k]
        part["build"].append(e[0].elapsed_time(e[1]))
        part["sample_iid"].append(e[1].elapsed_time(e[2]))
        part["backward"].append(e[3].elapsed_time(e[4]))
        part["sample_sorted"].append(e[5].elapsed_time(e[6]) if side is not stream
                                     else e[2].elapsed_time(e[3]))
    f.check_status()
    ms = max_over_ranks(total_ms / args.steps, dist, dev)

    # Each part of the step alone on one stream, after the timed region (the
    # per-kernel fractions of HBM; with two streams the spans above include
    # the time a part waits for SMs held by the other stream).
    def alone(fn, reps=3):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    alone_ms = {
        "build": alone(lambda: api.rtf_build(wd, M_BITS, forest=f)),
        "sample_iid": alone(lambda: api.rtf_sample(f, ui, idx_out=idx_i, pos_out=pos_i)),
        "sample_sorted": alone(lambda: api.rtf_sample(f, us, mode=SORTED_MODE, idx_out=idx_s,
                                                      pos_out=pos_s)),
        "backward": alone(lambda: api.rtf_sample_backward(f, wd, ui, None, idx_i, pos_i, gd,
                                                          grad_w=grad_w)),
    }
    f.check_status()

    # end-to-end through the API with host buffers (pinned), copies inside
    h_w = torch.from_numpy(w).pin_memory()
    h_ui = torch.from_numpy(u_iid.view(np.int32)).pin_memory()
    h_us = torch.from_numpy(u_sorted.view(np.int32)).pin_memory()
    h_g = torch.from_numpy(gx).pin_memory()
    o_idx_i = torch.empty(N_S, dtype=torch.int32).pin_memory()
    o_pos_i = torch.empty(N_S, dtype=torch.float32).pin_memory()
    o_idx_s = torch.empty_like(o_idx_i).pin_memory()
    o_pos_s = torch.empty_like(o_pos_i).pin_memory()
    o_gw = torch.empty_like(h_w).pin_memory()

    # The end-to-end step through the public API: the weights go up on a side
    # stream, the samples stream through the pipelined sampler (copies in,
    # sampling and copies back of different chunks overlap), and dL/dpos goes
    # up once the sample sets' inputs are in (the copies back bound the step;
    # uploading dL/dpos beside the first sample chunks delays them: 30.5 vs
    # 26.6 ms per step on GB300); the step ends when every result is back in
    # host memory.
    s_up = torch.cuda.Stream(dev)
    ev_w, ev_g, ev_in = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
    ev_i, ev_s = torch.cuda.Event(), torch.cuda.Event()
    chunk = 1 << 24

    def e2e_step():
        cur = torch.cuda.current_stream(dev)
        s_up.wait_stream(cur)
        with torch.cuda.stream(s_up):
            wd.copy_(h_w, non_blocking=True)
            ev_w.record(s_up)
        cur.wait_event(ev_w)
        api.rtf_build(wd, M_BITS, forest=f)
        api.rtf_sample_pipelined(f, h_ui, ui, idx_i, pos_i, o_idx_i, o_pos_i, chunk=chunk,
                                 done_event=ev_i)
        api.rtf_sample_pipelined(f, h_us, us, idx_s, pos_s, o_idx_s, o_pos_s, chunk=chunk,
                                 done_event=ev_s, mode=SORTED_MODE)
        ev_in.record(cur)  # both sets' inputs consumed
        s_up.wait_event(ev_in)
        with torch.cuda.stream(s_up):
            gd.copy_(h_g, non_blocking=True)
            ev_g.record(s_up)
        cur.wait_event(ev_g)
        api.rtf_sample_backward(f, wd, ui, None, idx_i, pos_i, gd, grad_w=grad_w)
        o_gw.copy_(grad_w, non_blocking=True)
        cur.wait_event(ev_i)
        cur.wait_event(ev_s)

    e2e_steps = max(1, min(args.steps, 3))
    e2e_step()
    torch.cuda.synchronize()
    es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    es.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    ee.record(stream)
    torch.cuda.synchronize()
    e2e_ms = es.elapsed_time(ee) / e2e_steps
    h2d = w.nbytes + u_iid.nbytes + u_sorted.nbytes + gx.nbytes
    d2h = 4 * 4 * N_S + w.nbytes

    peak, peak_kind = measured_peaks()
    avg = {k: float(np.mean(v)) for k, v in part.items()}
    # algorithmic bytes per launch; the build reads w three times (the largest
    # exponent, the tile sums, the forest pass) and writes each node record
    # (16 B), guide entry (4 B) and guide record (32 B) once
    alg = {
        "build": 28 * N_W + 36 * (1 << M_BITS),
        "sample_iid": 12 * N_S,
        "sample_sorted": 12 * N_S,
        "backward": 16 * N_S + 24 * N_W,
    }
    # The roofline is quoted for the i.i.d. sampler: the largest share of the
    # step when its kernels run one after another (the launch list).  With the
    # sorted set on a second stream, the sorted sampler's events also span the
    # time it waits for SMs held by the other stream, so its span is no
    # kernel duration.
    dom = "sample_iid"
    achieved = alg[dom] / (avg[dom] * 1e-3) / 1e9
    units = {"build": N_W, "sample_iid": N_S, "sample_sorted": N_S, "backward": N_S}
    per_unit, traffic_state = traffic_per_unit(dom)
    traffic = per_unit * units[dom] if per_unit is not None else None
    value = job_throughput(world, 2 * N_S, ms)
    lg = N_S.bit_length() - 1
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": workload_config(world, args.streams, args.sorted_dense),
        "breakdown_ms": avg,
        "build_elem_per_s": N_W / (alone_ms["build"] * 1e-3),
        "sample_iid_per_s": N_S / (alone_ms["sample_iid"] * 1e-3),
        "sample_sorted_per_s": N_S / (alone_ms["sample_sorted"] * 1e-3),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "traffic_GBps": traffic / (avg[dom] * 1e-3) / 1e9 if traffic else None,
                     # the DRAM bytes ncu measured for this kernel (random node and guide
                     # lines included) against the same peak
                     "traffic_frac": traffic / (avg[dom] * 1e-3) / 1e9 / peak if traffic else None,
                     "traffic_capture": traffic_state, "peak_kind": peak_kind},
        "alone_ms": alone_ms,
        "fractions_of_hbm": {k: alg[k] / (alone_ms[k] * 1e-3) / 1e9 / peak for k in alone_ms},
        "e2e": {"value": job_throughput(world, 2 * N_S, max_over_ranks(e2e_ms, dist, dev)),
                "unit": "samples/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": (LAUNCHES_PER_STEP_ACC if args.streams == 3 else LAUNCHES_PER_STEP)
                        * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_extras:
        line["extras"] = {"ragged_batch": extra_ragged(dev), "env_map_2d": extra_env_map(dev),
                          "backward_vs_forward": extra_backward(dev),
                          "forest_vs_binary_search": extra_methods(dev)}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, u_iid, u_sorted, gx)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# extra workloads (reported beside the main line)
# ---------------------------------------------------------------------------

def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def extra_ragged(dev, reps=3):
    """16384 distributions (sizes log-uniform in [8, 65536], lognormal(0, 1.5)),
    guide bits from the autotuner; batched build vs a loop of single builds;
    build + 2^27 tagged samples replayed as one CUDA graph."""
    import ctypes
    import torch
    from paper_1901_05423_gb300 import _native, api, autotune
    from paper_1901_05423_gb300 import workloads as W
    w_h, off = W.ragged_batch(16384, seed=0)
    sizes = np.diff(off)
    table = autotune.tune(dev)
    ms = autotune.guide_bits_for(sizes, table)
    w = torch.from_numpy(w_h).to(dev)
    f = api.rtf_build_batched(w, sizes, ms)
    ns = 1 << 27
    u = api.u32_tensor(W.iid_u32(ns, seed=1), dev)
    dist = torch.from_numpy(W.dist_ids(ns, len(sizes), seed=2)).to(dev)
    idx = torch.empty(ns, dtype=torch.int32, device=dev)
    pos = torch.empty(ns, dtype=torch.float32, device=dev)
    api.rtf_sample(f, u, dist_id=dist, idx_out=idx, pos_out=pos)
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    for _ in range(reps):
        api.rtf_build_batched(w, sizes, ms, forest=f, plan_dev=f._plan_dev)
    b.record()
    torch.cuda.synchronize()
    f.check_status()
    batched_ms = a.elapsed_time(b) / reps
    # the same builds one distribution at a time through rtf_build
    lib = _native.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    goff = f.guide_offsets
    nmax = int(sizes.max())
    ws = api.workspace(lib.rtf_build_workspace_size(nmax, 1, 1 << int(ms.max())), dev, "build")
    structs = []
    for d in range(len(sizes)):
        cf = _native.RtfForestC(
            num_dists=1, flags=0, num_elems=int(sizes[d]), num_cells=1 << int(ms[d]),
            max_m=int(ms[d]), nodes=f.nodes.data_ptr() + 16 * int(off[d]),
            guide=f.guide.data_ptr() + 4 * int(goff[d]),
            dists=f.dists.data_ptr() + 64 * d, status=f.status.data_ptr(),
            guide_recs=f.guide_recs.data_ptr() + 32 * int(goff[d]))
        structs.append((ctypes.c_void_p(w.data_ptr() + 4 * int(off[d])), int(sizes[d]),
                        int(ms[d]), cf))
    wsp, wsn = ctypes.c_void_p(ws.data_ptr()), ws.numel()
    for wp, n, m, cf in structs[:64]:
        lib.rtf_build(wp, n, m, ctypes.byref(cf), wsp, wsn, stream)
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    for wp, n, m, cf in structs:
        rc = lib.rtf_build(wp, n, m, ctypes.byref(cf), wsp, wsn, stream)
        if rc:
            raise RuntimeError(f"rtf_build failed ({rc})")
    b.record()
    torch.cuda.synchronize()
    looped_ms = a.elapsed_time(b)
    # the tagged sampler's launch shape from the autotuner (timed on the first
    # 2^24 samples), then build + tagged sampling captured once and replayed
    f = api.rtf_build_batched(w, sizes, ms, forest=f, plan_dev=f._plan_dev)
    kind, shape, shape_ms = autotune.tune_launch_shape(f, u[:1 << 24], dist[:1 << 24],
                                                       use_cache=False)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream(dev)
    st.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            api.rtf_build_batched(w, sizes, ms, forest=f, plan_dev=f._plan_dev)
            api.rtf_sample(f, u, dist_id=dist, idx_out=idx, pos_out=pos)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    for _ in range(reps):
        g.replay()
    b.record()
    torch.cuda.synchronize()
    f.check_status()
    graph_ms = a.elapsed_time(b) / reps
    api.reset_launch_shape()
    N = int(off[-1])
    return {
        "workload": "16384 ragged distributions, n_d log-uniform in [8,65536] (sum %d), "
                    "lognormal(0,1.5), autotuned guide bits and launch shape, "
                    "2^27 tagged iid samples" % N,
        "launch_shape": {"kind": kind, "blocks_per_sm": shape,
                         "ms_per_2^24_samples": {str(k): v for k, v in shape_ms.items()}},
        "batched_build_ms": batched_ms, "looped_build_ms": looped_ms,
        "batched_over_looped": looped_ms / batched_ms,
        "build_elem_per_s": N / (batched_ms * 1e-3),
        "build_hbm_frac": (28 * N + 36 * int(goff[-1])) / (batched_ms * 1e-3) / 1e9 / measured_peaks()[0],
        "graph_build_plus_sample_ms": graph_ms,
        "samples_per_s_in_graph": ns / (graph_ms * 1e-3),
        "guide_bits_table": {str(k): int(v) for k, v in table.items()},
    }


def extra_env_map(dev, reps=3):
    """4096 x 2048 map: marginal + 2048 conditionals in one batched build;
    2^26 (u1, u2) pairs; guide bits of the rows and of the marginal from the
    autotuner (build + 2^26 pairs on this map)."""
    import torch
    from paper_1901_05423_gb300 import api, autotune
    from paper_1901_05423_gb300 import workloads as W
    H, Wd = 2048, 4096
    ns = 1 << 26
    lum = torch.from_numpy(W.env_map(H, Wd, seed=0).reshape(-1)).to(dev)
    m_row, m_marg, tuned = autotune.tune_env_bits(lum, H, Wd, ns)
    sizes = [Wd] * H + [H]
    ms = [m_row] * H + [m_marg]
    f = api.rtf_build_batched(lum, sizes, ms, marginal=True)
    u = api.u32_tensor(W.iid_u32(2 * ns, seed=3), dev)
    idx = torch.empty((ns, 2), dtype=torch.int32, device=dev)
    pos = torch.empty((ns, 2), dtype=torch.float32, device=dev)
    api.rtf_sample(f, u, mode=api.SAMPLE_2D, idx_out=idx, pos_out=pos)
    torch.cuda.synchronize()
    a, b = _events()
    c = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        api.rtf_build_batched(lum, sizes, ms, marginal=True, forest=f, plan_dev=f._plan_dev)
    b.record()
    for _ in range(reps):
        api.rtf_sample(f, u, mode=api.SAMPLE_2D, idx_out=idx, pos_out=pos)
    c.record()
    torch.cuda.synchronize()
    f.check_status()
    bms = a.elapsed_time(b) / reps
    sms = b.elapsed_time(c) / reps
    return {"workload": f"env map 4096x2048 + marginal, 2^{m_row} guide cells per row and "
                        f"2^{m_marg} for the marginal (autotuned), 2^26 iid (u1,u2) pairs",
            "guide_bits": {"row": m_row, "marginal": m_marg,
                           "tuned_ms_build_plus_2^26_pairs": {f"{a},{b}": v
                                                               for (a, b), v in tuned.items()}},
            "build_ms": bms, "build_elem_per_s": (H * Wd + H) / (bms * 1e-3),
            "build_hbm_frac": (28 * (H * Wd + H) + 36 * (H << m_row) + 36 * (1 << m_marg))
                              / (bms * 1e-3) / 1e9 / measured_peaks()[0],
            "sample_ms": sms, "samples_2d_per_s": ns / (sms * 1e-3),
            "sample_hbm_frac": 24 * ns / (sms * 1e-3) / 1e9 / measured_peaks()[0]}


def extra_backward(dev, reps=5):
    """n = 2^20 lognormal(0,1), 2^24 iid samples: forward (build + sample) vs
    backward (dL/dw from dL/dx ~ N(0,1))."""
    import torch
    from paper_1901_05423_gb300 import api
    from paper_1901_05423_gb300 import workloads as W
    n, m, ns = 1 << 20, 18, 1 << 24
    w = torch.from_numpy(W.lognormal_weights(n, seed=10, sigma=1.0)).to(dev)
    u = api.u32_tensor(W.iid_u32(ns, seed=11), dev)
    g = torch.from_numpy(W.normal_f32(ns, seed=12)).to(dev)
    f = api.rtf_build(w, m)
    idx, pos = api.rtf_sample(f, u)
    gw = api.rtf_sample_backward(f, w, u, None, idx, pos, g)
    torch.cuda.synchronize()
    a, b = _events()
    c = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        api.rtf_build(w, m, forest=f)
        api.rtf_sample(f, u, idx_out=idx, pos_out=pos)
    b.record()
    for _ in range(reps):
        api.rtf_sample_backward(f, w, u, None, idx, pos, g, grad_w=gw)
    c.record()
    torch.cuda.synchronize()
    f.check_status()
    fwd = a.elapsed_time(b) / reps
    bwd = b.elapsed_time(c) / reps
    return {"workload": "n=2^20 lognormal(0,1), 2^18 guide cells, 2^24 iid samples",
            "forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd}


def extra_methods(dev, reps=5):
    """The radix forest against the paper's comparator, the cutpoint method
    with binary search, and against 4-ary records (two levels collapsed, the
    section on k-ary trees), all on the same structure: the load statistics of
    Table 1 (maximum, average, average over groups of 32 of the group maximum)
    for its four densities at n = 1024 with 2^10 cells and 2^20 i.i.d.
    samples, and the three methods timed at n = 2^24, 2^20 cells on 2^26 i.i.d.
    and 2^26 sorted samples (bins and positions are identical)."""
    import torch
    from paper_1901_05423_gb300 import api
    from paper_1901_05423_gb300 import workloads as W
    methods = (("radix_forest", api.SAMPLE_1D), ("binary_search", api.SAMPLE_1D | api.SAMPLE_BSEARCH))

    def loads_of(f, quad, u):
        out = {name: api.load_statistics(api.rtf_sample_loads(f, u, mode=mode))
               for name, mode in methods}
        lq = torch.empty(u.numel(), dtype=torch.int32, device=dev)
        api.rtf_sample_quad(f, quad, u, loads_out=lq)
        out["quad_records"] = api.load_statistics(lq)
        return out

    table = {}
    u = api.u32_tensor(W.iid_u32(1 << 20, seed=5), dev)
    for kind in W.TABLE1_KINDS:
        f = api.rtf_build(torch.from_numpy(W.table1_weights(kind)).to(dev), 10)
        table[kind] = loads_of(f, api.rtf_build_quad(f), u)
        f.check_status()
    w = torch.from_numpy(W.lognormal_weights(N_W, seed=0, sigma=2.0)).to(dev)
    f = api.rtf_build(w, M_BITS)
    quad = api.rtf_build_quad(f)
    main_loads = loads_of(f, quad, u)
    a, b = _events()
    a.record()
    for _ in range(reps):
        api.rtf_build_quad(f, quad)
    b.record()
    torch.cuda.synchronize()
    times = {"build_quad_ms": a.elapsed_time(b) / reps}
    ns = 1 << 26
    for set_name, uh in (("iid", W.iid_u32(ns, seed=6)), ("sorted", W.sorted_radical_inverse_u32(ns))):
        ud = api.u32_tensor(uh, dev)
        idx = torch.empty(ns, dtype=torch.int32, device=dev)
        pos = torch.empty(ns, dtype=torch.float32, device=dev)
        hint = api.SAMPLE_COHERENT if set_name == "sorted" else 0
        runs = [(name, lambda mode=mode0 | hint: api.rtf_sample(f, ud, mode=mode, idx_out=idx,
                                                                 pos_out=pos))
                for name, mode0 in methods]
        runs.append(("quad_records", lambda: api.rtf_sample_quad(f, quad, ud, mode=api.SAMPLE_1D | hint,
                                                                 idx_out=idx, pos_out=pos)))
        for name, run in runs:
            run()
            torch.cuda.synchronize()
            a, b = _events()
            a.record()
            for _ in range(reps):
                run()
            b.record()
            torch.cuda.synchronize()
            times[f"{set_name}_{name}_ms"] = a.elapsed_time(b) / reps
        del ud, idx, pos
    f.check_status()
    return {"workload": "Table 1 densities (n=1024, 2^10 cells, 2^20 iid samples); "
                        "n=2^24 lognormal(0,2), 2^20 cells, 2^26 iid / sorted samples",
            "table1_loads": table, "n24_loads": main_loads, **times}


def profile_batched():
    """Profiling aid (no timing, no output line): the batched paths at a size an
    ncu capture of every pass can hold (about 1 GB on the device): a ragged
    batch of 4096 distributions (sizes log-uniform in [8, 65536], guide bits
    round(log2 n)) built three times and 2^25 tagged samples mapped twice; the
    2048 x 4096 map (2^12 cells per row and for the marginal) built and 2^24
    pairs mapped twice."""
    import torch
    from paper_1901_05423_gb300 import api
    from paper_1901_05423_gb300 import workloads as W
    dev = torch.device("cuda:0")
    w_h, off = W.ragged_batch(4096, seed=0)
    sizes = np.diff(off)
    ms = np.clip(np.round(np.log2(sizes)).astype(int), 3, 16)
    w = torch.from_numpy(w_h).to(dev)
    f = api.rtf_build_batched(w, sizes, ms)
    for _ in range(2):
        api.rtf_build_batched(w, sizes, ms, forest=f, plan_dev=f._plan_dev)
    ns = 1 << 25
    u = api.u32_tensor(W.iid_u32(ns, seed=1), dev)
    dist = torch.from_numpy(W.dist_ids(ns, len(sizes), seed=2)).to(dev)
    for _ in range(2):
        api.rtf_sample(f, u, dist_id=dist)
    H, Wd = 2048, 4096
    lum = torch.from_numpy(W.env_map(H, Wd, seed=0).reshape(-1)).to(dev)
    fe = api.rtf_build_batched(lum, [Wd] * H + [H], [12] * (H + 1), marginal=True)
    u2 = api.u32_tensor(W.iid_u32(2 * (1 << 24), seed=3), dev)
    for _ in range(2):
        api.rtf_sample(fe, u2, mode=api.SAMPLE_2D)
    torch.cuda.synchronize()
    f.check_status()
    fe.check_status()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rtf", choices=["rtf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ragged-batch, 2-D map and backward measurements")
    ap.add_argument("--streams", type=int, default=2, choices=[1, 2, 3],
                    help="2: sample the sorted set on a second stream, concurrently with the "
                         "i.i.d. set and the backward; 3: also accumulate the backward chunk by "
                         "chunk on a third stream while the i.i.d. set is mapped")
    ap.add_argument("--sorted-dense", action="store_true",
                    help="with --samples-log2 below 28: the sorted set at the full-size density "
                         "(u = 16 j), a profiling aid")
    ap.add_argument("--samples-log2", type=int, default=28,
                    help="2^k samples per set; the benchmarked workload is k = 28, smaller k "
                         "gives the same structure with fewer samples (profiler captures)")
    ap.add_argument("--profile-batched", action="store_true",
                    help="profiling aid: only the ragged batch (4096 distributions) and the "
                         "2-D map paths at a size an ncu capture holds; prints nothing")
    args = ap.parse_args()
    if args.profile_batched:
        return profile_batched()
    global N_S
    N_S = 1 << args.samples_log2
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
