"""Python binding of the C interface in include/rtf.h.

Argument marshalling only: tensors are checked (device, dtype, contiguity),
caller-side buffers and workspaces are allocated with torch, and every step of
the method runs inside ``librtf.so`` on the tensors' CUDA device and the
current torch stream.  The function names are those of the C interface.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _native

RTF_OK = 0
STATUS_BAD_WEIGHT = 0x1
STATUS_ZERO_TOTAL = 0x2
STATUS_TIMEOUT = 0x4
STATUS_BAD_PLAN = 0x8
STATUS_INVARIANT = 0x10
FOREST_MARGINAL = 0x1
SAMPLE_1D = 0
SAMPLE_2D = 1
SAMPLE_BSEARCH = 0x100  # flag: cutpoint method + binary search instead of the forest
SAMPLE_COHERENT = 0x200  # hint: neighbouring samples are close (sorted / low-discrepancy order)
NODE_BYTES = 16
GUIDE_REC_BYTES = 32
QUAD_REC_BYTES = 32
QUAD_FAR = 1 << 63  # bit of a 4-ary record's middle split: references too far for 16 bits
DIST_BYTES = 64

_workspaces: dict = {}


class RtfError(RuntimeError):
    pass


def _check(code: int, what: str):
    if code != RTF_OK:
        msg = _native.load().rtf_status_string(code).decode()
        raise RtfError(f"{what}: {msg} (code {code})")


def _stream_ptr(device: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _need(t: torch.Tensor, dtype: torch.dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise RtfError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise RtfError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise RtfError(f"{name} must be contiguous")


def workspace(nbytes: int, device: torch.device, tag: str) -> torch.Tensor:
    """A device workspace of at least `nbytes`, cached per device and tag."""
    key = (str(device), tag)
    ws = _workspaces.get(key)
    if ws is None or ws.numel() < nbytes:
        ws = torch.zeros(max(nbytes, 256), dtype=torch.uint8, device=device)
        _workspaces[key] = ws
    return ws


@dataclass
class Forest:
    """Device buffers of a forest plus the host-side sizes of rtf_forest."""
    num_dists: int
    flags: int
    num_elems: int
    num_cells: int
    max_m: int
    device: torch.device
    nodes: torch.Tensor = field(init=False)   # uint8 [N * 16]
    guide: torch.Tensor = field(init=False)   # int32 [G]
    guide_recs: torch.Tensor = field(init=False)   # uint8 [G * 32]
    dists: torch.Tensor = field(init=False)   # uint8 [D * 64]
    status: torch.Tensor = field(init=False)  # int32 [1]
    offsets: np.ndarray | None = None         # host copy of the element offsets
    guide_offsets: np.ndarray | None = None
    m: np.ndarray | None = None

    def __post_init__(self):
        dev = self.device
        self.nodes = torch.empty(self.num_elems * NODE_BYTES, dtype=torch.uint8, device=dev)
        self.guide = torch.empty(self.num_cells, dtype=torch.int32, device=dev)
        self.guide_recs = torch.empty(self.num_cells * GUIDE_REC_BYTES, dtype=torch.uint8,
                                      device=dev)
        self.dists = torch.empty(self.num_dists * DIST_BYTES, dtype=torch.uint8, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)

    def c_struct(self) -> _native.RtfForestC:
        return _native.RtfForestC(
            num_dists=self.num_dists, flags=self.flags, num_elems=self.num_elems,
            num_cells=self.num_cells, max_m=self.max_m, reserved=0,
            nodes=self.nodes.data_ptr(), guide=self.guide.data_ptr(),
            dists=self.dists.data_ptr(), status=self.status.data_ptr(),
            guide_recs=self.guide_recs.data_ptr())

    # views of the device structure (for tests and inspection)
    def cdf(self) -> torch.Tensor:
        """C_j of every record, int64 view of the uint64 values [N]."""
        return self.nodes.view(torch.int64).view(self.num_elems, 2)[:, 0]

    def guide_records(self) -> torch.Tensor:
        """guide records as int64 [G, 4]: cdf, packed children, lo, hi."""
        return self.guide_recs.view(torch.int64).view(self.num_cells, 4)

    def children(self) -> torch.Tensor:
        """child[0], child[1] of every record, int32 [N, 2]."""
        return self.nodes.view(torch.int32).view(self.num_elems, 4)[:, 2:4]

    def dist_table(self) -> torch.Tensor:
        """rtf_dist records as int64 [D, 8] (elem_off, n, guide_off, total,
        recip, (m, scale), (shift, flags), reserved)."""
        return self.dists.view(torch.int64).view(self.num_dists, 8)

    def check_status(self):
        s = int(self.status.item())
        if s:
            names = [n for b, n in ((STATUS_BAD_WEIGHT, "bad weight"),
                                    (STATUS_ZERO_TOTAL, "zero total"),
                                    (STATUS_TIMEOUT, "timeout"),
                                    (STATUS_BAD_PLAN, "bad plan"),
                                    (STATUS_INVARIANT, "internal bound exceeded")) if s & b]
            raise RtfError(f"device status {s:#x}: {', '.join(names)}")
        return 0


def rtf_build(w: torch.Tensor, m: int, forest: Forest | None = None) -> Forest:
    """Build the guide table and radix forest of one distribution (``rtf_build``)."""
    _need(w, torch.float32, "w")
    n = w.numel()
    if forest is None:
        forest = Forest(1, 0, n, 1 << m, m, w.device)
    lib = _native.load()
    nbytes = lib.rtf_build_workspace_size(n, 1, 1 << m)
    ws = workspace(nbytes, w.device, "build")
    cf = forest.c_struct()
    _check(lib.rtf_build(_ptr(w), n, m, ctypes.byref(cf), _ptr(ws), ws.numel(),
                         _stream_ptr(w.device)), "rtf_build")
    return forest


def rtf_build_static(w: torch.Tensor, m: int, forest: Forest | None = None) -> Forest:
    """``rtf_build_static``: the build of ``rtf_build`` with the library's own
    fixed scratch array (n <= 2^20, m <= 16) for callers that cannot allocate
    a workspace; calls that overlap on the GPU race on that array."""
    _need(w, torch.float32, "w")
    n = w.numel()
    if forest is None:
        forest = Forest(1, 0, n, 1 << m, m, w.device)
    cf = forest.c_struct()
    _check(_native.load().rtf_build_static(_ptr(w), n, m, ctypes.byref(cf),
                                           _stream_ptr(w.device)), "rtf_build_static")
    return forest


def plan_batched(sizes, m, marginal: bool = False):
    """Host-side plan: element offsets, guide offsets, total sizes."""
    sizes = np.asarray(sizes, dtype=np.int64)
    m = np.asarray(m, dtype=np.int32)
    D = sizes.size
    if m.size != D:
        raise RtfError("one guide size per distribution is needed")
    if np.any(sizes < 1) or np.any(m < 0) or np.any(m > 30):
        raise RtfError("n_d >= 1 and 0 <= m_d <= 30 are required")
    if marginal and sizes[-1] != D - 1:
        raise RtfError("the marginal needs one weight per row")
    offsets = np.zeros(D + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    goff = np.zeros(D + 1, np.int64)
    goff[1:] = np.cumsum(np.left_shift(np.int64(1), m.astype(np.int64)))
    return offsets, goff, m


def rtf_build_batched(w: torch.Tensor, sizes, m, marginal: bool = False,
                      forest: Forest | None = None, plan_dev=None) -> Forest:
    """Build many distributions in one pass (``rtf_build_batched``).

    `sizes` and `m` are host sequences (one entry per distribution).  With
    `marginal`, the last distribution is the marginal over the others: its size
    must be D - 1 and `w` holds only the rows' weights."""
    _need(w, torch.float32, "w")
    offsets, goff, mm = plan_batched(sizes, m, marginal)
    D = len(mm)
    N = int(offsets[-1])
    G = int(goff[-1])
    Nw = N - (D - 1) if marginal else N
    if w.numel() != Nw:
        raise RtfError(f"w has {w.numel()} weights, the plan needs {Nw}")
    dev = w.device
    if forest is None:
        forest = Forest(D, FOREST_MARGINAL if marginal else 0, N, G, int(mm.max()), dev)
    forest.offsets, forest.guide_offsets, forest.m = offsets, goff, mm
    if plan_dev is None:
        plan_dev = (torch.from_numpy(offsets).to(dev), torch.from_numpy(mm).to(dev),
                    torch.from_numpy(goff).to(dev))
    d_off, d_m, d_goff = plan_dev
    lib = _native.load()
    nbytes = lib.rtf_build_workspace_size(N, D, G)
    ws = workspace(nbytes, dev, "build")
    cf = forest.c_struct()
    _check(lib.rtf_build_batched(_ptr(w), _ptr(d_off), _ptr(d_m), _ptr(d_goff), ctypes.byref(cf),
                                 _ptr(ws), ws.numel(), _stream_ptr(dev)), "rtf_build_batched")
    forest._plan_dev = plan_dev  # keep the device plan alive with the forest
    return forest


def rtf_sample(forest: Forest, u: torch.Tensor, dist_id: torch.Tensor | None = None,
               mode: int = SAMPLE_1D, idx_out: torch.Tensor | None = None,
               pos_out: torch.Tensor | None = None):
    """Map uint32 samples (given as int32 or uint32 tensors) to (idx, pos)."""
    if u.dtype not in (torch.int32, torch.uint32):
        raise RtfError("u must hold 32-bit samples (int32 or uint32 tensor)")
    _need(u, u.dtype, "u")
    if dist_id is not None:
        _need(dist_id, torch.int32, "dist_id")
    two_d = (mode & 0xFF) == SAMPLE_2D
    count = u.numel() // (2 if two_d else 1)
    shape = (count, 2) if two_d else (count,)
    if idx_out is None:
        idx_out = torch.empty(shape, dtype=torch.int32, device=u.device)
    if pos_out is None:
        pos_out = torch.empty(shape, dtype=torch.float32, device=u.device)
    lib = _native.load()
    cf = forest.c_struct()
    _check(lib.rtf_sample(ctypes.byref(cf), _ptr(u), _ptr(dist_id), count, mode, _ptr(idx_out),
                          _ptr(pos_out), _stream_ptr(u.device)), "rtf_sample")
    return idx_out, pos_out


def rtf_sample_pipelined(forest: Forest, u_host: torch.Tensor | None, u_dev: torch.Tensor,
                         idx_dev: torch.Tensor, pos_dev: torch.Tensor,
                         idx_host: torch.Tensor | None = None, pos_host: torch.Tensor | None = None,
                         dist_id_host: torch.Tensor | None = None,
                         dist_id_dev: torch.Tensor | None = None, mode: int = SAMPLE_1D,
                         chunk: int = 1 << 22, done_event: torch.cuda.Event | None = None):
    """``rtf_sample_pipelined``: samples from host memory, results to device
    and (optionally) host memory, copies overlapping the sampling chunk by
    chunk.  Host tensors should be page-locked (``Tensor.pin_memory()``).
    With `done_event` the current stream does not wait for the copies back;
    the event marks their end."""
    for t, name in ((u_host, "u_host"), (idx_host, "idx_host"), (pos_host, "pos_host"),
                    (dist_id_host, "dist_id_host")):
        if t is not None and (t.is_cuda or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous host tensor")
    two_d = (mode & 0xFF) == SAMPLE_2D
    count = u_dev.numel() // (2 if two_d else 1)
    lib = _native.load()
    cf = forest.c_struct()
    ev = ctypes.c_void_p(0)
    if done_event is not None:
        if not done_event.cuda_event:  # torch creates the event at its first record
            done_event.record(torch.cuda.current_stream(u_dev.device))
        ev = ctypes.c_void_p(done_event.cuda_event)
    _check(lib.rtf_sample_pipelined(ctypes.byref(cf), _ptr(u_host), _ptr(u_dev), _ptr(dist_id_host),
                                    _ptr(dist_id_dev), count, mode, _ptr(idx_dev), _ptr(pos_dev),
                                    _ptr(idx_host), _ptr(pos_host), chunk, ev,
                                    _stream_ptr(u_dev.device)), "rtf_sample_pipelined")
    return idx_dev, pos_dev


def rtf_sample_loads(forest: Forest, u: torch.Tensor, dist_id: torch.Tensor | None = None,
                     mode: int = SAMPLE_1D) -> torch.Tensor:
    """Structure loads per sample under the method of `mode` (``rtf_sample_loads``)."""
    if u.dtype not in (torch.int32, torch.uint32):
        raise TypeError("u must hold uint32 bit patterns (int32 or uint32 tensor)")
    count = u.numel()
    loads = torch.empty(count, dtype=torch.int32, device=u.device)
    lib = _native.load()
    cf = forest.c_struct()
    _check(lib.rtf_sample_loads(ctypes.byref(cf), _ptr(u), _ptr(dist_id), count, mode,
                                _ptr(loads), _stream_ptr(u.device)), "rtf_sample_loads")
    return loads


def rtf_build_quad(forest: Forest, quad: torch.Tensor | None = None) -> torch.Tensor:
    """4-ary records of a built forest (``rtf_build_quad``): int64 [N, 4] per
    node j, {C_a, C_j (| QUAD_FAR), C_b, four 16-bit grandchild references}."""
    dev = forest.nodes.device
    if quad is None:
        quad = torch.empty((forest.num_elems, 4), dtype=torch.int64, device=dev)
    elif quad.shape != (forest.num_elems, 4) or quad.dtype != torch.int64:
        raise RtfError("quad must be int64 [num_elems, 4]")
    lib = _native.load()
    cf = forest.c_struct()
    _check(lib.rtf_build_quad(ctypes.byref(cf), _ptr(quad), _stream_ptr(dev)), "rtf_build_quad")
    return quad


def rtf_sample_quad(forest: Forest, quad: torch.Tensor, u: torch.Tensor,
                    dist_id: torch.Tensor | None = None, mode: int = SAMPLE_1D,
                    idx_out: torch.Tensor | None = None, pos_out: torch.Tensor | None = None,
                    loads_out: torch.Tensor | None = None):
    """rtf_sample through the 4-ary records (``rtf_sample_quad``); loads_out
    (int32, one per output) receives the structure loads of each sample."""
    if u.dtype not in (torch.int32, torch.uint32):
        raise RtfError("u must hold 32-bit samples (int32 or uint32 tensor)")
    _need(u, u.dtype, "u")
    _need(quad, torch.int64, "quad")
    if dist_id is not None:
        _need(dist_id, torch.int32, "dist_id")
    two_d = (mode & 0xFF) == SAMPLE_2D
    count = u.numel() // (2 if two_d else 1)
    shape = (count, 2) if two_d else (count,)
    if idx_out is None:
        idx_out = torch.empty(shape, dtype=torch.int32, device=u.device)
    if pos_out is None:
        pos_out = torch.empty(shape, dtype=torch.float32, device=u.device)
    if loads_out is not None:
        _need(loads_out, torch.int32, "loads_out")
    lib = _native.load()
    cf = forest.c_struct()
    _check(lib.rtf_sample_quad(ctypes.byref(cf), _ptr(quad), _ptr(u), _ptr(dist_id), count, mode,
                               _ptr(idx_out), _ptr(pos_out), _ptr(loads_out),
                               _stream_ptr(u.device)), "rtf_sample_quad")
    return idx_out, pos_out


LAUNCH_KINDS = ("single_large", "single", "tagged", "pairs")


def get_launch_shape() -> dict:
    """Blocks per SM of each kind of sampling launch (``rtf_get_launch_shape``)."""
    lib = _native.load()
    c = _native.RtfLaunchShapeC()
    _check(lib.rtf_get_launch_shape(ctypes.byref(c)), "rtf_get_launch_shape")
    return {k: int(getattr(c, k)) for k in LAUNCH_KINDS}


def set_launch_shape(**kinds) -> dict:
    """Set blocks per SM for some kinds (others keep their current value);
    returns the shape in effect (``rtf_set_launch_shape``)."""
    unknown = set(kinds) - set(LAUNCH_KINDS)
    if unknown:
        raise RtfError(f"unknown launch kinds {sorted(unknown)}")
    cur = get_launch_shape()
    cur.update({k: int(v) for k, v in kinds.items()})
    lib = _native.load()
    c = _native.RtfLaunchShapeC(**cur)
    _check(lib.rtf_set_launch_shape(ctypes.byref(c)), "rtf_set_launch_shape")
    return get_launch_shape()


def reset_launch_shape() -> dict:
    """Back to the built-in launch shape."""
    lib = _native.load()
    _check(lib.rtf_set_launch_shape(None), "rtf_set_launch_shape")
    return get_launch_shape()


def check_bounded_wait(device=None) -> int:
    """Run the library's bounded wait on a status word nothing publishes
    (``rtf_check_bounded_wait``); returns the status bits it raised (the
    wait gives up after about a second and sets STATUS_TIMEOUT)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    scratch = torch.zeros(2, dtype=torch.int64, device=dev)
    lib = _native.load()
    _check(lib.rtf_check_bounded_wait(_ptr(status), _ptr(scratch), _stream_ptr(dev)),
           "rtf_check_bounded_wait")
    return int(status.item())


def load_statistics(loads, group: int = 32) -> dict:
    """Maximum, average and average over consecutive groups of `group` samples
    of the group's maximum (the cost of samples that run in lockstep), the
    three columns of the paper's Table 1."""
    a = np.asarray(loads.cpu() if torch.is_tensor(loads) else loads, dtype=np.int64)
    if a.size == 0 or (a < 0).any():
        raise ValueError("load counts must be non-empty and non-negative")
    g = a[: a.size - a.size % group].reshape(-1, group) if a.size >= group else a.reshape(1, -1)
    return {"maximum": int(a.max()), "average": float(a.mean()),
            "average32": float(g.max(axis=1).mean())}


def rtf_sample_backward(forest: Forest, w: torch.Tensor, u: torch.Tensor,
                        dist_id: torch.Tensor | None, idx: torch.Tensor, pos: torch.Tensor,
                        grad_pos: torch.Tensor, mode: int = SAMPLE_1D,
                        grad_w: torch.Tensor | None = None) -> torch.Tensor:
    """dL/dw from dL/dpos (``rtf_sample_backward``)."""
    _need(w, torch.float32, "w")
    _need(grad_pos, torch.float32, "grad_pos")
    count = u.numel() // (2 if mode == SAMPLE_2D else 1)
    if grad_w is None:
        grad_w = torch.empty_like(w)
    lib = _native.load()
    nbytes = lib.rtf_backward_workspace_size(forest.num_elems, forest.num_dists)
    ws = workspace(nbytes, w.device, "backward")
    cf = forest.c_struct()
    _check(lib.rtf_sample_backward(ctypes.byref(cf), _ptr(w), _ptr(u), _ptr(dist_id), _ptr(idx),
                                   _ptr(pos), _ptr(grad_pos), count, mode, _ptr(grad_w),
                                   _ptr(ws), ws.numel(), _stream_ptr(w.device)),
           "rtf_sample_backward")
    return grad_w


class GradientAccumulator:
    """``rtf_backward_begin`` / ``_accumulate`` / ``_finish`` with a workspace of
    its own: dL/dw summed over any number of sample batches, each call on the
    current stream (the caller orders calls made on different streams)."""

    def __init__(self, forest: Forest, mode: int = SAMPLE_1D):
        self.forest = forest
        self.mode = mode
        self.lib = _native.load()
        nbytes = self.lib.rtf_backward_workspace_size(forest.num_elems, forest.num_dists)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=forest.device)
        self.cf = forest.c_struct()

    def begin(self):
        _check(self.lib.rtf_backward_begin(ctypes.byref(self.cf), _ptr(self.ws), self.ws.numel(),
                                           _stream_ptr(self.ws.device)), "rtf_backward_begin")
        return self

    def accumulate(self, idx: torch.Tensor, pos: torch.Tensor, grad_pos: torch.Tensor,
                   dist_id: torch.Tensor | None = None):
        _need(grad_pos, torch.float32, "grad_pos")
        count = pos.numel() // (2 if (self.mode & 0xFF) == SAMPLE_2D else 1)
        _check(self.lib.rtf_backward_accumulate(ctypes.byref(self.cf), _ptr(dist_id), _ptr(idx),
                                                _ptr(pos), _ptr(grad_pos), count, self.mode,
                                                _ptr(self.ws), self.ws.numel(),
                                                _stream_ptr(self.ws.device)),
               "rtf_backward_accumulate")

    def finish(self, w: torch.Tensor, grad_w: torch.Tensor | None = None) -> torch.Tensor:
        _need(w, torch.float32, "w")
        if grad_w is None:
            grad_w = torch.empty_like(w)
        _check(self.lib.rtf_backward_finish(ctypes.byref(self.cf), _ptr(w), self.mode,
                                            _ptr(grad_w), _ptr(self.ws), self.ws.numel(),
                                            _stream_ptr(self.ws.device)), "rtf_backward_finish")
        return grad_w


def u32_tensor(a: np.ndarray, device) -> torch.Tensor:
    """Host uint32 samples -> device int32 tensor holding the same bits."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).to(device)
