"""Python face of the CPU oracle (``oracle/rtf_oracle.cpp``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It never imports the
CUDA package and the CUDA package never imports it.

The oracle is a plain sequential statement of the method of Binder & Keller,
"Massively Parallel Construction of Radix Tree Forests for the Efficient
Sampling of Discrete or Piecewise Constant Probability Distributions":

* Sec. 1 (inverse CDF, P^{-1}(xi) = i <=> P_{i-1} <= xi < P_i) made exact by
  32-bit samples and an integer CDF (``scale``, ``quantize``, ``cdf``,
  ``index``, ``position``);
* Algorithm 1 run sequentially (``forest``), the guide table of the Cutpoint
  method with the two's complement encoding of Sec. 3.2 (``guide``);
* Algorithm 2 (``descend``), and over 4-ary records that collapse two binary
  levels (``quad``, ``descend_quad``; the section on k-ary trees);
* the 2-D component-wise scheme of Sec. 5 (``build_env``, ``sample_env``);
* the fp64 gradient of the in-bin position (``grad``, ``grad_env``; not in the
  paper): the gradient of the computed forward x = (xi T - C_i) / q_i with the
  floor of the quantisation passed straight through, i.e. the relaxation
  x = (xi W' - C'_i) / w'_i differentiated at the quantised weights
  w' = floor(w 2^S) 2^-S.

Each wrapper names the C function it calls; the citations are in the C file.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rtf_oracle.cpp")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
BAD_WEIGHT = 1
ZERO_TOTAL = 2


def compile_lib(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (plain g++)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(compile_lib())
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        sig = {
            "orc_scale": (ctypes.c_int, [P, i64, i64, P]),
            "orc_quantize": (None, [P, i64, i32, P]),
            "orc_cdf": (None, [P, i64, P]),
            "orc_index": (i64, [P, i64, ctypes.c_uint32]),
            "orc_position": (ctypes.c_double, [P, i64, ctypes.c_uint32, i64]),
            "orc_sample": (None, [P, i64, P, i64, P, P]),
            "orc_keys": (None, [P, i64, i64, P, P]),
            "orc_forest": (None, [P, P, i64, P]),
            "orc_guide": (None, [P, P, P, i64, i64, P]),
            "orc_descend": (i64, [P, P, P, i64, ctypes.c_uint32]),
            "orc_descend_steps": (i32, [P, P, P, i64, ctypes.c_uint32]),
            "orc_quad": (None, [P, i64, P, P]),
            "orc_descend_quad": (i64, [P, P, P, P, P, i64, ctypes.c_uint32, P]),
            "orc_build": (ctypes.c_int, [P, i64, i64, i64, P, P, P, P]),
            "orc_build_int": (ctypes.c_int, [P, i64, i64, P, P, P]),
            "orc_grad_q": (None, [P, i64, i32, P, P, P, i64, P]),
            "orc_quantized_weights": (None, [P, i64, i32, P]),
            "orc_grad64": (None, [P, i64, P, P, P, i64, P]),
            "orc_relaxed_position": (None, [P, i64, P, P, i64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(w):
    return np.ascontiguousarray(w, dtype=np.float32)


class OracleError(ValueError):
    pass


def scale(w, n_group: int | None = None) -> int:
    """``orc_scale``: exponent S of the fixed-point quantisation."""
    w = _f32(w)
    S = np.zeros(1, np.int32)
    st = _load().orc_scale(_p(w), w.size, n_group or w.size, _p(S))
    if st != OK:
        raise OracleError(f"oracle rejected the weights (status {st})")
    return int(S[0])


def quantize(w, S: int) -> np.ndarray:
    """``orc_quantize``: q_i = floor(w_i 2^S) as uint64."""
    w = _f32(w)
    q = np.zeros(w.size, np.uint64)
    _load().orc_quantize(_p(w), w.size, int(S), _p(q))
    return q


def cdf(q) -> np.ndarray:
    """``orc_cdf``: C[0] = 0, C[k+1] = C[k] + q[k]; C[n] = T."""
    q = np.ascontiguousarray(q, dtype=np.uint64)
    C = np.zeros(q.size + 1, np.uint64)
    _load().orc_cdf(_p(q), q.size, _p(C))
    return C


def keys(C, M: int):
    """``orc_keys``: K_j = ceil(C_j 2^32 / T) (uint64, K_n = 2^32) and cells."""
    C = np.ascontiguousarray(C, dtype=np.uint64)
    n = C.size - 1
    K = np.zeros(n + 1, np.uint64)
    cell = np.zeros(n, np.int64)
    _load().orc_keys(_p(C), n, int(M), _p(K), _p(cell))
    return K, cell


def index(C, u: int) -> int:
    C = np.ascontiguousarray(C, dtype=np.uint64)
    return int(_load().orc_index(_p(C), C.size - 1, int(u)))


def position(C, u: int, i: int) -> float:
    C = np.ascontiguousarray(C, dtype=np.uint64)
    return float(_load().orc_position(_p(C), C.size - 1, int(u), int(i)))


def sample(C, u, threads: int = 1):
    """``orc_sample``: (idx int32, pos fp64) for each uint32 sample.

    With ``threads`` > 1 the samples are cut into that many contiguous chunks,
    each mapped by one ``orc_sample`` call on its own thread (the samples are
    independent; ctypes releases the interpreter lock during the call)."""
    C = np.ascontiguousarray(C, dtype=np.uint64)
    u = np.ascontiguousarray(u, dtype=np.uint32)
    idx = np.zeros(u.size, np.int32)
    pos = np.zeros(u.size, np.float64)
    lib = _load()
    threads = max(1, min(int(threads), u.size // 4096 or 1))
    if threads == 1:
        lib.orc_sample(_p(C), C.size - 1, _p(u), u.size, _p(idx), _p(pos))
        return idx, pos
    cuts = np.linspace(0, u.size, threads + 1).astype(np.int64)

    def run(k):
        a, b = int(cuts[k]), int(cuts[k + 1])
        lib.orc_sample(_p(C), C.size - 1, _p(u[a:b]), b - a, _p(idx[a:b]), _p(pos[a:b]))

    pool = [threading.Thread(target=run, args=(k,)) for k in range(threads)]
    for t in pool:
        t.start()
    for t in pool:
        t.join()
    return idx, pos


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def forest(K, cell) -> np.ndarray:
    """``orc_forest`` (Algorithm 1, sequential): nodes int32[n, 2]."""
    K = np.ascontiguousarray(K, dtype=np.uint64)
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    n = cell.size
    nodes = np.zeros(2 * n, np.int32)
    _load().orc_forest(_p(K), _p(cell), n, _p(nodes))
    return nodes.reshape(n, 2)


def guide(C, K, cell, M: int) -> np.ndarray:
    """``orc_guide``: int32[M] guide table (root id, or ~i for one interval)."""
    C = np.ascontiguousarray(C, dtype=np.uint64)
    K = np.ascontiguousarray(K, dtype=np.uint64)
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    g = np.zeros(int(M), np.int32)
    _load().orc_guide(_p(C), _p(K), _p(cell), cell.size, int(M), _p(g))
    return g


def descend(guide_tab, nodes, K, M: int, u: int) -> int:
    """``orc_descend`` (Algorithm 2)."""
    g = np.ascontiguousarray(guide_tab, dtype=np.int32)
    nd = np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1)
    K = np.ascontiguousarray(K, dtype=np.uint64)
    return int(_load().orc_descend(_p(g), _p(nd), _p(K), int(M), int(u)))


def descend_steps(guide_tab, nodes, K, M: int, u: int) -> int:
    g = np.ascontiguousarray(guide_tab, dtype=np.int32)
    nd = np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1)
    K = np.ascontiguousarray(K, dtype=np.uint64)
    return int(_load().orc_descend_steps(_p(g), _p(nd), _p(K), int(M), int(u)))


def quad(nodes):
    """``orc_quad`` (two binary levels collapsed into one 4-ary record):
    split node ids int32[n, 3] and grandchildren int32[n, 4]."""
    nd = np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1)
    n = nd.size // 2
    split = np.zeros(3 * n, np.int32)
    child = np.zeros(4 * n, np.int32)
    _load().orc_quad(_p(nd), n, _p(split), _p(child))
    return split.reshape(n, 3), child.reshape(n, 4)


def descend_quad(guide_tab, nodes, split, child, K, M: int, u: int):
    """``orc_descend_quad``: (interval, 4-ary records read)."""
    g = np.ascontiguousarray(guide_tab, dtype=np.int32)
    nd = np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1)
    sp = np.ascontiguousarray(split, dtype=np.int32).reshape(-1)
    ch = np.ascontiguousarray(child, dtype=np.int32).reshape(-1)
    K = np.ascontiguousarray(K, dtype=np.uint64)
    r = np.zeros(1, np.int32)
    i = int(_load().orc_descend_quad(_p(g), _p(nd), _p(sp), _p(ch), _p(K), int(M), int(u), _p(r)))
    return i, int(r[0])


class Structure:
    """One distribution's auxiliary structure as the oracle builds it."""

    def __init__(self, S, C, nodes, guide_tab, M):
        self.S = S
        self.C = C
        self.nodes = nodes
        self.guide = guide_tab
        self.M = M

    @property
    def n(self):
        return self.C.size - 1

    @property
    def T(self):
        return int(self.C[-1])


def build(w, M: int, n_group: int | None = None) -> Structure:
    """``orc_build``: scale, quantise, CDF, keys, forest, guide (M cells)."""
    w = _f32(w)
    n = w.size
    S = np.zeros(1, np.int32)
    C = np.zeros(n + 1, np.uint64)
    nodes = np.zeros(2 * n, np.int32)
    g = np.zeros(int(M), np.int32)
    st = _load().orc_build(_p(w), n, n_group or n, int(M), _p(S), _p(C),
                           _p(nodes), _p(g))
    if st != OK:
        raise OracleError(f"oracle rejected the weights (status {st})")
    return Structure(int(S[0]), C, nodes.reshape(n, 2), g, int(M))


def build_int(q, M: int) -> Structure:
    """``orc_build_int``: build over exact integer weights (no quantisation)."""
    q = np.ascontiguousarray(q, dtype=np.uint64)
    n = q.size
    C = np.zeros(n + 1, np.uint64)
    nodes = np.zeros(2 * n, np.int32)
    g = np.zeros(int(M), np.int32)
    st = _load().orc_build_int(_p(q), n, int(M), _p(C), _p(nodes), _p(g))
    if st != OK:
        raise OracleError(f"oracle rejected the weights (status {st})")
    return Structure(None, C, nodes.reshape(n, 2), g, int(M))


def build_batched(w, offsets, M_per_dist) -> list[Structure]:
    """Independent distributions w[offsets[d]:offsets[d+1]], one scale each."""
    w = _f32(w)
    return [build(w[offsets[d]:offsets[d + 1]], int(M_per_dist[d]))
            for d in range(len(offsets) - 1)]


def build_env(lum, M_row: int, M_col: int):
    """2-D piecewise constant map (Sec. 5): one CDF per row and one over the
    rows.  All pixels share one scale (n_group = rows x cols); the marginal's
    weights are the exact integer row totals.  Returns (rows, marginal)."""
    lum = np.ascontiguousarray(lum, dtype=np.float32)
    H, W = lum.shape
    S = scale(lum.reshape(-1), n_group=H * W)
    rows = []
    totals = np.zeros(H, np.uint64)
    for r in range(H):
        q = quantize(lum[r], S)
        st = build_int(q, M_col)
        st.S = S
        rows.append(st)
        totals[r] = st.T
    marg = build_int(totals, M_row)
    marg.S = S
    return rows, marg


def sample_env(rows, marg, u1, u2):
    """Component-wise 2-D sampling (Sec. 5): the row from the marginal with u1,
    the column from that row's conditional with u2."""
    u1 = np.ascontiguousarray(u1, dtype=np.uint32)
    u2 = np.ascontiguousarray(u2, dtype=np.uint32)
    r, pr = sample(marg.C, u1)
    c = np.zeros_like(r)
    pc = np.zeros_like(pr)
    order = np.argsort(r, kind="stable")
    rs = r[order]
    bounds = np.searchsorted(rs, np.arange(len(rows) + 1))
    for row in np.unique(rs):
        sel = order[bounds[row]:bounds[row + 1]]
        ci, pi = sample(rows[row].C, u2[sel])
        c[sel] = ci
        pc[sel] = pi
    return r, c, pr, pc


def quantized_weights(w, S: int) -> np.ndarray:
    """``orc_quantized_weights``: w' = floor(w 2^S) 2^-S in fp64 (exact)."""
    w = _f32(w)
    out = np.zeros(w.size, np.float64)
    _load().orc_quantized_weights(_p(w), w.size, int(S), _p(out))
    return out


def grad_q(C, S: int, u, idx, gx) -> np.ndarray:
    """``orc_grad_q``: fp64 dL/dw of the positions of one distribution given by
    its integer CDF C[0..n] and scale S (the relaxation at w' = q 2^-S, with x
    from the exact integers)."""
    C = np.ascontiguousarray(C, dtype=np.uint64)
    u = np.ascontiguousarray(u, dtype=np.uint32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    gx = np.ascontiguousarray(gx, dtype=np.float32)
    n = C.size - 1
    out = np.zeros(n, np.float64)
    _load().orc_grad_q(_p(C), n, int(S), _p(u), _p(idx), _p(gx), u.size, _p(out))
    return out


def grad(w, u, idx, gx, n_group: int | None = None) -> np.ndarray:
    """fp64 dL/dw of the in-bin positions of one distribution (``orc_scale``,
    ``orc_quantize``, ``orc_cdf``, then ``orc_grad_q``)."""
    w = _f32(w)
    S = scale(w, n_group)
    return grad_q(cdf(quantize(w, S)), S, u, idx, gx)


def grad_env(lum, u1, u2, r, c, g_row, g_col) -> np.ndarray:
    """Gradient of the 2-D positions (Sec. 5, component-wise) with respect to
    the map: each row's column positions differentiate through that row's
    quantised weights; the row positions through the marginal, whose weights
    are the exact row totals T_r (in real units T_r 2^-S = sum_c w'(r, c)), so
    dL/dR_r is added to every weight of row r.  All pixels share one scale."""
    lum = np.ascontiguousarray(lum, dtype=np.float32)
    H, Wd = lum.shape
    S = scale(lum.reshape(-1), n_group=H * Wd)
    out = np.zeros((H, Wd), np.float64)
    Crows = [cdf(quantize(lum[r_], S)) for r_ in range(H)]
    totals = np.array([int(Cr[-1]) for Cr in Crows], np.uint64)
    gR = grad_q(cdf(totals), S, u1, r, g_row)
    out += gR[:, None]
    order = np.argsort(r, kind="stable")
    rs = r[order]
    bounds = np.searchsorted(rs, np.arange(H + 1))
    for row in np.unique(rs):
        sel = order[bounds[row]:bounds[row + 1]]
        out[row] += grad_q(Crows[row], S, u2[sel], c[sel], g_col[sel])
    return out


def relaxed_position(w64, u, idx) -> np.ndarray:
    """``orc_relaxed_position``: fp64 x = (xi W - C_i) / w_i at fixed bins."""
    w64 = np.ascontiguousarray(w64, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.uint32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    x = np.zeros(u.size, np.float64)
    _load().orc_relaxed_position(_p(w64), w64.size, _p(u), _p(idx), u.size,
                                 _p(x))
    return x
