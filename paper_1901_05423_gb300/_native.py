"""Build and load the CUDA library ``librtf.so`` (sm_103a).

The library is compiled in-tree with nvcc (one translation unit per file of
``csrc/``, compiled in parallel, then linked as a shared object).  Loading
fails loudly when the library is missing or cannot be built: there is no CPU
fallback anywhere in this package.
"""

from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
_OUT_DIR = os.path.join(_PKG, "_lib")
LIB_PATH = os.path.join(_OUT_DIR, "librtf.so")
SOURCES = ["build.cu", "sample.cu", "backward.cu", "api.cu", "static_ws.cu", "pipeline.cu",
           "quad.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the rtf CUDA library cannot be built")
    return cand


def _deps():
    files = [os.path.join(_CSRC, s) for s in SOURCES]
    files += [os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith(".cuh")]
    files += [os.path.join(_INCLUDE, "rtf.h"), os.path.abspath(__file__)]
    return files


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile ``csrc/*.cu`` for sm_103a into ``_lib/librtf.so``."""
    with _lock:
        if not force and not _stale():
            return LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        nvcc = _nvcc()
        common = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                  "-I", _INCLUDE, "-I", _CSRC]
        if verbose:
            common += ["-Xptxas", "-v"]

        def compile_one(src):
            obj = os.path.join(_OUT_DIR, os.path.splitext(src)[0] + ".o")
            cmd = common + ["-c", os.path.join(_CSRC, src), "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
            return obj, r.stderr

        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            results = list(ex.map(compile_one, SOURCES))
        objs = [o for o, _ in results]
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc, ARCH, "-shared", "-o", tmp] + objs,
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
        os.replace(tmp, LIB_PATH)
        if verbose:
            for _, log in results:
                print(log)
        return LIB_PATH


class RtfForestC(ctypes.Structure):
    """Mirror of ``rtf_forest`` in include/rtf.h (72 bytes)."""
    _fields_ = [
        ("num_dists", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("num_elems", ctypes.c_int64),
        ("num_cells", ctypes.c_int64),
        ("max_m", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("nodes", ctypes.c_void_p),
        ("guide", ctypes.c_void_p),
        ("dists", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
        ("guide_recs", ctypes.c_void_p),
    ]


class RtfLaunchShapeC(ctypes.Structure):
    """Mirror of ``rtf_launch_shape`` in include/rtf.h (16 bytes)."""
    _fields_ = [("single_large", ctypes.c_int32), ("single", ctypes.c_int32),
                ("tagged", ctypes.c_int32), ("pairs", ctypes.c_int32)]


EXPORTS = {
    # name: (restype, argtypes)
    "rtf_version": (ctypes.c_char_p, []),
    "rtf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rtf_build_workspace_size": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64]),
    "rtf_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                 ctypes.POINTER(RtfForestC), ctypes.c_void_p, ctypes.c_size_t,
                                 ctypes.c_void_p]),
    "rtf_build_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.POINTER(RtfForestC), ctypes.c_void_p]),
    "rtf_build_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(RtfForestC),
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "rtf_sample": (ctypes.c_int, [ctypes.POINTER(RtfForestC), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p]),
    "rtf_sample_pipelined": (ctypes.c_int, [ctypes.POINTER(RtfForestC)] + [ctypes.c_void_p] * 4
                             + [ctypes.c_int64, ctypes.c_int32] + [ctypes.c_void_p] * 4
                             + [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "rtf_sample_loads": (ctypes.c_int, [ctypes.POINTER(RtfForestC), ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "rtf_build_quad": (ctypes.c_int, [ctypes.POINTER(RtfForestC), ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "rtf_sample_quad": (ctypes.c_int, [ctypes.POINTER(RtfForestC), ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "rtf_check_bounded_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "rtf_set_launch_shape": (ctypes.c_int, [ctypes.POINTER(RtfLaunchShapeC)]),
    "rtf_get_launch_shape": (ctypes.c_int, [ctypes.POINTER(RtfLaunchShapeC)]),
    "rtf_backward_begin": (ctypes.c_int, [ctypes.POINTER(RtfForestC), ctypes.c_void_p,
                                          ctypes.c_size_t, ctypes.c_void_p]),
    "rtf_backward_accumulate": (ctypes.c_int, [ctypes.POINTER(RtfForestC)] + [ctypes.c_void_p] * 4
                                + [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                   ctypes.c_size_t, ctypes.c_void_p]),
    "rtf_backward_finish": (ctypes.c_int, [ctypes.POINTER(RtfForestC), ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_void_p]),
    "rtf_backward_workspace_size": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int32]),
    "rtf_sample_backward": (ctypes.c_int, [ctypes.POINTER(RtfForestC), ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_void_p]),
}


def load(build_if_needed: bool = True):
    """Load ``librtf.so`` (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"rtf CUDA library missing: {LIB_PATH}")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
