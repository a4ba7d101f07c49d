"""CPU oracle for the FNR impulse filter (arXiv 1201.3972, Sec. 3.3-3.4).

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA library is
checked against. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package; the library itself never
does, and the two share no code.

The arithmetic lives in ``fnr_oracle.c`` (plain C, compiled with gcc on first
use). This module only marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fnr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_fnr.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, portable flags). Returns its path."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-Wall", "-Wextra",
                   "-o", tmp, _SRC]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        path = build()
        lib = ctypes.CDLL(path)
        vp, ll, i32 = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int
        lib.oracle_fnr.argtypes = [vp, ll, vp, ll, i32, i32, i32, i32]
        lib.oracle_fnr.restype = ll
        lib.oracle_fnr_mt.argtypes = [vp, ll, vp, ll, i32, i32, i32, i32, i32]
        lib.oracle_fnr_mt.restype = ll
        lib.oracle_fnr_stack.argtypes = [vp, vp, ll, i32, i32, i32, i32, i32]
        lib.oracle_fnr_stack.restype = ll
        lib.oracle_fnr_border.argtypes = [vp, ll, vp, ll, i32, i32, i32, i32, i32]
        lib.oracle_fnr_border.restype = ll
        lib.oracle_fnr_directional.argtypes = [vp, ll, vp, ll, i32, i32, i32, i32, i32]
        lib.oracle_fnr_directional.restype = ll
        lib.oracle_median_filter.argtypes = [vp, ll, vp, ll, i32, i32, i32, i32]
        lib.oracle_median_filter.restype = ll
        lib.oracle_introsort.argtypes = [vp, ctypes.c_long, i32]
        lib.oracle_introsort.restype = None
        _lib = lib
    return _lib


def _check_frame(frame: np.ndarray) -> int:
    if frame.ndim != 2:
        raise ValueError("frame must be 2-D (H, W)")
    if frame.dtype not in (np.uint8, np.uint16):
        raise TypeError("frame must be uint8 or uint16")
    if frame.strides[1] != frame.itemsize or frame.strides[0] < frame.shape[1] * frame.itemsize:
        raise ValueError("frame rows must be contiguous with a non-negative row pitch")
    return frame.itemsize


def fnr(frame: np.ndarray, k: int):
    """One FNR pass with window k. Returns (filtered frame, flagged count)."""
    lib = _load()
    es = _check_frame(frame)
    out = np.empty(frame.shape, dtype=frame.dtype)
    H, W = frame.shape
    f = lib.oracle_fnr(frame.ctypes.data, frame.strides[0], out.ctypes.data, out.strides[0],
                       H, W, es, int(k))
    if f < 0:
        raise ValueError(f"oracle rejected arguments (H={H}, W={W}, k={k})")
    return out, int(f)


BORDERS = {"replicate": 0, "mirror": 1, "zero": 2}


def fnr_border(frame: np.ndarray, k: int, border: str):
    """FNR with a border reading: "replicate" (default elsewhere), "mirror"
    (reflect without repeating the edge pixel) or "zero"."""
    lib = _load()
    es = _check_frame(frame)
    out = np.empty(frame.shape, dtype=frame.dtype)
    H, W = frame.shape
    f = lib.oracle_fnr_border(frame.ctypes.data, frame.strides[0], out.ctypes.data, out.strides[0],
                              H, W, es, int(k), BORDERS[border])
    if f < 0:
        raise ValueError("oracle rejected arguments")
    return out, int(f)


def fnr_directional(frame: np.ndarray, k: int, border: str = "replicate"):
    """FNR with the directional detector (Fig. 1): a pixel is noisy iff along
    none of the four lines through it (horizontal, vertical, two diagonals)
    it lies strictly between its two neighbours; noisy pixels take the k x k
    window median. Returns (filtered frame, flagged count)."""
    lib = _load()
    es = _check_frame(frame)
    out = np.empty(frame.shape, dtype=frame.dtype)
    H, W = frame.shape
    f = lib.oracle_fnr_directional(frame.ctypes.data, frame.strides[0], out.ctypes.data, out.strides[0],
                                   H, W, es, int(k), BORDERS[border])
    if f < 0:
        raise ValueError("oracle rejected arguments")
    return out, int(f)


def fnr_mt(frame: np.ndarray, k: int, threads: int):
    """Same result as :func:`fnr`, rows split across ``threads`` host threads."""
    lib = _load()
    es = _check_frame(frame)
    out = np.empty(frame.shape, dtype=frame.dtype)
    H, W = frame.shape
    f = lib.oracle_fnr_mt(frame.ctypes.data, frame.strides[0], out.ctypes.data, out.strides[0],
                          H, W, es, int(k), int(threads))
    if f < 0:
        raise ValueError("oracle rejected arguments")
    return out, int(f)


def fnr_stack(frames: np.ndarray, k: int):
    """Filter every frame of a contiguous (count, H, W) stack independently.
    Returns (outputs, total flagged count)."""
    lib = _load()
    frames = np.ascontiguousarray(frames)
    if frames.ndim != 3 or frames.dtype not in (np.uint8, np.uint16):
        raise ValueError("expected a (count, H, W) uint8/uint16 stack")
    c, H, W = frames.shape
    out = np.empty_like(frames)
    f = lib.oracle_fnr_stack(frames.ctypes.data, out.ctypes.data, W * frames.itemsize, c, H, W,
                             frames.itemsize, int(k))
    if f < 0:
        raise ValueError("oracle rejected arguments")
    return out, int(f)


def median_filter(frame: np.ndarray, k: int):
    """The standard median filter (Sec. 2, Table 1 "MF"): every pixel takes its
    window median. Returns (filtered frame, number of medians)."""
    lib = _load()
    es = _check_frame(frame)
    out = np.empty(frame.shape, dtype=frame.dtype)
    H, W = frame.shape
    f = lib.oracle_median_filter(frame.ctypes.data, frame.strides[0], out.ctypes.data, out.strides[0],
                                 H, W, es, int(k))
    if f < 0:
        raise ValueError("oracle rejected arguments")
    return out, int(f)


def fnr_passes(frame: np.ndarray, k: int, passes: int, threads: int = 1):
    """Iterative FNR (Figs. 3-6 use two passes): each pass filters the previous
    pass's output. Returns (final frame, flagged count of every pass)."""
    counts = []
    cur = frame
    for _ in range(int(passes)):
        cur, f = fnr_mt(cur, k, threads) if threads > 1 else fnr(cur, k)
        counts.append(f)
    return cur, counts


def introsort(values, depth_limit: int = -1) -> np.ndarray:
    """Sort a copy of ``values`` with the oracle's introsort (Sec. 3.4).
    depth_limit=-1 uses 2*floor(log2 n); 0 forces the heapsort fallback."""
    lib = _load()
    a = np.ascontiguousarray(np.asarray(values, dtype=np.uint32)).copy()
    lib.oracle_introsort(a.ctypes.data, a.size, int(depth_limit))
    return a


def median(values) -> int:
    """Element of rank (n-1)//2 of the introsorted values (odd n)."""
    a = introsort(values)
    return int(a[(a.size - 1) // 2])
