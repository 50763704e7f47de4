"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

Holds none of the method's arithmetic: it draws R-MAT edge lists (sorted by
(dst, src), self-loops and duplicates removed), Zipf benefit weights and
uniform variates for arrival processes.  The C source is compiled on first use
(or by ``build()``) into ``inputs/libssa_inputs.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmat.c")
_LIB = os.path.join(_HERE, "libssa_inputs.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator with gcc (host code, same flags on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.rmat_generate.restype = ctypes.c_int64
        lib.rmat_generate.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p]
        lib.zipf_weights.restype = ctypes.c_int
        lib.zipf_weights.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p]
        lib.uniform_doubles.restype = None
        lib.uniform_doubles.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass
class EdgeList:
    n: int
    src: np.ndarray  # int32, sorted by (dst, src)
    dst: np.ndarray  # int32

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def rmat(scale: int, m_draw: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, threads: int | None = None) -> EdgeList:
    """Directed R-MAT graph on 2**scale nodes from m_draw draws (unique edges kept)."""
    lib = _load()
    threads = threads or min(64, os.cpu_count() or 1)
    src = np.empty(max(m_draw, 1), dtype=np.int32)
    dst = np.empty(max(m_draw, 1), dtype=np.int32)
    m = lib.rmat_generate(scale, m_draw, a, b, c, seed & 0xFFFFFFFFFFFFFFFF, threads,
                          src.ctypes.data, dst.ctypes.data)
    if m < 0:
        raise RuntimeError("rmat_generate failed")
    return EdgeList(n=1 << scale, src=src[:m].copy(), dst=dst[:m].copy())


def zipf_benefit(n: int, s: float = 1.2, seed: int = 1) -> np.ndarray:
    """uint32 benefit weights max(1, floor(2^20 / rank^s)), ranks a keyed permutation."""
    lib = _load()
    w = np.empty(max(n, 1), dtype=np.uint32)
    if lib.zipf_weights(n, s, seed & 0xFFFFFFFFFFFFFFFF, w.ctypes.data) != 0:
        raise RuntimeError("zipf_weights failed")
    return w[:n].copy()


def uniforms(count: int, seed: int) -> np.ndarray:
    """count uniform doubles in [0,1) keyed by seed."""
    lib = _load()
    out = np.empty(max(count, 1), dtype=np.float64)
    lib.uniform_doubles(seed & 0xFFFFFFFFFFFFFFFF, count, out.ctypes.data)
    return out[:count].copy()


def edges(n: int, pairs) -> EdgeList:
    """Hand-written edge list (tests): pairs of (src, dst), kept as given."""
    arr = np.asarray(list(pairs), dtype=np.int64).reshape(-1, 2)
    return EdgeList(n=n, src=arr[:, 0].astype(np.int32), dst=arr[:, 1].astype(np.int32))
