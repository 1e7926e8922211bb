"""Host FP64 block-sparse Chebyshev recurrence (o2_recurrence.c) -- oracle, test and baseline
only.

A plain C/OpenMP implementation of Eq. poly_PQ (S = I) on the block-sparse H and the probe moments
of Sec. II.C.2, written independently of the CUDA library: the full-size parity check of the
moments where no dense oracle fits, and the CPU recurrence baseline of the benchmark (the same
work per moment as the GPU path, in the same unit).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "o2_recurrence.c")
LIB = os.path.join(HERE, "libo2.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libo2.so with gcc (-O3, OpenMP) next to its source."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.o2_moments.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                    C.c_double, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_void_p]
        _lib.o2_moments.restype = C.c_int
    return _lib


def moments(row_ptr, col, blocks, emin, emax, seed, s, order, doubled=False):
    """(moments (order,), block products run) of s probes on the BSR H (blocks: nnzb x B x B)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(blocks, dtype=np.float64)
    B = val.shape[-1]
    out = np.zeros(order)
    n = _load().o2_moments(len(rp) - 1, B, rp.ctypes.data, cl.ctypes.data, val.ctypes.data, float(emin),
                           float(emax), C.c_uint64(int(seed)), int(s), int(order), int(doubled),
                           out.ctypes.data)
    if n < 0:
        raise ValueError("o2_moments: bad arguments")
    return out, n
