"""CPU baseline: the paper's shared-memory method (Alg. 1 path compression
with per-thread active lists, Alg. 3 connected components) on all host
cores with OpenMP, in ``paper_omp.c``.

Test and benchmark infrastructure only, and not the oracle: the tests check
it against the oracle, and the benchmark's CPU-baseline leg times it.  The
library never loads it.  ``threads`` is the number of OpenMP threads the
calls use (``OMP_NUM_THREADS`` or all cores by default).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paper_omp.c")
_LIB = os.path.join(_HERE, "libmsc_paper_omp.so")


class BaselineError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"OpenMP baseline {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "po_threads": (ctypes.c_int, []),
            "po_order": (ctypes.c_int, [P, i64, P]),
            "po_steepest_grid": (ctypes.c_int, [P, i32, i32, i32, P, P]),
            "po_compress": (None, [P, i64]),
            "po_ms": (ctypes.c_int, [P, P, i64, P, P]),
            "po_segment_grid": (ctypes.c_int, [P, i32, i32, i32, P, P, P, P, P, P]),
            "po_cc_grid": (ctypes.c_int, [P, i32, i32, i32, i32, P]),
            "po_cc_csr": (ctypes.c_int, [P, P, i32, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().po_threads())


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _check(code: int, what: str) -> None:
    if code != 0:
        raise BaselineError(int(code), what)


def order(f) -> np.ndarray:
    f = _c(f, np.float32).ravel()
    out = np.empty(f.size, np.int32)
    _check(_load().po_order(f.ctypes.data, f.size, out.ctypes.data), "order")
    return out


def compress(ptr) -> np.ndarray:
    p = _c(ptr, np.int32).ravel().copy()
    _load().po_compress(p.ctypes.data, p.size)
    return p


def segment_grid(f, dims):
    """(order, asc, desc, ms, num_cells, seconds per stage: order, steepest,
    compression, cell ids)."""
    nx, ny, nz = dims
    f = _c(f, np.float32).ravel()
    n = f.size
    outs = [np.empty(n, np.int32) for _ in range(4)]
    k = ctypes.c_int32()
    secs = (ctypes.c_double * 4)()
    _check(_load().po_segment_grid(f.ctypes.data, nx, ny, nz, *[o.ctypes.data for o in outs], ctypes.byref(k), secs),
           "segment_grid")
    return (*outs, k.value, list(secs))


def cc_grid(mask, dims, conn: int = 6) -> np.ndarray:
    nx, ny, nz = dims
    m = _c(mask, np.uint8).ravel()
    out = np.empty(m.size, np.int32)
    _check(_load().po_cc_grid(m.ctypes.data, nx, ny, nz, conn, out.ctypes.data), "cc_grid")
    return out


def cc_csr(row, col) -> np.ndarray:
    row = _c(row, np.int32)
    col = _c(col, np.int32) if np.asarray(col).size else np.zeros(1, np.int32)
    n = row.size - 1
    out = np.empty(max(n, 1), np.int32)
    _check(_load().po_cc_csr(row.ctypes.data, col.ctypes.data, n, out.ctypes.data), "cc_csr")
    return out[:n]
