"""Plain sequential CPU oracle (test infrastructure only).

The oracle restates, one definition at a time, what the GPU path computes
(arXiv 2409.03771: SoS vertex order, steepest pointers, path compression,
Morse-Smale cell ids, connected components).  It is plain C in
``msc_oracle.c``, compiled with gcc and called here through ctypes on numpy
arrays.  Only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import this package; the library never does.

Every wrapper raises ``OracleError`` on a non-zero return code:
-1 bad argument, -4 NaN in the field, -5 cycle (a walk never reached a fixed
point), -8 out of memory.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msc_oracle.c")
_LIB = os.path.join(_HERE, "libmsc_oracle.so")

ERR_ARG, ERR_NAN, ERR_CYCLE, ERR_OOM = -1, -4, -5, -8


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle (plain gcc, portable flags) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        sig = {
            "oracle_order": (i32, [P, i64, P]),
            "oracle_order_at": (i64, [P, i64, i64]),
            "oracle_steepest_grid": (i32, [P, i32, i32, i32, P, P]),
            "oracle_steepest_csr": (i32, [P, P, P, i32, P, P]),
            "oracle_steepest_at": (i32, [P, i32, i32, i32, i64, P, P]),
            "oracle_labels_at": (i32, [P, i32, i32, i32, i64, P, P]),
            "oracle_walk": (i32, [P, i64, P]),
            "oracle_walk_memo": (i32, [P, i64, P]),
            "oracle_jump_sync": (i32, [P, i64, P]),
            "oracle_ms": (i32, [P, P, i64, P, P]),
            "oracle_segment_grid": (i32, [P, i32, i32, i32, P, P, P, P, P]),
            "oracle_cc_grid": (i32, [P, i32, i32, i32, i32, P]),
            "oracle_cc_csr": (i32, [P, P, i32, P]),
            "oracle_cc_grid_at": (i32, [P, i32, i32, i32, i32, i64, P, P]),
            "oracle_adjacency_grid": (i32, [P, i32, i32, i32, i32, P, P, i64, P]),
            "oracle_extremum_graph": (i32, [P, P, i32, i32, i32, i32, i32, P, P, P, i64, P]),
            "oracle_adjacency_csr": (i32, [P, P, P, P, i32, i32, P, P, P, i64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _check(code: int, what: str) -> None:
    if code != 0:
        raise OracleError(int(code), what)


def order(f) -> np.ndarray:
    f = _c(f, np.float32).ravel()
    out = np.empty(f.size, np.int32)
    _check(_load().oracle_order(_ptr(f), f.size, _ptr(out)), "order")
    return out


def order_at(f, v: int) -> int:
    f = _c(f, np.float32).ravel()
    r = _load().oracle_order_at(_ptr(f), f.size, int(v))
    if r < 0:
        raise OracleError(int(r), "order_at")
    return int(r)


def steepest_grid(order_field, dims):
    nx, ny, nz = dims
    o = _c(order_field, np.int32).ravel()
    asc = np.empty(o.size, np.int32)
    desc = np.empty(o.size, np.int32)
    _check(_load().oracle_steepest_grid(_ptr(o), nx, ny, nz, _ptr(asc), _ptr(desc)), "steepest_grid")
    return asc, desc


def steepest_csr(order_field, row, col):
    o = _c(order_field, np.int32).ravel()
    row = _c(row, np.int32)
    col = _c(col, np.int32)
    n = row.size - 1
    asc = np.empty(n, np.int32)
    desc = np.empty(n, np.int32)
    _check(_load().oracle_steepest_csr(_ptr(o), _ptr(row), _ptr(col), n, _ptr(asc), _ptr(desc)), "steepest_csr")
    return asc, desc


def steepest_at(f, dims, v: int):
    nx, ny, nz = dims
    f = _c(f, np.float32).ravel()
    a, d = ctypes.c_int32(), ctypes.c_int32()
    _check(_load().oracle_steepest_at(_ptr(f), nx, ny, nz, int(v), ctypes.byref(a), ctypes.byref(d)), "steepest_at")
    return a.value, d.value


def labels_at(f, dims, v: int):
    nx, ny, nz = dims
    f = _c(f, np.float32).ravel()
    a, d = ctypes.c_int32(), ctypes.c_int32()
    _check(_load().oracle_labels_at(_ptr(f), nx, ny, nz, int(v), ctypes.byref(a), ctypes.byref(d)), "labels_at")
    return a.value, d.value


def walk(ptr) -> np.ndarray:
    p = _c(ptr, np.int32).ravel()
    out = np.empty(p.size, np.int32)
    _check(_load().oracle_walk(_ptr(p), p.size, _ptr(out)), "walk")
    return out


def walk_memo(ptr) -> np.ndarray:
    p = _c(ptr, np.int32).ravel()
    out = np.empty(p.size, np.int32)
    _check(_load().oracle_walk_memo(_ptr(p), p.size, _ptr(out)), "walk_memo")
    return out


def jump_sync(ptr) -> np.ndarray:
    p = _c(ptr, np.int32).ravel()
    out = np.empty(p.size, np.int32)
    _check(_load().oracle_jump_sync(_ptr(p), p.size, _ptr(out)), "jump_sync")
    return out


def ms(asc, desc):
    a = _c(asc, np.int32).ravel()
    d = _c(desc, np.int32).ravel()
    out = np.empty(a.size, np.int32)
    k = ctypes.c_int32()
    _check(_load().oracle_ms(_ptr(a), _ptr(d), a.size, _ptr(out), ctypes.byref(k)), "ms")
    return out, k.value


def segment_grid(f, dims):
    """order, asc label, desc label, ms id, number of cells."""
    nx, ny, nz = dims
    f = _c(f, np.float32).ravel()
    n = f.size
    order_ = np.empty(n, np.int32)
    asc = np.empty(n, np.int32)
    desc = np.empty(n, np.int32)
    ms_ = np.empty(n, np.int32)
    k = ctypes.c_int32()
    _check(
        _load().oracle_segment_grid(
            _ptr(f), nx, ny, nz, _ptr(order_), _ptr(asc), _ptr(desc), _ptr(ms_), ctypes.byref(k)
        ),
        "segment_grid",
    )
    return order_, asc, desc, ms_, k.value


def cc_grid(mask, dims, conn: int = 6) -> np.ndarray:
    nx, ny, nz = dims
    m = _c(mask, np.uint8).ravel()
    out = np.empty(m.size, np.int32)
    _check(_load().oracle_cc_grid(_ptr(m), nx, ny, nz, conn, _ptr(out)), "cc_grid")
    return out


def cc_csr(row, col) -> np.ndarray:
    row = _c(row, np.int32)
    col = _c(col, np.int32)
    n = row.size - 1
    out = np.empty(n, np.int32)
    _check(_load().oracle_cc_csr(_ptr(row), _ptr(col), n, _ptr(out)), "cc_csr")
    return out


def cc_grid_at(mask, dims, conn: int, v: int):
    """(smallest id of v's component or -1, component size)."""
    nx, ny, nz = dims
    m = _c(mask, np.uint8).ravel()
    mn, sz = ctypes.c_int32(), ctypes.c_int64()
    _check(
        _load().oracle_cc_grid_at(_ptr(m), nx, ny, nz, conn, int(v), ctypes.byref(mn), ctypes.byref(sz)),
        "cc_grid_at",
    )
    return mn.value, sz.value


def adjacency_grid(label, dims, conn: int = 14):
    """Distinct pairs (a, b), a < b, of different non-negative labels joined by
    an edge of the triangulation (conn 14) or of the face grid (conn 6),
    sorted: two int32 arrays."""
    nx, ny, nz = dims
    lab = _c(label, np.int32).ravel()
    cnt = ctypes.c_int64()
    _check(_load().oracle_adjacency_grid(_ptr(lab), nx, ny, nz, conn, 0, 0, 0, ctypes.byref(cnt)), "adjacency_grid")
    a = np.empty(max(cnt.value, 1), np.int32)
    b = np.empty(max(cnt.value, 1), np.int32)
    _check(_load().oracle_adjacency_grid(_ptr(lab), nx, ny, nz, conn, _ptr(a), _ptr(b), cnt.value,
                                         ctypes.byref(cnt)), "adjacency_grid")
    return a[:cnt.value], b[:cnt.value]


def extremum_graph(label, order, dims, conn: int = 14, sense: int = 1):
    """Arcs (a, b, saddle) of the extremum graph: pairs of different
    non-negative labels (maximum labels for sense +1, minimum labels for -1)
    that meet across an edge, in lexicographic order, each with the end
    vertex of its highest (maxima) or lowest (minima) crossing edge in the
    order: three int32 arrays."""
    nx, ny, nz = dims
    lab = _c(label, np.int32).ravel()
    o = _c(order, np.int32).ravel()
    cnt = ctypes.c_int64()
    _check(_load().oracle_extremum_graph(_ptr(lab), _ptr(o), nx, ny, nz, conn, sense, 0, 0, 0, 0,
                                         ctypes.byref(cnt)), "extremum_graph")
    k = cnt.value
    a, b, s = (np.empty(max(k, 1), np.int32) for _ in range(3))
    _check(_load().oracle_extremum_graph(_ptr(lab), _ptr(o), nx, ny, nz, conn, sense, _ptr(a), _ptr(b), _ptr(s), k,
                                         ctypes.byref(cnt)), "extremum_graph")
    return a[:k], b[:k], s[:k]


def adjacency_csr(label, row, col, order=None, sense: int = 1):
    """Over an explicit mesh (symmetric CSR): the distinct label pairs (a, b),
    a < b, across its edges, and with `order` also each pair's saddle (the
    crossing vertex of its highest (sense +1) or lowest (-1) edge).  Returns
    (a, b) or (a, b, saddle)."""
    lab = _c(label, np.int32).ravel()
    r = _c(row, np.int32).ravel()
    c = _c(col, np.int32).ravel() if np.asarray(col).size else np.zeros(1, np.int32)
    o = None if order is None else _c(order, np.int32).ravel()
    n = lab.size
    cnt = ctypes.c_int64()
    op = 0 if o is None else _ptr(o)
    _check(_load().oracle_adjacency_csr(_ptr(lab), op, _ptr(r), _ptr(c), n, sense, 0, 0, 0, 0, ctypes.byref(cnt)),
           "adjacency_csr")
    k = cnt.value
    a, b, s = (np.empty(max(k, 1), np.int32) for _ in range(3))
    _check(_load().oracle_adjacency_csr(_ptr(lab), op, _ptr(r), _ptr(c), n, sense, _ptr(a), _ptr(b), _ptr(s), k,
                                        ctypes.byref(cnt)), "adjacency_csr")
    return (a[:k], b[:k]) if o is None else (a[:k], b[:k], s[:k])
