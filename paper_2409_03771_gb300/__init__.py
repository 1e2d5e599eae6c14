"""Python binding of libmsc (include/msc.h): Morse-Smale segmentation and
connected components by path compression on one GB300 GPU.

Two layers, both argument marshalling only -- every step runs in the CUDA
kernels of libmsc.so:

* ``msc_*`` functions mirror the C ABI one to one: torch CUDA tensors in,
  raw device pointers and the current torch stream passed down, the C
  status code returned.
* ``order``, ``steepest_grid``, ``steepest_csr``, ``compress``, ``ms_id``,
  ``segment``, ``cc_mask``, ``cc_mesh`` allocate outputs and workspace with
  torch on the input's device, call the C ABI, synchronise and raise
  ``MSCError`` on any host or device error.

There is no CPU fallback: if libmsc.so is missing or no CUDA device is
present, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

__all__ = [
    "MSCError", "load", "lib_path",
    "msc_workspace_bytes", "msc_status_string", "msc_order", "msc_steepest_grid", "msc_steepest_csr",
    "msc_compress", "msc_compress_noalloc", "msc_ms_id", "msc_segment", "msc_cc_mask", "msc_cc_mesh",
    "order", "steepest_grid", "steepest_csr", "compress", "ms_id", "segment", "cc_mask", "cc_mesh",
    "OP_ORDER", "OP_COMPRESS", "OP_MS_ID", "OP_SEGMENT", "OP_CC_MASK", "OP_CC_MESH",
    "msc_launch_count", "msc_trace_enable", "msc_trace_reset", "msc_trace_collect",
    "Tune", "msc_batch_workspace_bytes", "msc_batch_segment", "msc_batch_plan_create", "msc_batch_plan_launch",
    "msc_batch_plan_kernels", "msc_batch_plan_destroy", "msc_batch_autotune", "Batch",
    "Job", "Result", "JOB_SEGMENT", "JOB_CC_MASK", "msc_server_create", "msc_server_submit", "msc_server_poll",
    "msc_server_wait", "msc_server_release", "msc_server_stats", "msc_server_destroy", "Server",
    "OP_ADJACENCY", "msc_adjacency_grid", "adjacency_grid", "OP_EXTREMUM_GRAPH", "msc_extremum_graph",
    "extremum_graph", "OP_ADJACENCY_CSR", "OP_EXTREMUM_GRAPH_CSR", "msc_adjacency_csr", "msc_extremum_graph_csr",
    "adjacency_csr", "extremum_graph_csr",
]

OK, ERR_ARG, ERR_WS, ERR_CUDA, ERR_NAN, ERR_NOT_CONVERGED, ERR_BUDGET, ERR_INTERNAL = 0, -1, -2, -3, -4, -5, -6, -7
ERR_TOO_LARGE = -8
NOALLOC_MAX_N = 1 << 22
PENDING = 1
OP_ORDER, OP_COMPRESS, OP_MS_ID, OP_SEGMENT, OP_CC_MASK, OP_CC_MESH, OP_ADJACENCY = 1, 2, 3, 4, 5, 6, 7
OP_EXTREMUM_GRAPH, OP_ADJACENCY_CSR, OP_EXTREMUM_GRAPH_CSR = 8, 9, 10
JOB_SEGMENT, JOB_CC_MASK = 1, 2


class MSCError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {msc_status_string(code)} ({code})")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class Tune(ctypes.Structure):
    """msc_tune: steepest_shape (-1 = tuned/default, 0..3), build_shift (0 = tuned/default, 1..30)."""
    _fields_ = [("steepest_shape", ctypes.c_int32), ("build_shift", ctypes.c_int32)]


class Job(ctypes.Structure):
    """msc_job: one served request."""
    _fields_ = [("kind", ctypes.c_int32), ("g", Grid), ("conn", ctypes.c_int32), ("input", ctypes.c_void_p)]


class Result(ctypes.Structure):
    """msc_result: a served request's state and device outputs."""
    _fields_ = [("status", ctypes.c_int32), ("num_cells", ctypes.c_int32), ("n", ctypes.c_int64),
                ("order", ctypes.c_void_p), ("asc", ctypes.c_void_p), ("desc", ctypes.c_void_p),
                ("ms", ctypes.c_void_p), ("label", ctypes.c_void_p), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double), ("group_size", ctypes.c_int32)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libmsc.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"libmsc.so is not built ({_build.LIB}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "msc_workspace_bytes": (SZ, [ctypes.c_int, I64, I64]),
        "msc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "msc_order": (ctypes.c_int, [P, I64, P, P, SZ, P, P]),
        "msc_steepest_grid": (ctypes.c_int, [P, Grid, P, P, P]),
        "msc_steepest_csr": (ctypes.c_int, [P, P, P, I32, P, P, P, P]),
        "msc_compress": (ctypes.c_int, [P, I32, P, SZ, P, P]),
        "msc_compress_noalloc": (ctypes.c_int, [P, I32, P, P]),
        "msc_ms_id": (ctypes.c_int, [P, P, I32, P, P, P, SZ, P, P]),
        "msc_segment": (ctypes.c_int, [P, Grid, P, P, P, P, P, P, SZ, P, P]),
        "msc_cc_mask": (ctypes.c_int, [P, Grid, I32, P, P, SZ, P, P]),
        "msc_cc_mesh": (ctypes.c_int, [P, P, I32, P, P, SZ, P, P]),
        "msc_adjacency_grid": (ctypes.c_int, [P, Grid, I32, I32, P, P, I64, P, P, SZ, P, P]),
        "msc_extremum_graph": (ctypes.c_int, [P, P, Grid, I32, I32, I32, P, P, P, I64, P, P, SZ, P, P]),
        "msc_adjacency_csr": (ctypes.c_int, [P, P, P, I32, I64, I32, P, P, I64, P, P, SZ, P, P]),
        "msc_extremum_graph_csr": (ctypes.c_int, [P, P, P, P, I32, I64, I32, I32, P, P, P, I64, P, P, SZ, P, P]),
        "msc_launch_count": (ctypes.c_ulonglong, []),
        "msc_trace_enable": (None, [ctypes.c_int]),
        "msc_trace_reset": (None, []),
        "msc_trace_collect": (ctypes.c_int, [ctypes.c_char_p, SZ]),
        "msc_batch_workspace_bytes": (SZ, [P, I32]),
        "msc_batch_segment": (ctypes.c_int, [P, I32, P, P, P, P, P, P, P, SZ, P, P, P]),
        "msc_batch_plan_create": (ctypes.c_int, [P, I32, P, P, P, P, P, P, P, SZ, P, P, P,
                                                 ctypes.POINTER(ctypes.c_void_p)]),
        "msc_batch_plan_launch": (ctypes.c_int, [P, P]),
        "msc_batch_plan_kernels": (ctypes.c_int, [P]),
        "msc_batch_plan_destroy": (None, [P]),
        "msc_batch_autotune": (ctypes.c_int, [P, I32, P, P, P, P, P, P, P, SZ, P, P, I32,
                                              ctypes.POINTER(Tune), ctypes.POINTER(ctypes.c_float)]),
        "msc_server_create": (P, [SZ, I32, I64]),
        "msc_server_submit": (ctypes.c_int, [P, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)]),
        "msc_server_poll": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(Result)]),
        "msc_server_wait": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(Result)]),
        "msc_server_release": (ctypes.c_int, [P, ctypes.c_uint64]),
        "msc_server_stats": (ctypes.c_int, [P, ctypes.POINTER(SZ), ctypes.POINTER(I32), ctypes.POINTER(I32),
                                            ctypes.POINTER(I32)]),
        "msc_server_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# C ABI mirror


def _p(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _grid(dims) -> Grid:
    nx, ny, nz = (int(d) for d in dims)
    return Grid(nx, ny, nz)


def msc_workspace_bytes(op: int, n: int, nnz: int = 0) -> int:
    return int(load().msc_workspace_bytes(op, n, nnz))


def msc_status_string(code: int) -> str:
    try:
        return load().msc_status_string(code).decode()
    except Exception:  # library not loadable: still describe the code
        return str(code)


def msc_order(f, n, order, ws, ws_bytes, status, stream=None) -> int:
    return load().msc_order(_p(f), n, _p(order), _p(ws), ws_bytes, _p(status), _stream(stream))


def msc_steepest_grid(order, dims, asc_ptr, desc_ptr, stream=None) -> int:
    return load().msc_steepest_grid(_p(order), _grid(dims), _p(asc_ptr), _p(desc_ptr), _stream(stream))


def msc_steepest_csr(order, row, col, n, asc_ptr, desc_ptr, status, stream=None) -> int:
    return load().msc_steepest_csr(_p(order), _p(row), _p(col), n, _p(asc_ptr), _p(desc_ptr), _p(status),
                                   _stream(stream))


def msc_compress(ptr, n, ws, ws_bytes, status, stream=None) -> int:
    return load().msc_compress(_p(ptr), n, _p(ws), ws_bytes, _p(status), _stream(stream))


def msc_compress_noalloc(ptr, n, status, stream=None) -> int:
    """Path compression with no workspace (static device scratch, n <= NOALLOC_MAX_N)."""
    return load().msc_compress_noalloc(_p(ptr), n, _p(status), _stream(stream))


def msc_ms_id(asc, desc, n, ms, num_cells, ws, ws_bytes, status, stream=None) -> int:
    return load().msc_ms_id(_p(asc), _p(desc), n, _p(ms), _p(num_cells), _p(ws), ws_bytes, _p(status),
                            _stream(stream))


def msc_segment(f, dims, order, asc, desc, ms, num_cells, ws, ws_bytes, status, stream=None) -> int:
    return load().msc_segment(_p(f), _grid(dims), _p(order), _p(asc), _p(desc), _p(ms), _p(num_cells),
                              _p(ws), ws_bytes, _p(status), _stream(stream))


def msc_cc_mask(mask, dims, conn, label, ws, ws_bytes, status, stream=None) -> int:
    return load().msc_cc_mask(_p(mask), _grid(dims), conn, _p(label), _p(ws), ws_bytes, _p(status),
                              _stream(stream))


def msc_cc_mesh(row, col, n, label, ws, ws_bytes, status, stream=None) -> int:
    return load().msc_cc_mesh(_p(row), _p(col), n, _p(label), _p(ws), ws_bytes, _p(status), _stream(stream))


def msc_adjacency_grid(label, dims, conn, label_bound, a, b, cap, num_pairs, ws, ws_bytes, status,
                       stream=None) -> int:
    return load().msc_adjacency_grid(_p(label), _grid(dims), conn, label_bound, _p(a), _p(b), cap, _p(num_pairs),
                                     _p(ws), ws_bytes, _p(status), _stream(stream))


def msc_extremum_graph(label, order, dims, conn, label_bound, sense, a, b, saddle, cap, num_arcs, ws, ws_bytes,
                       status, stream=None) -> int:
    return load().msc_extremum_graph(_p(label), _p(order), _grid(dims), conn, label_bound, sense, _p(a), _p(b),
                                     _p(saddle), cap, _p(num_arcs), _p(ws), ws_bytes, _p(status), _stream(stream))


def msc_adjacency_csr(label, row, col, n, nnz, label_bound, a, b, cap, num_pairs, ws, ws_bytes, status,
                      stream=None) -> int:
    return load().msc_adjacency_csr(_p(label), _p(row), _p(col), n, nnz, label_bound, _p(a), _p(b), cap,
                                    _p(num_pairs), _p(ws), ws_bytes, _p(status), _stream(stream))


def msc_extremum_graph_csr(label, order, row, col, n, nnz, label_bound, sense, a, b, saddle, cap, num_arcs, ws,
                           ws_bytes, status, stream=None) -> int:
    return load().msc_extremum_graph_csr(_p(label), _p(order), _p(row), _p(col), n, nnz, label_bound, sense, _p(a),
                                         _p(b), _p(saddle), cap, _p(num_arcs), _p(ws), ws_bytes, _p(status),
                                         _stream(stream))


def msc_launch_count() -> int:
    return int(load().msc_launch_count())


def msc_trace_enable(on: bool) -> None:
    load().msc_trace_enable(1 if on else 0)


def msc_trace_reset() -> None:
    load().msc_trace_reset()


def msc_trace_collect() -> dict:
    """{label: (launches, total device ms)} of the launches recorded while
    tracing was enabled (waits for them to finish)."""
    import json

    cap = 1 << 16
    buf = ctypes.create_string_buffer(cap)
    code = load().msc_trace_collect(buf, cap)
    if code != OK:
        raise MSCError(code, "msc_trace_collect")
    return {k: (int(v[0]), float(v[1])) for k, v in json.loads(buf.value.decode()).items()}


def _grids(dims_list):
    arr = (Grid * max(len(dims_list), 1))()
    for i, d in enumerate(dims_list):
        arr[i] = _grid(d)
    return arr


def _tune(tune):
    if tune is None:
        return None
    if isinstance(tune, Tune):
        return ctypes.byref(tune)
    shape, shift = tune
    return ctypes.byref(Tune(int(shape), int(shift)))


def msc_batch_workspace_bytes(dims_list) -> int:
    return int(load().msc_batch_workspace_bytes(_grids(dims_list), len(dims_list)))


def msc_batch_segment(dims_list, f, order, asc, desc, ms, num_cells, ws, ws_bytes, tune, status,
                      stream=None) -> int:
    return load().msc_batch_segment(_grids(dims_list), len(dims_list), _p(f), _p(order), _p(asc), _p(desc),
                                    _p(ms), _p(num_cells), _p(ws), ws_bytes, _tune(tune), _p(status),
                                    _stream(stream))


def msc_batch_plan_create(dims_list, f, order, asc, desc, ms, num_cells, ws, ws_bytes, tune, status,
                          stream=None):
    """Returns (code, plan handle as int)."""
    h = ctypes.c_void_p()
    code = load().msc_batch_plan_create(_grids(dims_list), len(dims_list), _p(f), _p(order), _p(asc), _p(desc),
                                        _p(ms), _p(num_cells), _p(ws), ws_bytes, _tune(tune), _p(status),
                                        _stream(stream), ctypes.byref(h))
    return code, (h.value or 0)


def msc_batch_plan_launch(plan: int, stream=None) -> int:
    return load().msc_batch_plan_launch(plan, _stream(stream))


def msc_batch_plan_kernels(plan: int) -> int:
    return int(load().msc_batch_plan_kernels(plan))


def msc_batch_plan_destroy(plan: int) -> None:
    load().msc_batch_plan_destroy(plan)


def msc_batch_autotune(dims_list, f, order, asc, desc, ms, num_cells, ws, ws_bytes, status, reps=2,
                       stream=None):
    """Returns (code, Tune, mean ms of the winner)."""
    best = Tune(-1, 0)
    t = ctypes.c_float(0.0)
    code = load().msc_batch_autotune(_grids(dims_list), len(dims_list), _p(f), _p(order), _p(asc), _p(desc),
                                     _p(ms), _p(num_cells), _p(ws), ws_bytes, _p(status), _stream(stream),
                                     int(reps), ctypes.byref(best), ctypes.byref(t))
    return code, best, float(t.value)


# ---------------------------------------------------------------------------
# convenience layer


def _dev(t: torch.Tensor) -> torch.device:
    if not t.is_cuda:
        raise MSCError(ERR_ARG, "input must be a CUDA tensor (there is no CPU path)")
    return t.device


def _check(code: int, where: str):
    if code != OK:
        raise MSCError(code, where)


def _finish(status: torch.Tensor, where: str):
    code = int(status.item())  # synchronises the stream
    _check(code, where)


def _ws(op: int, n: int, dev, nnz: int = 0) -> torch.Tensor:
    return torch.empty(max(msc_workspace_bytes(op, n, nnz), 1), dtype=torch.uint8, device=dev)


def _flat(t: torch.Tensor, dtype) -> torch.Tensor:
    if t.dtype != dtype:
        raise MSCError(ERR_ARG, f"expected {dtype}, got {t.dtype}")
    return t.contiguous().view(-1)


def _cols(col: torch.Tensor) -> torch.Tensor:
    """CSR columns; an edgeless graph still gets a valid (unread) pointer."""
    col = _flat(col, torch.int32)
    return col if col.numel() else torch.zeros(1, dtype=torch.int32, device=col.device)


def order(f: torch.Tensor) -> torch.Tensor:
    dev = _dev(f)
    f = _flat(f, torch.float32)
    n = f.numel()
    out = torch.empty(n, dtype=torch.int32, device=dev)
    ws = _ws(OP_ORDER, n, dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    _check(msc_order(f, n, out, ws, ws.numel(), st), "msc_order")
    _finish(st, "msc_order")
    return out


def steepest_grid(order_field: torch.Tensor, dims):
    dev = _dev(order_field)
    o = _flat(order_field, torch.int32)
    asc = torch.empty_like(o)
    desc = torch.empty_like(o)
    _check(msc_steepest_grid(o, dims, asc, desc), "msc_steepest_grid")
    torch.cuda.current_stream(dev).synchronize()
    return asc, desc


def steepest_csr(order_field: torch.Tensor, row: torch.Tensor, col: torch.Tensor):
    dev = _dev(order_field)
    o = _flat(order_field, torch.int32)
    row = _flat(row, torch.int32)
    col = _cols(col)
    n = row.numel() - 1
    asc = torch.empty(n, dtype=torch.int32, device=dev)
    desc = torch.empty(n, dtype=torch.int32, device=dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    _check(msc_steepest_csr(o, row, col, n, asc, desc, st), "msc_steepest_csr")
    _finish(st, "msc_steepest_csr")
    return asc, desc


def compress(ptr: torch.Tensor, inplace: bool = False) -> torch.Tensor:
    dev = _dev(ptr)
    p = _flat(ptr, torch.int32)
    if not inplace:
        p = p.clone()
    n = p.numel()
    ws = _ws(OP_COMPRESS, n, dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    _check(msc_compress(p, n, ws, ws.numel(), st), "msc_compress")
    _finish(st, "msc_compress")
    return p


def ms_id(asc: torch.Tensor, desc: torch.Tensor):
    dev = _dev(asc)
    a = _flat(asc, torch.int32)
    d = _flat(desc, torch.int32)
    n = a.numel()
    ms = torch.empty(n, dtype=torch.int32, device=dev)
    k = torch.empty(1, dtype=torch.int32, device=dev)
    ws = _ws(OP_MS_ID, n, dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    _check(msc_ms_id(a, d, n, ms, k, ws, ws.numel(), st), "msc_ms_id")
    _finish(st, "msc_ms_id")
    return ms, int(k.item())


def segment(f: torch.Tensor, dims, ws: torch.Tensor | None = None):
    """order, asc (minimum label), desc (maximum label), ms, num_cells."""
    dev = _dev(f)
    f = _flat(f, torch.float32)
    n = f.numel()
    if n != int(dims[0]) * int(dims[1]) * int(dims[2]):
        raise MSCError(ERR_ARG, "segment: dims do not match the field size")
    outs = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(4)]
    k = torch.empty(1, dtype=torch.int32, device=dev)
    if ws is None:
        ws = _ws(OP_SEGMENT, n, dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    _check(msc_segment(f, dims, *outs, k, ws, ws.numel(), st), "msc_segment")
    _finish(st, "msc_segment")
    return (*outs, int(k.item()))


def cc_mask(mask: torch.Tensor, dims, conn: int = 6) -> torch.Tensor:
    dev = _dev(mask)
    m = _flat(mask, torch.uint8)
    n = m.numel()
    if n != int(dims[0]) * int(dims[1]) * int(dims[2]):
        raise MSCError(ERR_ARG, "cc_mask: dims do not match the mask size")
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    ws = _ws(OP_CC_MASK, n, dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    _check(msc_cc_mask(m, dims, conn, lab, ws, ws.numel(), st), "msc_cc_mask")
    _finish(st, "msc_cc_mask")
    return lab


def cc_mesh(row: torch.Tensor, col: torch.Tensor) -> torch.Tensor:
    dev = _dev(row)
    row = _flat(row, torch.int32)
    col = _cols(col)
    n = row.numel() - 1
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    ws = _ws(OP_CC_MESH, n, dev, col.numel())
    st = torch.empty(1, dtype=torch.int32, device=dev)
    _check(msc_cc_mesh(row, col, n, lab, ws, ws.numel(), st), "msc_cc_mesh")
    _finish(st, "msc_cc_mesh")
    return lab


def adjacency_grid(label: torch.Tensor, dims, conn: int = 14, label_bound: int | None = None,
                   cap: int | None = None, ws: torch.Tensor | None = None):
    """Distinct pairs (a, b), a < b, of different non-negative labels that
    meet across an edge of the grid (conn 14: the triangulation, 6: the face
    grid), in lexicographic order, as two int32 tensors.  label_bound
    (default n) bounds every label.  The pairs are first collected into
    `cap` slots (default min(7n, 2^24)); a call that finds more runs again
    with room for all of them."""
    dev = _dev(label)
    lab = _flat(label, torch.int32)
    n = lab.numel()
    if n != int(dims[0]) * int(dims[1]) * int(dims[2]):
        raise MSCError(ERR_ARG, "adjacency_grid: dims do not match the label size")
    bound = max(n, 1) if label_bound is None else int(label_bound)
    cap = min(7 * n, 1 << 24) if cap is None else int(cap)
    if ws is None:
        ws = _ws(OP_ADJACENCY, n, dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    k = torch.empty(1, dtype=torch.int64, device=dev)
    while True:
        a = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        b = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        _check(msc_adjacency_grid(lab, dims, conn, bound, a, b, cap, k, ws, ws.numel(), st), "msc_adjacency_grid")
        _finish(st, "msc_adjacency_grid")
        K = int(k.item())
        if K <= cap:
            return a[:K], b[:K]
        cap = K


def extremum_graph(label: torch.Tensor, order_field: torch.Tensor, dims, sense: int = 1, conn: int = 14,
                   label_bound: int | None = None, cap: int | None = None, ws: torch.Tensor | None = None):
    """Arcs (a, b) of the extremum graph with their saddle vertices: pairs of
    maximum (sense +1) or minimum (sense -1) regions that touch, in
    lexicographic order, each with the end vertex of its highest (maxima) or
    lowest (minima) crossing edge in the order.  Three int32 tensors."""
    dev = _dev(label)
    lab = _flat(label, torch.int32)
    o = _flat(order_field, torch.int32)
    n = lab.numel()
    if n != int(dims[0]) * int(dims[1]) * int(dims[2]) or o.numel() != n:
        raise MSCError(ERR_ARG, "extremum_graph: dims do not match the label / order size")
    bound = max(n, 1) if label_bound is None else int(label_bound)
    cap = min(7 * n, 1 << 24) if cap is None else int(cap)
    if ws is None:
        ws = _ws(OP_EXTREMUM_GRAPH, n, dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    k = torch.empty(1, dtype=torch.int64, device=dev)
    while True:
        a, b, s = (torch.empty(max(cap, 1), dtype=torch.int32, device=dev) for _ in range(3))
        _check(msc_extremum_graph(lab, o, dims, conn, bound, sense, a, b, s, cap, k, ws, ws.numel(), st),
               "msc_extremum_graph")
        _finish(st, "msc_extremum_graph")
        K = int(k.item())
        if K <= cap:
            return a[:K], b[:K], s[:K]
        cap = K


def _csr_pairs(label, row, col, order, sense, label_bound, cap, ws):
    dev = _dev(label)
    lab = _flat(label, torch.int32)
    row = _flat(row, torch.int32)
    nnz = int(col.numel())
    col = _cols(col)
    n = lab.numel()
    if row.numel() != n + 1:
        raise MSCError(ERR_ARG, "CSR row array must have n + 1 entries")
    o = None if order is None else _flat(order, torch.int32)
    bound = max(n, 1) if label_bound is None else int(label_bound)
    cap = min(max(nnz, 1), 1 << 24) if cap is None else int(cap)
    op = OP_ADJACENCY_CSR if o is None else OP_EXTREMUM_GRAPH_CSR
    if ws is None:
        ws = _ws(op, n, dev, nnz)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    k = torch.empty(1, dtype=torch.int64, device=dev)
    while True:
        a, b, s = (torch.empty(max(cap, 1), dtype=torch.int32, device=dev) for _ in range(3))
        if o is None:
            code = msc_adjacency_csr(lab, row, col, n, nnz, bound, a, b, cap, k, ws, ws.numel(), st)
        else:
            code = msc_extremum_graph_csr(lab, o, row, col, n, nnz, bound, sense, a, b, s, cap, k, ws, ws.numel(), st)
        where = "msc_adjacency_csr" if o is None else "msc_extremum_graph_csr"
        _check(code, where)
        _finish(st, where)
        K = int(k.item())
        if K <= cap:
            return (a[:K], b[:K]) if o is None else (a[:K], b[:K], s[:K])
        cap = K


def adjacency_csr(label: torch.Tensor, row: torch.Tensor, col: torch.Tensor, label_bound: int | None = None,
                  cap: int | None = None, ws: torch.Tensor | None = None):
    """Distinct label pairs (a, b), a < b, across the edges of a mesh given
    as its symmetric CSR vertex adjacency: two int32 tensors."""
    return _csr_pairs(label, row, col, None, 1, label_bound, cap, ws)


def extremum_graph_csr(label: torch.Tensor, order_field: torch.Tensor, row: torch.Tensor, col: torch.Tensor,
                       sense: int = 1, label_bound: int | None = None, cap: int | None = None,
                       ws: torch.Tensor | None = None):
    """Extremum-graph arcs (a, b) with their saddle vertices over a mesh
    given as its symmetric CSR vertex adjacency: three int32 tensors."""
    return _csr_pairs(label, row, col, order_field, sense, label_bound, cap, ws)


class Batch:
    """A batch of grids packed into one vertex space with its outputs and
    workspace (torch CUDA tensors), run by plain launches (``run``) or a
    captured CUDA graph (``plan`` then ``launch``).  Outputs are
    instance-local: ``split`` cuts a packed array into per-instance views."""

    def __init__(self, dims_list, device="cuda"):
        self.dims = [tuple(int(x) for x in d) for d in dims_list]
        self.sizes = [d[0] * d[1] * d[2] for d in self.dims]
        self.offsets = [0]
        for n in self.sizes:
            self.offsets.append(self.offsets[-1] + n)
        self.total = self.offsets[-1]
        dev = torch.device(device)
        self.f = torch.empty(self.total, dtype=torch.float32, device=dev)
        self.order, self.asc, self.desc, self.ms = (torch.empty(max(self.total, 1), dtype=torch.int32, device=dev)
                                                    for _ in range(4))
        self.num_cells = torch.empty(len(self.dims), dtype=torch.int32, device=dev)
        nbytes = msc_batch_workspace_bytes(self.dims)
        if nbytes == 0:
            raise MSCError(ERR_ARG, "Batch: invalid grids")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.status = torch.empty(1, dtype=torch.int32, device=dev)
        self._plan = 0

    def _bufs(self):
        return (self.f, self.order, self.asc, self.desc, self.ms, self.num_cells, self.ws, self.ws.numel())

    def run(self, tune=None, sync=True):
        _check(msc_batch_segment(self.dims, *self._bufs(), tune, self.status), "msc_batch_segment")
        if sync:
            _finish(self.status, "msc_batch_segment")

    def plan(self, tune=None):
        self.close()
        code, h = msc_batch_plan_create(self.dims, *self._bufs(), tune, self.status)
        _check(code, "msc_batch_plan_create")
        self._plan = h
        return msc_batch_plan_kernels(h)

    def launch(self, sync=True):
        if not self._plan:
            raise MSCError(ERR_ARG, "Batch.launch: no plan (call plan() first)")
        _check(msc_batch_plan_launch(self._plan), "msc_batch_plan_launch")
        if sync:
            _finish(self.status, "msc_batch_plan_launch")

    def autotune(self, reps=2):
        code, best, ms = msc_batch_autotune(self.dims, *self._bufs(), self.status, reps)
        _check(code, "msc_batch_autotune")
        return (best.steepest_shape, best.build_shift), ms

    def split(self, t: torch.Tensor):
        return [t[a:b] for a, b in zip(self.offsets[:-1], self.offsets[1:])]

    def close(self):
        if self._plan:
            msc_batch_plan_destroy(self._plan)
            self._plan = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# serving


def msc_server_create(budget: int, slots: int = 4, group_max_vertices: int = 1 << 21) -> int:
    return load().msc_server_create(budget, slots, group_max_vertices) or 0


def msc_server_submit(srv: int, job: Job):
    t = ctypes.c_uint64()
    code = load().msc_server_submit(srv, ctypes.byref(job), ctypes.byref(t))
    return code, int(t.value)


def msc_server_poll(srv: int, ticket: int):
    r = Result()
    return load().msc_server_poll(srv, ticket, ctypes.byref(r)), r


def msc_server_wait(srv: int, ticket: int, timeout_ms: float = -1.0):
    r = Result()
    return load().msc_server_wait(srv, ticket, float(timeout_ms), ctypes.byref(r)), r


def msc_server_release(srv: int, ticket: int) -> int:
    return load().msc_server_release(srv, ticket)


def msc_server_stats(srv: int):
    used, q, run, done = ctypes.c_size_t(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    code = load().msc_server_stats(srv, ctypes.byref(used), ctypes.byref(q), ctypes.byref(run), ctypes.byref(done))
    _check(code, "msc_server_stats")
    return {"arena_used": used.value, "queued": q.value, "running": run.value, "done": done.value}


def msc_server_destroy(srv: int) -> None:
    load().msc_server_destroy(srv)


class _DeviceArray:
    """A device int32 array by address (zero-copy view through the CUDA array interface)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False), "version": 2,
                                         "strides": None}


class Server:
    """msc_server with torch inputs: submit fields / masks, wait, view the
    device-resident outputs as torch tensors (valid until ``release``)."""

    def __init__(self, budget: int, slots: int = 4, group_max_vertices: int = 1 << 21):
        self.h = msc_server_create(int(budget), int(slots), int(group_max_vertices))
        if not self.h:
            raise MSCError(ERR_BUDGET, "msc_server_create (bad arguments or arena allocation failed)")
        self._inputs = {}

    def _submit(self, kind, t, dims, conn):
        n = int(dims[0]) * int(dims[1]) * int(dims[2])
        if t.numel() != n or not t.is_cuda or not t.is_contiguous():
            raise MSCError(ERR_ARG, "submit: input must be a contiguous CUDA tensor of the grid's size")
        code, ticket = msc_server_submit(self.h, Job(kind, _grid(dims), conn, t.data_ptr()))
        _check(code, "msc_server_submit")
        self._inputs[ticket] = t  # the input must outlive the request
        return ticket

    def submit_segment(self, f: torch.Tensor, dims) -> int:
        return self._submit(JOB_SEGMENT, _flat(f, torch.float32), dims, 0)

    def submit_cc(self, mask: torch.Tensor, dims, conn: int = 6) -> int:
        return self._submit(JOB_CC_MASK, _flat(mask, torch.uint8), dims, conn)

    def poll(self, ticket: int) -> Result:
        code, r = msc_server_poll(self.h, ticket)
        if code not in (OK, PENDING):
            raise MSCError(code, "msc_server_poll")
        return r

    def wait(self, ticket: int, timeout_ms: float = -1.0) -> Result:
        code, r = msc_server_wait(self.h, ticket, timeout_ms)
        if code not in (OK, PENDING):
            raise MSCError(code, "msc_server_wait")
        return r

    @staticmethod
    def view(r: Result, field: str) -> torch.Tensor:
        ptr = getattr(r, field)
        if not ptr:
            raise MSCError(ERR_ARG, f"result has no {field}")
        return torch.as_tensor(_DeviceArray(ptr, int(r.n)), device="cuda")

    def outputs(self, ticket: int) -> dict:
        """Copies of the request's outputs (waits for it)."""
        r = self.wait(ticket)
        _check(r.status, "served request")
        if r.label:
            return {"label": self.view(r, "label").clone()}
        out = {k: self.view(r, k).clone() for k in ("order", "asc", "desc", "ms")}
        out["num_cells"] = int(r.num_cells)
        return out

    def release(self, ticket: int) -> None:
        code = msc_server_release(self.h, ticket)
        _check(code, "msc_server_release")
        self._inputs.pop(ticket, None)

    def stats(self) -> dict:
        return msc_server_stats(self.h)

    def close(self):
        if self.h:
            msc_server_destroy(self.h)
            self.h = 0
            self._inputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
