"""The C-ABI library builds, loads and exports every entry point that
include/msc.h declares; host-side queries work without a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2409_03771_gb300 as m
    from paper_2409_03771_gb300 import _build

    _build.build()
    return m.load()


def declared_symbols():
    out = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            out += re.findall(r"MSC_API\s+[\w\s\*]+?\b(msc_\w+)\s*\(", text)
    return out


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["msc_order", "msc_steepest_grid", "msc_steepest_csr", "msc_compress", "msc_ms_id",
                 "msc_segment", "msc_cc_mask", "msc_cc_mesh", "msc_adjacency_grid", "msc_workspace_bytes",
                 "msc_status_string"]:
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_workspace_and_status_queries(lib):
    import paper_2409_03771_gb300 as m

    assert m.msc_status_string(m.ERR_NAN) == "NaN in scalar field"
    assert m.msc_status_string(m.ERR_NOT_CONVERGED).startswith("pointer jumping")
    n = 512 ** 3
    seg = m.msc_workspace_bytes(m.OP_SEGMENT, n)
    assert seg > m.msc_workspace_bytes(m.OP_ORDER, n) // 2 > 0
    assert m.msc_workspace_bytes(m.OP_COMPRESS, 100) > 0
    assert m.msc_workspace_bytes(99, 100) == 0
    assert m.msc_workspace_bytes(m.OP_ORDER, -1) == 0
    assert m.msc_workspace_bytes(m.OP_ORDER, 2 ** 31) == 0


def test_host_argument_checks_need_no_gpu(lib):
    import paper_2409_03771_gb300 as m

    # null pointers and bad grids are refused before any CUDA call
    assert m.msc_steepest_grid(0, (4, 4, 4), 0, 0, stream=0) == m.ERR_ARG
    assert m.msc_steepest_grid(16, (0, 4, 4), 16, 16, stream=0) == m.ERR_ARG
    assert m.msc_cc_mask(16, (4, 4, 4), 7, 16, 16, 256, 16, stream=0) == m.ERR_ARG
    assert m.msc_segment(16, (4, 4, 4), 16, 16, 16, 16, 16, 256, 10, 16, stream=0) == m.ERR_WS
    assert m.msc_compress(16, 10, 256, 0, 16, stream=0) == m.ERR_WS
    # a workspace that is not 256-byte aligned is refused before any launch
    assert m.msc_compress(16, 10, 16 + 4, 1 << 20, 16, stream=0) == m.ERR_ARG
    assert m.msc_order(16, 10, 16, 256 + 16, 1 << 30, 16, stream=0) == m.ERR_ARG
    # the batch and serving entry points check their arguments on the host too
    assert m.msc_batch_workspace_bytes([(4, 4, 4), (2, 3, 5)]) > m.msc_batch_workspace_bytes([(4, 4, 4)]) > 0
    assert m.msc_batch_workspace_bytes([(4, 4, 0)]) == 0
    assert m.msc_batch_segment([(4, 4, 4)], 0, 0, 0, 0, 0, 0, 0, 0, None, 0, stream=0) == m.ERR_ARG
    assert m.msc_batch_segment([(4, 4, 4)], 16, 16, 16, 16, 16, 16, 256, 10, (9, 0), 16, stream=0) == m.ERR_ARG
    assert m.msc_server_create(0, 1, 0) == 0
    assert m.msc_server_create(1 << 20, 0, 0) == 0
    assert m.msc_server_submit(0, m.Job())[0] == m.ERR_ARG
    # region adjacency: connectivity, label bound, capacity, workspace size and alignment
    ws = m.msc_workspace_bytes(m.OP_ADJACENCY, 64)
    assert ws > 7 * 64 * 8 * 2
    assert m.msc_workspace_bytes(m.OP_ADJACENCY, (2 ** 31) // 7 + 1) == 0
    args = dict(a=16, b=16, cap=4, num_pairs=16, ws=256, ws_bytes=ws, status=16, stream=0)
    assert m.msc_adjacency_grid(16, (4, 4, 4), 8, 64, **args) == m.ERR_ARG
    assert m.msc_adjacency_grid(16, (4, 4, 4), 14, 0, **args) == m.ERR_ARG
    assert m.msc_adjacency_grid(16, (4, 4, 4), 14, 64, **dict(args, cap=-1)) == m.ERR_ARG
    assert m.msc_adjacency_grid(16, (4, 4, 4), 14, 64, **dict(args, a=0)) == m.ERR_ARG
    assert m.msc_adjacency_grid(16, (4, 4, 4), 14, 64, **dict(args, ws=256 + 8)) == m.ERR_ARG
    assert m.msc_adjacency_grid(16, (4, 4, 4), 14, 64, **dict(args, ws_bytes=ws - 1)) == m.ERR_WS
    assert m.msc_adjacency_grid(16, (1024, 1024, 1024), 6, 64, **args) == m.ERR_TOO_LARGE
    # extremum graph: the order is required, sense is +1 or -1, the saddle output is needed
    gws = m.msc_workspace_bytes(m.OP_EXTREMUM_GRAPH, 64)
    assert gws > ws
    gargs = dict(a=16, b=16, saddle=16, cap=4, num_arcs=16, ws=256, ws_bytes=gws, status=16, stream=0)
    assert m.msc_extremum_graph(16, 0, (4, 4, 4), 14, 64, 1, **gargs) == m.ERR_ARG
    assert m.msc_extremum_graph(16, 16, (4, 4, 4), 14, 64, 0, **gargs) == m.ERR_ARG
    assert m.msc_extremum_graph(16, 16, (4, 4, 4), 14, 64, 1, **dict(gargs, saddle=0)) == m.ERR_ARG
    assert m.msc_extremum_graph(16, 16, (4, 4, 4), 14, 64, -1, **dict(gargs, ws_bytes=ws)) == m.ERR_WS
    # mesh variants: sizes, bounds, workspace
    cws = m.msc_workspace_bytes(m.OP_ADJACENCY_CSR, 100, 1000)
    assert m.msc_workspace_bytes(m.OP_EXTREMUM_GRAPH_CSR, 100, 1000) > cws > 1000 * 16
    assert m.msc_workspace_bytes(m.OP_ADJACENCY_CSR, 100, 2 ** 31) == 0
    assert m.msc_adjacency_csr(16, 16, 16, 100, 1000, 0, 16, 16, 4, 16, 256, cws, 16, stream=0) == m.ERR_ARG
    assert m.msc_adjacency_csr(16, 16, 16, 100, -1, 100, 16, 16, 4, 16, 256, cws, 16, stream=0) == m.ERR_ARG
    assert m.msc_adjacency_csr(16, 16, 16, 100, 1000, 100, 16, 16, 4, 16, 256, cws - 1, 16, stream=0) == m.ERR_WS
    assert m.msc_extremum_graph_csr(16, 0, 16, 16, 100, 1000, 100, 1, 16, 16, 16, 4, 16, 256, cws, 16,
                                    stream=0) == m.ERR_ARG


def test_no_cpu_fallback():
    import torch

    import paper_2409_03771_gb300 as m

    with pytest.raises(m.MSCError):
        m.order(torch.zeros(8))
