"""Host-side pieces of the benchmark that need no GPU: the algorithmic-byte
table, the per-kernel DRAM-traffic lookup and its source hashes."""
import json
import os

import bench


def test_algorithmic_bytes_scale_with_the_sizes():
    n, nm, nnz = 1 << 20, 1 << 16, 1 << 18
    assert bench.algorithmic_bytes("order.down", n, nm, nnz) == 16 * n
    assert bench.algorithmic_bytes("order.up", n, nm, nnz) == 4 * n
    assert bench.algorithmic_bytes("steepest.grid", n, nm, nnz) == 12 * n
    assert bench.algorithmic_bytes("mesh.flatten", n, nm, nnz) == 8 * nm
    assert bench.algorithmic_bytes("mesh.hook", n, nm, nnz) is None  # data-dependent


def test_committed_traffic_follows_the_kernel_sources():
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    t = json.load(open(path))
    for label, e in t["kernels"].items():
        got = bench.committed_traffic(label)
        # an entry is used exactly while its kernel's sources hash as captured
        if e["sha"] == bench.sources_sha([e["source"]]):
            assert got == float(e["dram_bytes_per_vertex"])
        else:
            assert got is None
    assert bench.committed_traffic("no.such.kernel") is None


def test_sources_sha_depends_on_the_named_file_only():
    a = bench.sources_sha(["compress.cu"])
    assert a == bench.sources_sha(["compress.cu"])
    assert a != bench.sources_sha(["sort.cu"])
    assert len(a) == 16


def test_every_stage_prefix_matches_a_traced_label_family():
    labels = ["order.up", "order.down", "steepest.grid", "compress.jump", "msid.insert", "cc.local", "mesh.link"]
    for name, prefix in bench.STAGES.items():
        assert any(l.startswith(prefix) for l in labels), name
