"""Pins for the oracle's path compression (walk) and Morse-Smale ids.

The walk is pinned to the paper's worked example (Fig. 2: rank-local
compression with ghost vertices as maxima, the synchronous pointer-doubling
table, the final label), to forests whose roots are known by construction,
and to cycle detection.  The Morse-Smale id is pinned to numpy's own
de-duplication (a different method) and to the definition's properties.
"""
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig2_spiral.txt")


def load_fig2():
    spec = {"owned": {}, "local": {}, "table": {}}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tag, *rest = line.split()
        if tag == "polyline":
            spec["polyline"] = rest
        elif tag == "owned":
            spec["owned"][rest[0]] = rest[1:]
        elif tag == "local":
            spec["local"][rest[0]] = dict(t.split(":") for t in rest[1:])
        elif tag == "table":
            spec["table"][rest[0]] = rest[1:]
        elif tag == "final":
            spec["final"] = rest[0]
    return spec


def polyline_csr(names, keep):
    """CSR of the polyline restricted to the vertex subset ``keep``."""
    idx = {v: i for i, v in enumerate(names)}
    nbrs = {v: [] for v in names}
    for a, b in zip(names[:-1], names[1:]):
        if a in keep and b in keep:
            nbrs[a].append(idx[b])
            nbrs[b].append(idx[a])
    row = [0]
    col = []
    for v in names:
        col += sorted(nbrs[v])
        row.append(len(col))
    return np.array(row, np.int32), np.array(col, np.int32)


def test_fig2_global_label_is_P(oracle_mod):
    spec = load_fig2()
    names = spec["polyline"]
    order = np.arange(len(names), dtype=np.int32)  # f increases alphabetically
    row, col = polyline_csr(names, set(names))
    asc_ptr, desc_ptr = oracle_mod.steepest_csr(order, row, col)
    desc = oracle_mod.walk(desc_ptr)
    assert all(names[d] == spec["final"] for d in desc)
    assert all(names[a] == "A" for a in oracle_mod.walk(asc_ptr))


def test_fig2_rank_local_compression(oracle_mod):
    """Panel b: each rank compresses its own vertices, ghosts act as maxima."""
    spec = load_fig2()
    names = spec["polyline"]
    idx = {v: i for i, v in enumerate(names)}
    order = np.arange(len(names), dtype=np.int32)
    for rank, owned in spec["owned"].items():
        ghosts = set()
        for v in owned:
            i = idx[v]
            for j in (i - 1, i + 1):
                if 0 <= j < len(names) and names[j] not in owned:
                    ghosts.add(names[j])
        row, col = polyline_csr(names, set(owned) | ghosts)
        _, desc_ptr = oracle_mod.steepest_csr(order, row, col)
        for g in ghosts:  # Alg. 1: ghost vertices point at themselves
            desc_ptr[idx[g]] = idx[g]
        for v in names:  # vertices outside this rank's view are inert
            if v not in owned and v not in ghosts:
                desc_ptr[idx[v]] = idx[v]
        local = oracle_mod.walk(desc_ptr)
        got = {v: names[local[idx[v]]] for v in owned}
        assert got == spec["local"][rank], rank


def test_fig2_doubling_table(oracle_mod):
    """The P0..P3 columns are synchronous pointer doubling on the ghosts."""
    spec = load_fig2()
    names = spec["polyline"]
    idx = {v: i for i, v in enumerate(names)}
    p = np.arange(len(names), dtype=np.int32)  # non-ghosts: fixed points
    for g, cols in spec["table"].items():
        p[idx[g]] = idx[cols[0]]
    for k in range(1, 4):
        nxt = oracle_mod.jump_sync(p)
        for g, cols in spec["table"].items():
            want = cols[k]
            if want == "-":  # converged: unchanged
                assert nxt[idx[g]] == p[idx[g]]
            else:
                assert names[nxt[idx[g]]] == want, (g, k)
        p = nxt
    assert all(names[p[idx[g]]] == "P" for g in spec["table"])


def random_forest(n, rng, n_roots):
    """Parent pointers with the root of every vertex known by construction."""
    perm = rng.permutation(n)
    ptr = np.empty(n, np.int32)
    root = np.empty(n, np.int32)
    for i, v in enumerate(perm):
        if i < n_roots:
            ptr[v] = v
            root[v] = v
        else:
            p = perm[rng.integers(max(0, i - 50), i)]  # an earlier vertex
            ptr[v] = p
            root[v] = root[p]
    return ptr, root


@pytest.mark.parametrize("seed", range(3))
def test_walk_on_forests(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    ptr, root = random_forest(5000, rng, 7)
    np.testing.assert_array_equal(oracle_mod.walk(ptr), root)
    np.testing.assert_array_equal(oracle_mod.walk_memo(ptr), root)


def test_walk_keeps_inactive_entries(oracle_mod):
    ptr = np.array([0, 0, -1, 1, -1, 4], np.int32)
    ptr[5] = 5
    np.testing.assert_array_equal(oracle_mod.walk(ptr), [0, 0, -1, 0, -1, 5])


@pytest.mark.parametrize("fn", ["walk", "walk_memo"])
def test_walk_detects_cycles_and_bad_pointers(oracle_mod, fn):
    with pytest.raises(oracle_mod.OracleError) as e:
        getattr(oracle_mod, fn)(np.array([1, 0, 2], np.int32))
    assert e.value.code == oracle_mod.ERR_CYCLE
    with pytest.raises(oracle_mod.OracleError) as e:
        getattr(oracle_mod, fn)(np.array([5, 1], np.int32))
    assert e.value.code == oracle_mod.ERR_ARG


# ---------------------------------------------------------------------------
# Morse-Smale ids


def numpy_dense_pairs(asc, desc):
    keys = np.stack([asc, desc], axis=1)
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    return inv.reshape(-1).astype(np.int32), uniq.shape[0]


@pytest.mark.parametrize("seed", range(3))
def test_ms_matches_numpy_unique(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    asc = rng.integers(0, 40, 3000).astype(np.int32)
    desc = rng.integers(0, 3000, 3000).astype(np.int32)
    ms, k = oracle_mod.ms(asc, desc)
    want, wk = numpy_dense_pairs(asc, desc)
    assert k == wk
    np.testing.assert_array_equal(ms, want)


def test_ms_properties_on_field(oracle_mod):
    dims = (18, 16, 14)
    f = workloads.smooth_field(dims, 8, (1.5, 3.5), seed=4, noise_amp=1e-3).numpy().ravel()
    order, asc, desc, ms, k = oracle_mod.segment_grid(f, dims)
    key = asc.astype(np.int64) * f.size + desc
    assert k == np.unique(key).size  # K = number of distinct pairs
    s = np.argsort(key, kind="stable")  # ms monotone in the pair key, dense
    steps = np.diff(ms[s])
    assert ((steps == 0) | (steps == 1)).all() and ms[s][0] == 0 and ms[s][-1] == k - 1
    assert ((steps == 1) == (np.diff(key[s]) > 0)).all()
    for c in range(k):  # every cell's vertices share one (min, max) pair
        members = ms == c
        assert np.unique(asc[members]).size == 1 and np.unique(desc[members]).size == 1
