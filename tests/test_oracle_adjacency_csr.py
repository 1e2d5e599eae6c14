"""Pins of the oracle's region adjacency and extremum graph over an explicit
mesh (symmetric CSR): brute force over the CSR entries written out here,
agreement with the (pinned) grid versions on the CSR of the grid's own
edges, valleys on a path graph, and the bad-column error."""
import numpy as np
import pytest

from test_oracle_adjacency import face_edges, kuhn_edges


def to_csr(n, edges):
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    row = np.zeros(n + 1, np.int32)
    for v in range(n):
        row[v + 1] = row[v] + len(adj[v])
    col = np.array([u for v in range(n) for u in sorted(adj[v])], np.int32)
    return row, col


def brute(label, order, row, col, sense):
    best = {}
    n = label.size
    for v in range(n):
        for e in range(row[v], row[v + 1]):
            u = int(col[e])
            la, lb = int(label[v]), int(label[u])
            if la < 0 or lb < 0 or la == lb:
                continue
            key = (min(la, lb), max(la, lb))
            if order is None:
                best[key] = 0
                continue
            w = (v if order[v] < order[u] else u) if sense > 0 else (v if order[v] > order[u] else u)
            if key not in best or (order[w] > order[best[key]] if sense > 0 else order[w] < order[best[key]]):
                best[key] = w
    keys = sorted(best)
    return [k[0] for k in keys], [k[1] for k in keys], [best[k] for k in keys]


@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_match_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(5, 80))
    m = int(rng.integers(0, 4 * n))
    edges = {(int(min(a, b)), int(max(a, b))) for a, b in rng.integers(0, n, (m, 2)) if a != b}
    row, col = to_csr(n, edges)
    lab = rng.integers(-1, 7, n).astype(np.int32)
    order = rng.permutation(n).astype(np.int32)
    a, b = oracle_mod.adjacency_csr(lab, row, col)
    wa, wb, _ = brute(lab, None, row, col, 1)
    assert a.tolist() == wa and b.tolist() == wb
    for sense in (1, -1):
        a, b, s = oracle_mod.adjacency_csr(lab, row, col, order, sense)
        wa, wb, ws = brute(lab, order, row, col, sense)
        assert a.tolist() == wa and b.tolist() == wb and s.tolist() == ws


@pytest.mark.parametrize("conn", [6, 14])
def test_grid_edges_as_a_mesh_equal_the_grid_versions(oracle_mod, conn):
    dims = (7, 5, 6)
    n = 7 * 5 * 6
    rng = np.random.default_rng(conn)
    row, col = to_csr(n, kuhn_edges(dims) if conn == 14 else face_edges(dims))
    lab = rng.integers(-1, 9, n).astype(np.int32)
    order = rng.permutation(n).astype(np.int32)
    ga, gb = oracle_mod.adjacency_grid(lab, dims, conn)
    ma, mb = oracle_mod.adjacency_csr(lab, row, col)
    np.testing.assert_array_equal(ga, ma)
    np.testing.assert_array_equal(gb, mb)
    for sense in (1, -1):
        want = oracle_mod.extremum_graph(lab, order, dims, conn, sense)
        got = oracle_mod.adjacency_csr(lab, row, col, order, sense)
        for x, y in zip(got, want):
            np.testing.assert_array_equal(x, y)


def test_path_graph_saddles_are_the_valleys(oracle_mod):
    rng = np.random.default_rng(8)
    L = 60
    f = rng.permutation(L)
    row, col = to_csr(L, {(i, i + 1) for i in range(L - 1)})
    order = np.argsort(np.argsort(f)).astype(np.int32)  # f is a permutation: order = f
    # maximum labels by walking up the path, from f alone
    def climb(i, up):
        while True:
            nb = [j for j in (i - 1, i + 1) if 0 <= j < L]
            j = max(nb, key=lambda t: f[t]) if up else min(nb, key=lambda t: f[t])
            if (f[j] > f[i]) if up else (f[j] < f[i]):
                i = j
            else:
                return i
    for sense in (1, -1):
        lab = np.array([climb(i, sense > 0) for i in range(L)], np.int32)
        g = f if sense > 0 else -f
        peaks = sorted(set(lab.tolist()))
        want = [(p, q, p + int(np.argmin(g[p:q + 1]))) for p, q in zip(peaks, peaks[1:])]
        a, b, s = oracle_mod.adjacency_csr(lab, row, col, order, sense)
        assert list(zip(a.tolist(), b.tolist(), s.tolist())) == want


def test_bad_column_is_an_error(oracle_mod):
    row = np.array([0, 1, 2], np.int32)
    col = np.array([1, 5], np.int32)
    with pytest.raises(RuntimeError):
        oracle_mod.adjacency_csr(np.zeros(2, np.int32), row, col)
