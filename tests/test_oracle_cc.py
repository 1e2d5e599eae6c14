"""Pins for the oracle's connected components.

BFS labelling is compared with an independent union-find written here, with
closed forms (all-ones, checkerboard, separated slabs, a complete and an
empty mesh), and with a literal replay of Alg. 3 (labels = largest id) in
the two readings the paper leaves open: one stitching pass (which can split
a component -- the counter-example below) and stitching iterated to a fixed
point (which gives BFS's partition).
"""
import itertools

import numpy as np
import pytest

import workloads

OFF6 = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
OFF14 = OFF6 + [(1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


def grid_edges(mask, dims, conn):
    nx, ny, nz = dims
    m = mask.reshape(nz, ny, nx).astype(bool)
    edges = []
    for dx, dy, dz in OFF6 if conn == 6 else OFF14:
        a = m[: nz - dz, : ny - dy, : nx - dx] & m[dz:, dy:, dx:]
        z, y, x = np.nonzero(a)
        v = x + nx * (y + ny * z)
        u = (x + dx) + nx * ((y + dy) + ny * (z + dz))
        edges.append(np.stack([v, u], 1))
    return np.concatenate(edges)


def union_find_labels(mask, edges):
    n = mask.size
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in edges:
        ra, rb = find(int(a)), find(int(b))
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    lab = np.array([find(v) for v in range(n)], np.int32)
    # root = smallest id only if hooking always keeps the smaller root
    lab[mask.ravel() == 0] = -1
    return lab


@pytest.mark.parametrize("conn", [6, 14])
@pytest.mark.parametrize("seed,density", [(0, 0.3), (1, 0.5), (2, 0.7)])
def test_bfs_matches_union_find(oracle_mod, conn, seed, density):
    dims = (9, 8, 7)
    rng = np.random.default_rng(seed)
    mask = (rng.random(int(np.prod(dims))) < density).astype(np.uint8)
    got = oracle_mod.cc_grid(mask, dims, conn)
    want = union_find_labels(mask, grid_edges(mask, dims, conn))
    np.testing.assert_array_equal(got, want)


def test_closed_forms(oracle_mod):
    dims = (6, 5, 4)
    n = 120
    assert (oracle_mod.cc_grid(np.ones(n, np.uint8), dims, 6) == 0).all()
    assert (oracle_mod.cc_grid(np.zeros(n, np.uint8), dims, 14) == -1).all()
    z, y, x = np.meshgrid(range(4), range(5), range(6), indexing="ij")
    cb = ((x + y + z) % 2 == 0).astype(np.uint8).ravel()
    lab = oracle_mod.cc_grid(cb, dims, 6)
    v = np.arange(n)
    assert (lab[cb == 1] == v[cb == 1]).all() and (lab[cb == 0] == -1).all()
    slabs = (z % 2 == 0).astype(np.uint8).ravel()  # z = 0, 2: two slabs
    lab = oracle_mod.cc_grid(slabs, dims, 14)
    assert set(np.unique(lab[slabs == 1])) == {0, 60}
    assert (lab[(z == 2).ravel()] == 60).all()


def test_mesh_closed_forms(oracle_mod):
    row, col = workloads.tet_mesh_csr(edge=5, delete_frac=0.0, seed=0)
    assert (oracle_mod.cc_csr(row.numpy(), col.numpy()) == 0).all()
    row, col = workloads.tet_mesh_csr(edge=5, delete_frac=1.0, seed=0)
    assert (oracle_mod.cc_csr(row.numpy(), col.numpy()) == np.arange(125)).all()


def test_mesh_matches_union_find(oracle_mod):
    row, col = workloads.tet_mesh_csr(edge=9, delete_frac=0.75, seed=3)
    row, col = row.numpy(), col.numpy()
    n = row.size - 1
    src = np.repeat(np.arange(n), np.diff(row))
    got = oracle_mod.cc_csr(row, col)
    want = union_find_labels(np.ones(n, np.uint8), np.stack([src, col], 1))
    np.testing.assert_array_equal(got, want)


def test_mesh_csr_is_symmetric_and_sorted():
    row, col = workloads.tet_mesh_csr(edge=6, delete_frac=0.4, seed=3)
    row, col = row.numpy(), col.numpy()
    n = row.size - 1
    src = np.repeat(np.arange(n), np.diff(row))
    fwd = set(zip(src.tolist(), col.tolist()))
    assert fwd == {(b, a) for a, b in fwd}
    assert all(np.all(np.diff(col[row[v]:row[v + 1]]) > 0) for v in range(n))
    assert all(a != b for a, b in fwd)


def test_sampled_component_matches_full(oracle_mod):
    dims = (12, 11, 10)
    rng = np.random.default_rng(9)
    mask = (rng.random(1320) < 0.45).astype(np.uint8)
    for conn in (6, 14):
        lab = oracle_mod.cc_grid(mask, dims, conn)
        for v in rng.integers(0, 1320, 30):
            mn, size = oracle_mod.cc_grid_at(mask, dims, conn, int(v))
            assert mn == lab[v]
            assert size == (0 if lab[v] < 0 else int((lab == lab[v]).sum()))


# ---------------------------------------------------------------------------
# literal Alg. 3 (largest-id labels) on an explicit graph


def alg3_replay(n, nbrs, mask, iterate):
    d = np.full(n, -1, np.int64)
    for v in range(n):  # init: largest masked neighbour, or v itself
        if mask[v]:
            d[v] = max([v] + [u for u in nbrs[v] if mask[u]])

    def compress():
        changed = True
        while changed:
            changed = False
            for v in range(n):
                if d[v] >= 0 and d[d[v]] != d[v]:
                    d[v] = d[d[v]]
                    changed = True

    compress()
    while True:
        before = d.copy()
        for v in range(n):  # stitching: hook own root to a larger one
            if mask[v]:
                for u in nbrs[v]:
                    if mask[u] and d[u] > d[v]:
                        d[d[v]] = d[u]
        compress()
        if not iterate or np.array_equal(before, d):
            return d


def partition(labels):
    groups = {}
    for v, l in enumerate(labels):
        if l >= 0:
            groups.setdefault(int(l), set()).add(v)
    return sorted(map(sorted, groups.values()))


def test_alg3_single_stitch_can_split_a_component(oracle_mod):
    """Counter-example: the path 4-0-2-1-3.  After the first compression the
    segments are {4,0} (root 4), {2} (root 2) and {1,3} (root 3).  Root 2
    borders both larger segments; the in-place write "d[d[v]] <- d[u]" sends
    it to 4, after which the test "d[u] > d[v]" no longer fires for the
    neighbour in segment 3, so one stitching pass leaves {1,3} apart."""
    edges = [(4, 0), (0, 2), (2, 1), (1, 3)]
    n = 5
    nbrs = {v: [] for v in range(n)}
    for a, b in edges:
        nbrs[a].append(b)
        nbrs[b].append(a)
    mask = np.ones(n, bool)
    row = np.cumsum([0] + [len(nbrs[v]) for v in range(n)]).astype(np.int32)
    col = np.array([u for v in range(n) for u in sorted(nbrs[v])], np.int32)
    truth = partition(oracle_mod.cc_csr(row, col))
    assert truth == [list(range(n))]
    one = partition(alg3_replay(n, nbrs, mask, iterate=False))
    assert one == [[0, 2, 4], [1, 3]]  # the literal single pass splits it
    fixed = partition(alg3_replay(n, nbrs, mask, iterate=True))
    assert fixed == truth


@pytest.mark.parametrize("seed", range(4))
def test_alg3_fixed_point_partition_equals_bfs(oracle_mod, seed):
    dims = (7, 6, 5)
    n = 210
    rng = np.random.default_rng(seed)
    mask = rng.random(n) < 0.5
    edges = grid_edges(mask.astype(np.uint8), dims, 14)
    nbrs = {v: [] for v in range(n)}
    for a, b in edges:
        nbrs[int(a)].append(int(b))
        nbrs[int(b)].append(int(a))
    d = alg3_replay(n, nbrs, mask, iterate=True)
    lab = oracle_mod.cc_grid(mask.astype(np.uint8), dims, 14)
    assert partition(d) == partition(lab)
    # largest-id labels (paper) and smallest-id labels (here) name the same sets
    for v in range(n):
        if lab[v] >= 0:
            comp = np.nonzero(lab == lab[v])[0]
            assert d[v] == comp.max() and lab[v] == comp.min()


def test_mesh_components_match_networkx(oracle_mod):
    """The components of a thinned Kuhn mesh equal networkx's connected
    components (a library routine), with the smallest id as the label."""
    nx_ = pytest.importorskip("networkx")
    row, col = workloads.tet_mesh_csr(edge=10, delete_frac=0.5, seed=21)
    row, col = row.numpy(), col.numpy()
    n = row.size - 1
    g = nx_.Graph()
    g.add_nodes_from(range(n))
    for v in range(n):
        g.add_edges_from((v, int(u)) for u in col[row[v]:row[v + 1]])
    want = np.empty(n, np.int32)
    for comp in nx_.connected_components(g):
        want[list(comp)] = min(comp)
    np.testing.assert_array_equal(oracle_mod.cc_csr(row, col), want)


@pytest.mark.parametrize("conn", [6, 14])
def test_grid_components_match_networkx(oracle_mod, conn):
    nx_ = pytest.importorskip("networkx")
    dims = (9, 7, 5)
    rng = np.random.default_rng(conn)
    mask = (rng.random(9 * 7 * 5) < 0.45).astype(np.uint8)
    offs = [(1, 0, 0), (0, 1, 0), (0, 0, 1)] + ([(1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)] if conn == 14 else [])
    g = nx_.Graph()
    ids = [v for v in range(mask.size) if mask[v]]
    g.add_nodes_from(ids)
    for v in ids:
        x, y, z = v % 9, (v // 9) % 7, v // 63
        for dx, dy, dz in offs:
            if x + dx < 9 and y + dy < 7 and z + dz < 5:
                u = (x + dx) + 9 * ((y + dy) + 7 * (z + dz))
                if mask[u]:
                    g.add_edge(v, u)
    want = np.full(mask.size, -1, np.int32)
    for comp in nx_.connected_components(g):
        want[list(comp)] = min(comp)
    np.testing.assert_array_equal(oracle_mod.cc_grid(mask, dims, conn), want)
