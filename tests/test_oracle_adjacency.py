"""Pins of the oracle's region adjacency (the pairs of labels that meet
across an edge of the triangulation or of the face grid).

The edges are taken here from an explicit construction -- the six
tetrahedra of the Kuhn split of every grid cube, or the three face
directions -- not from the oracle's offset table; closed forms and the
segmentation of a ramp pin the rest."""
import itertools

import numpy as np
import pytest


def kuhn_edges(dims):
    """All edges of the Kuhn triangulation of an nx x ny x nz grid (every
    extent at least 2), as (u, v) vertex-id pairs with u < v: every pair of
    vertices of every tetrahedron 0 -> e_a -> e_a + e_b -> (1,1,1) of every
    cube."""
    nx, ny, nz = dims
    step = [1, nx, nx * ny]
    edges = set()
    for z in range(nz - 1):
        for y in range(ny - 1):
            for x in range(nx - 1):
                base = x + nx * (y + ny * z)
                for p in itertools.permutations(range(3)):
                    v1 = base + step[p[0]]
                    v2 = v1 + step[p[1]]
                    v3 = v2 + step[p[2]]
                    for a, b in itertools.combinations((base, v1, v2, v3), 2):
                        edges.add((min(a, b), max(a, b)))
    return edges


def face_edges(dims):
    nx, ny, nz = dims
    edges = set()
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                v = x + nx * (y + ny * z)
                if x + 1 < nx:
                    edges.add((v, v + 1))
                if y + 1 < ny:
                    edges.add((v, v + nx))
                if z + 1 < nz:
                    edges.add((v, v + nx * ny))
    return edges


def brute_pairs(label, edges):
    out = set()
    for u, v in edges:
        a, b = int(label[u]), int(label[v])
        if a >= 0 and b >= 0 and a != b:
            out.add((min(a, b), max(a, b)))
    out = sorted(out)
    return np.array([p[0] for p in out], np.int32), np.array([p[1] for p in out], np.int32)


@pytest.mark.parametrize("dims", [(4, 3, 5), (6, 5, 4), (2, 2, 2), (7, 3, 3)])
def test_vertex_ids_as_labels_give_every_edge(oracle_mod, dims):
    n = dims[0] * dims[1] * dims[2]
    lab = np.arange(n, dtype=np.int32)
    a, b = oracle_mod.adjacency_grid(lab, dims, 14)
    got = set(zip(a.tolist(), b.tolist()))
    assert got == kuhn_edges(dims)
    a6, b6 = oracle_mod.adjacency_grid(lab, dims, 6)
    nx, ny, nz = dims
    assert a6.size == 3 * n - (ny * nz + nx * nz + nx * ny)  # edges of the face grid
    assert set(zip(a6.tolist(), b6.tolist())) == face_edges(dims)


@pytest.mark.parametrize("conn", [6, 14])
@pytest.mark.parametrize("seed", range(6))
def test_random_labels_match_brute_force(oracle_mod, conn, seed):
    rng = np.random.default_rng(seed)
    dims = tuple(int(x) for x in rng.integers(2, 7, 3))
    n = dims[0] * dims[1] * dims[2]
    lab = rng.integers(-1, 5, n).astype(np.int32)  # few labels, some vertices unlabelled
    a, b = oracle_mod.adjacency_grid(lab, dims, conn)
    wa, wb = brute_pairs(lab, kuhn_edges(dims) if conn == 14 else face_edges(dims))
    np.testing.assert_array_equal(a, wa)
    np.testing.assert_array_equal(b, wb)


def test_closed_forms(oracle_mod):
    dims = (10, 7, 6)
    n = 10 * 7 * 6
    for conn in (6, 14):
        assert oracle_mod.adjacency_grid(np.full(n, 3, np.int32), dims, conn)[0].size == 0
        assert oracle_mod.adjacency_grid(np.full(n, -1, np.int32), dims, conn)[0].size == 0
        x = np.arange(n) % 10
        halves = (x >= 5).astype(np.int32) * 7 + 2  # labels 2 and 9
        a, b = oracle_mod.adjacency_grid(halves, dims, conn)
        assert a.tolist() == [2] and b.tolist() == [9]
        # three slabs along z: 0-1 and 1-2 touch, 0-2 do not
        z = np.arange(n) // 70
        slabs = np.minimum(z // 2, 2).astype(np.int32)
        a, b = oracle_mod.adjacency_grid(slabs, dims, conn)
        assert list(zip(a.tolist(), b.tolist())) == [(0, 1), (1, 2)]


def test_ramp_segmentation_has_no_boundaries(oracle_mod):
    dims = (9, 8, 7)
    x, y, z = np.meshgrid(np.arange(9), np.arange(8), np.arange(7), indexing="ij")
    f = (x + 2 * y + 4 * z).transpose(2, 1, 0).astype(np.float32).ravel()
    order, asc, desc, ms, k = oracle_mod.segment_grid(f, dims)
    assert k == 1
    for lab in (asc, desc, ms):
        assert oracle_mod.adjacency_grid(lab, dims, 14)[0].size == 0


def test_two_bumps_give_adjacent_cells(oracle_mod):
    """Two Gaussian bumps: two maxima whose descending manifolds touch, and
    every cell pair reported is a pair of distinct existing cells."""
    dims = (24, 10, 10)
    x, y, z = np.meshgrid(np.arange(24), np.arange(10), np.arange(10), indexing="ij")
    f = np.exp(-((x - 5.0) ** 2 + (y - 5) ** 2 + (z - 5) ** 2) / 18.0) + \
        0.9 * np.exp(-((x - 18.0) ** 2 + (y - 4) ** 2 + (z - 5) ** 2) / 18.0) + 1e-3 * x
    f = f.transpose(2, 1, 0).astype(np.float32).ravel()
    order, asc, desc, ms, k = oracle_mod.segment_grid(f, dims)
    maxima = np.unique(desc)
    a, b = oracle_mod.adjacency_grid(desc, dims, 14)
    assert maxima.size >= 2 and a.size >= 1
    assert set(a.tolist()) | set(b.tolist()) <= set(maxima.tolist())
    assert (a < b).all()
    a, b = oracle_mod.adjacency_grid(ms, dims, 14)
    assert (a < b).all() and b.max() < k
