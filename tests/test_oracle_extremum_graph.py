"""Pins of the oracle's extremum-graph arcs: pairs of maximum (minimum)
regions that touch, each with the end vertex of its highest (lowest)
crossing edge.

The pins do not use the oracle's offset table or its sort: on a line the
saddle of two neighbouring maxima is the minimum of f between them (a
closed form computed here from f alone); on small grids a brute force over
the edges of an explicit Kuhn split (or the face grid) and a random vertex
order gives every arc and saddle; the pairs equal the region adjacency."""
import numpy as np
import pytest

from test_oracle_adjacency import face_edges, kuhn_edges


def line_field(length, rng):
    """Distinct values on a line (a random permutation, so no ties)."""
    return rng.permutation(length).astype(np.float32)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("seed", range(5))
def test_saddles_on_a_line_are_the_valleys(oracle_mod, axis, seed):
    rng = np.random.default_rng(seed)
    L = 40
    dims = [1, 1, 1]
    dims[axis] = L
    dims = tuple(dims)
    step = [1, dims[0], dims[0] * dims[1]][axis]
    f = line_field(L, rng)
    order, asc, desc, ms, k = oracle_mod.segment_grid(f, dims)
    for sense, lab in ((1, desc), (-1, asc)):
        g = f if sense > 0 else -f
        # extrema of g on the line, from f alone
        peaks = [i for i in range(L) if (i == 0 or g[i] > g[i - 1]) and (i == L - 1 or g[i] > g[i + 1])]
        want = []
        for p, q in zip(peaks, peaks[1:]):
            valley = p + int(np.argmin(g[p:q + 1]))  # lowest point between two neighbouring peaks
            want.append((p * step, q * step, valley * step))
        for conn in (6, 14):
            a, b, s = oracle_mod.extremum_graph(lab, order, dims, conn, sense)
            assert list(zip(a.tolist(), b.tolist(), s.tolist())) == want


def brute_arcs(label, order, edges, sense):
    best = {}
    for u, v in edges:
        la, lb = int(label[u]), int(label[v])
        if la < 0 or lb < 0 or la == lb:
            continue
        lower, upper = (u, v) if order[u] < order[v] else (v, u)
        w = lower if sense > 0 else upper
        key = (min(la, lb), max(la, lb))
        if key not in best or (order[w] > order[best[key]] if sense > 0 else order[w] < order[best[key]]):
            best[key] = w
    keys = sorted(best)
    return [k[0] for k in keys], [k[1] for k in keys], [best[k] for k in keys]


@pytest.mark.parametrize("sense", [1, -1])
@pytest.mark.parametrize("conn", [6, 14])
@pytest.mark.parametrize("seed", range(5))
def test_random_labels_and_orders_match_brute_force(oracle_mod, sense, conn, seed):
    rng = np.random.default_rng(100 + seed)
    dims = tuple(int(x) for x in rng.integers(2, 7, 3))
    n = dims[0] * dims[1] * dims[2]
    lab = rng.integers(-1, 6, n).astype(np.int32)
    order = rng.permutation(n).astype(np.int32)
    a, b, s = oracle_mod.extremum_graph(lab, order, dims, conn, sense)
    wa, wb, ws = brute_arcs(lab, order, kuhn_edges(dims) if conn == 14 else face_edges(dims), sense)
    assert a.tolist() == wa and b.tolist() == wb and s.tolist() == ws


def test_arcs_are_the_region_adjacency_and_saddles_sit_below_both_maxima(oracle_mod):
    """Smooth field with several bumps: the arcs are exactly the adjacent
    pairs of maxima, every saddle lies in one of its two regions next to
    the other, and no saddle is higher than either of its maxima."""
    import workloads

    dims = (30, 24, 18)
    f = workloads.smooth_field(dims, 10, (3.0, 7.0), seed=12).reshape(-1).numpy()
    order, asc, desc, ms, k = oracle_mod.segment_grid(f, dims)
    for sense, lab in ((1, desc), (-1, asc)):
        a, b, s = oracle_mod.extremum_graph(lab, order, dims, 14, sense)
        pa, pb = oracle_mod.adjacency_grid(lab, dims, 14)
        np.testing.assert_array_equal(a, pa)
        np.testing.assert_array_equal(b, pb)
        assert a.size >= 2
        for x, y, w in zip(a, b, s):
            assert lab[w] in (x, y)
            if sense > 0:
                assert order[w] < min(order[x], order[y])
            else:
                assert order[w] > max(order[x], order[y])
