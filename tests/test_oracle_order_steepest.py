"""Pins for the oracle's vertex order and steepest pointers.

Each check compares the oracle with something other than itself: counting
instead of sorting, neighbour sets taken from an explicit Kuhn tetrahedral
split instead of the offset table, exhaustive enumeration of every order of
tiny grids, closed forms (a monotone ramp, a single bump), and invariants of
the definitions (section "Ascending and Descending Manifolds").
"""
import itertools

import numpy as np
import pytest

import workloads


def count_order(f):
    """order[v] = #{u : (f[u], u) < (f[v], v)} by O(n^2) counting."""
    f = np.asarray(f, np.float32)
    ids = np.arange(f.size)
    less = (f[None, :] < f[:, None]) | ((f[None, :] == f[:, None]) & (ids[None, :] < ids[:, None]))
    return less.sum(axis=1).astype(np.int32)


@pytest.mark.parametrize("seed", range(4))
def test_order_matches_counting(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    f = rng.integers(-3, 4, size=777).astype(np.float32)  # heavy ties
    f[::17] = -0.0
    f[5] = np.inf
    f[9] = -np.inf
    o = oracle_mod.order(f)
    np.testing.assert_array_equal(o, count_order(f))
    assert np.array_equal(np.sort(o), np.arange(f.size))


def test_order_ties_and_signed_zero(oracle_mod):
    f = np.zeros(100, np.float32)
    np.testing.assert_array_equal(oracle_mod.order(f), np.arange(100))
    f[::2] = -0.0  # -0.0 == +0.0: the id alone decides
    np.testing.assert_array_equal(oracle_mod.order(f), np.arange(100))


def test_order_nan_is_an_error(oracle_mod):
    f = np.ones(10, np.float32)
    f[3] = np.nan
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.order(f)
    assert e.value.code == oracle_mod.ERR_NAN


def test_order_at_matches_order(oracle_mod):
    rng = np.random.default_rng(7)
    f = (rng.random(5000, dtype=np.float32) * 50).round()
    o = oracle_mod.order(f)
    for v in rng.integers(0, f.size, 40):
        assert oracle_mod.order_at(f, int(v)) == o[v]


# ---------------------------------------------------------------------------
# neighbour sets from an explicit Kuhn split (independent of the offset table)


def kuhn_neighbours(dims):
    nx, ny, nz = dims
    vid = lambda x, y, z: x + nx * (y + ny * z)  # noqa: E731
    nb = {v: set() for v in range(nx * ny * nz)}
    for z, y, x in itertools.product(range(nz - 1 if nz > 1 else 1), range(ny - 1 if ny > 1 else 1),
                                     range(nx - 1 if nx > 1 else 1)):
        # a degenerate axis of extent 1 keeps the tetrahedra's lower faces
        for p in itertools.permutations(range(3)):
            pts = [(x, y, z)]
            cur = [x, y, z]
            for a in p:
                cur = list(cur)
                cur[a] += 1
                pts.append(tuple(cur))
            ids = [vid(*q) for q in pts if q[0] < nx and q[1] < ny and q[2] < nz]
            for a, b in itertools.combinations(ids, 2):
                if a != b:
                    nb[a].add(b)
                    nb[b].add(a)
    return nb


def brute_steepest(order, nb):
    n = len(order)
    asc = np.arange(n, dtype=np.int32)
    desc = np.arange(n, dtype=np.int32)
    for v in range(n):
        for u in nb[v]:
            if order[u] > order[desc[v]]:
                desc[v] = u
            if order[u] < order[asc[v]]:
                asc[v] = u
    return asc, desc


def test_kuhn_neighbours_are_the_14_stencil():
    nb = kuhn_neighbours((5, 5, 5))
    centre = 2 + 5 * (2 + 5 * 2)
    got = sorted((u % 5 - 2, u // 5 % 5 - 2, u // 25 - 2) for u in nb[centre])
    want = sorted(tuple(s * c for c in o) for o in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0),
                                                    (1, 0, 1), (0, 1, 1), (1, 1, 1)] for s in (1, -1))
    assert want == got


@pytest.mark.parametrize("dims", [(2, 2, 2), (1, 2, 3), (3, 2, 1)])
def test_steepest_exhaustive_tiny(oracle_mod, dims):
    """Every order of a 2x2x2 (8! = 40320) and 1x2x3 / 3x2x1 (720) grid."""
    nb = kuhn_neighbours(dims)
    n = int(np.prod(dims))
    for perm in itertools.permutations(range(n)):
        order = np.array(perm, np.int32)
        asc, desc = oracle_mod.steepest_grid(order, dims)
        ba, bd = brute_steepest(order, nb)
        assert np.array_equal(asc, ba) and np.array_equal(desc, bd), perm


@pytest.mark.parametrize("dims", [(4, 3, 5), (6, 6, 6)])
def test_steepest_random_orders(oracle_mod, dims):
    nb = kuhn_neighbours(dims)
    rng = np.random.default_rng(3)
    n = int(np.prod(dims))
    for _ in range(50):
        order = rng.permutation(n).astype(np.int32)
        asc, desc = oracle_mod.steepest_grid(order, dims)
        ba, bd = brute_steepest(order, nb)
        np.testing.assert_array_equal(asc, ba)
        np.testing.assert_array_equal(desc, bd)


def test_ramp_has_one_cell(oracle_mod):
    dims = (7, 5, 4)
    z, y, x = np.meshgrid(*[np.arange(d) for d in dims[::-1]], indexing="ij")
    f = (x + 2 * y + 4 * z).astype(np.float32).ravel()
    o, asc, desc, ms, k = oracle_mod.segment_grid(f, dims)
    n = f.size
    assert (asc == 0).all() and (desc == n - 1).all()
    assert k == 1 and (ms == 0).all()


def test_single_bump_has_one_maximum(oracle_mod):
    dims = (17, 17, 17)
    f = workloads.gaussian_sum(dims, np.array([[8.0, 8.0, 8.0]]), np.array([4.0]), np.array([1.0]))
    o, asc, desc, ms, k = oracle_mod.segment_grid(f.numpy().ravel(), dims)
    centre = 8 + 17 * (8 + 17 * 8)
    assert (desc == centre).all()


def check_invariants(order, dims, asc_ptr, desc_ptr, asc, desc):
    nb = kuhn_neighbours(dims) if np.prod(dims) <= 4096 else None
    n = order.size
    v = np.arange(n)
    # labels are fixed points of themselves
    assert (desc[desc] == desc).all() and (asc[asc] == asc).all()
    assert (desc_ptr[desc] == desc).all() and (asc_ptr[asc] == asc).all()
    # order strictly increases along desc_ptr, decreases along asc_ptr
    moved = desc_ptr != v
    assert (order[desc_ptr[moved]] > order[v[moved]]).all()
    moved = asc_ptr != v
    assert (order[asc_ptr[moved]] < order[v[moved]]).all()
    # distinct labels = self-pointers
    assert np.unique(desc).size == int((desc_ptr == v).sum())
    assert np.unique(asc).size == int((asc_ptr == v).sum())
    if nb is not None:  # a label has no larger (smaller) neighbour
        for m in np.unique(desc):
            assert all(order[u] < order[m] for u in nb[int(m)])
        for m in np.unique(asc):
            assert all(order[u] > order[m] for u in nb[int(m)])


@pytest.mark.parametrize("edge", [12, 16])
def test_invariants_on_gaussian_field(oracle_mod, edge):
    dims = (edge, edge - 1, edge + 2)
    f = workloads.smooth_field(dims, 6, (1.5, 4.0), seed=edge, noise_amp=1e-3).numpy().ravel()
    order = oracle_mod.order(f)
    asc_ptr, desc_ptr = oracle_mod.steepest_grid(order, dims)
    asc = oracle_mod.walk(asc_ptr)
    desc = oracle_mod.walk(desc_ptr)
    check_invariants(order, dims, asc_ptr, desc_ptr, asc, desc)


def test_invariants_on_white_noise(oracle_mod):
    dims = (15, 13, 11)
    f = workloads.white_noise(dims, seed=5).numpy().ravel()
    f = np.round(f * 64) / 64  # many exact ties
    order = oracle_mod.order(f)
    asc_ptr, desc_ptr = oracle_mod.steepest_grid(order, dims)
    check_invariants(order, dims, asc_ptr, desc_ptr, oracle_mod.walk(asc_ptr), oracle_mod.walk(desc_ptr))


def test_sampled_helpers_match_full_arrays(oracle_mod):
    dims = (20, 18, 16)
    f = workloads.smooth_field(dims, 5, (2.0, 5.0), seed=11).numpy().ravel()
    f[::7] = 0.25  # ties resolved by id in both
    order = oracle_mod.order(f)
    asc_ptr, desc_ptr = oracle_mod.steepest_grid(order, dims)
    asc, desc = oracle_mod.walk(asc_ptr), oracle_mod.walk(desc_ptr)
    for v in np.random.default_rng(0).integers(0, f.size, 60):
        assert oracle_mod.steepest_at(f, dims, int(v)) == (asc_ptr[v], desc_ptr[v])
        assert oracle_mod.labels_at(f, dims, int(v)) == (asc[v], desc[v])


def test_order_matches_numpy_lexsort(oracle_mod):
    """At a size counting cannot reach: the rank under (f, id) from numpy's
    stable lexsort (a library routine), with heavy ties and signed zeros."""
    rng = np.random.default_rng(44)
    n = 200_003
    f = (rng.integers(-300, 300, n) / 8.0).astype(np.float32)
    f[::11] = -0.0
    f[5::13] = np.inf
    f[7::17] = -np.inf
    perm = np.lexsort((np.arange(n), f))  # sorted ids: by f, ties by id (-0.0 == +0.0)
    want = np.empty(n, np.int32)
    want[perm] = np.arange(n, dtype=np.int32)
    np.testing.assert_array_equal(oracle_mod.order(f), want)
