"""The OpenMP CPU baseline (the paper's shared-memory Alg. 1 and Alg. 3 on
all host cores) gives the oracle's results: it is a second, parallel
implementation of the same definitions, so the benchmark's CPU leg is
timed on correct work."""
import numpy as np
import pytest

import workloads
from oracle import paper_omp


@pytest.fixture(scope="module")
def po():
    paper_omp.build()
    return paper_omp


def test_runs_on_several_threads(po):
    assert po.threads() >= 1


@pytest.mark.parametrize("n", [1, 7, 4096, 300_007])
def test_order_with_ties_and_signed_zeros(po, oracle_mod, n):
    rng = np.random.default_rng(n)
    f = rng.integers(-50, 50, n).astype(np.float32) / 8
    f[::5] = -0.0
    f[1::7] = 0.0
    np.testing.assert_array_equal(po.order(f), oracle_mod.order(f))


def test_order_nan_is_an_error(po):
    f = np.zeros(100, np.float32)
    f[37] = np.nan
    with pytest.raises(paper_omp.BaselineError) as e:
        po.order(f)
    assert e.value.code == -4


def test_compress_reaches_every_root(po, oracle_mod):
    rng = np.random.default_rng(3)
    n = 200_000
    perm = rng.permutation(n)
    ptr = np.empty(n, np.int32)
    ptr[perm[0]] = perm[0]
    back = rng.integers(1, 4, n)
    for i in range(1, n):  # long chains through a random permutation
        ptr[perm[i]] = perm[max(0, i - back[i])]
    np.testing.assert_array_equal(po.compress(ptr), oracle_mod.walk_memo(ptr))


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 1, 7), (37, 29, 23), (64, 40, 33)])
def test_segment_smooth_equals_oracle(po, oracle_mod, dims):
    f = workloads.smooth_field(dims, 6, (2.0, 6.0), seed=sum(dims)).numpy().ravel()
    got = po.segment_grid(f, dims)
    want = oracle_mod.segment_grid(f, dims)
    for g, w in zip(got[:4], want[:4]):
        np.testing.assert_array_equal(g, w)
    assert got[4] == want[4]
    assert len(got[5]) == 4 and all(t >= 0 for t in got[5])


def test_segment_noise_with_ties_equals_oracle(po, oracle_mod):
    dims = (48, 40, 36)
    f = np.round(workloads.white_noise(dims, seed=1).numpy().ravel() * 256) / 256
    got = po.segment_grid(f.astype(np.float32), dims)
    want = oracle_mod.segment_grid(f.astype(np.float32), dims)
    for g, w in zip(got[:4], want[:4]):
        np.testing.assert_array_equal(g, w)
    assert got[4] == want[4]


@pytest.mark.parametrize("conn", [6, 14])
@pytest.mark.parametrize("density", [0.2, 0.5, 0.8])
def test_cc_grid_random_masks_equal_bfs(po, oracle_mod, conn, density):
    dims = (70, 19, 13)
    rng = np.random.default_rng(int(density * 10) + conn)
    mask = (rng.random(np.prod(dims)) < density).astype(np.uint8)
    np.testing.assert_array_equal(po.cc_grid(mask, dims, conn), oracle_mod.cc_grid(mask, dims, conn))


def test_cc_grid_blobs_and_closed_forms(po, oracle_mod):
    dims = (64, 48, 40)
    mask = workloads.feature_mask(dims, 20, (3.0, 8.0), 0.2, seed=5).numpy().ravel()
    np.testing.assert_array_equal(po.cc_grid(mask, dims, 6), oracle_mod.cc_grid(mask, dims, 6))
    ones = np.ones(np.prod(dims), np.uint8)
    assert (po.cc_grid(ones, dims, 14) == 0).all()
    z, y, x = np.meshgrid(*[np.arange(s) for s in dims[::-1]], indexing="ij")
    checker = ((x + y + z) % 2 == 0).astype(np.uint8).ravel()
    lab = po.cc_grid(checker, dims, 6)
    ids = np.arange(checker.size)
    assert (lab[checker == 1] == ids[checker == 1]).all() and (lab[checker == 0] == -1).all()


@pytest.mark.parametrize("frac", [0.0, 0.4, 0.9, 1.0])
def test_cc_csr_thinned_mesh_equals_bfs(po, oracle_mod, frac):
    row, col = workloads.tet_mesh_csr(edge=20, delete_frac=frac, seed=7)
    r, c = row.numpy(), col.numpy()
    np.testing.assert_array_equal(po.cc_csr(r, c), oracle_mod.cc_csr(r, c))


def test_cc_csr_long_rows_and_bad_column(po, oracle_mod):
    # a star: one vertex joined to every other (rows far longer than a mesh's)
    n = 1000
    a = np.concatenate([np.zeros(n - 1, np.int64), np.arange(1, n)])
    b = np.concatenate([np.arange(1, n), np.zeros(n - 1, np.int64)])
    order = np.lexsort((b, a))
    row = np.searchsorted(a[order], np.arange(n + 1)).astype(np.int32)
    col = b[order].astype(np.int32)
    assert (po.cc_csr(row, col) == 0).all()
    with pytest.raises(paper_omp.BaselineError):
        po.cc_csr(np.array([0, 1], np.int32), np.array([5], np.int32))
