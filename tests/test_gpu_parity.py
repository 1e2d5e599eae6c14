"""GPU path vs the CPU oracle, element by element, through the C ABI.

Every output here is an integer (order ranks, vertex ids, cell ids, labels),
so the bar is bit-exact equality.  Sizes span several tiles and ragged
tails (dimensions that are not multiples of the 32x8x8 / 64x8x8 tiles, n
not a multiple of 4 or of the 4096-key sort tile), degenerate grids, and
both the TMA (nx % 4 == 0) and plain-load stencil paths.
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import paper_2409_03771_gb300 as msc
    from paper_2409_03771_gb300 import _build

    _build.build()
    msc.load()
    return msc


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


# ---------------------------------------------------------------------------
# order


@pytest.mark.parametrize("n", [1, 2, 3, 4095, 4096, 4097, 70001, 262144 + 13])
def test_order_random_with_ties(m, oracle_mod, n):
    rng = np.random.default_rng(n)
    f = rng.integers(-50, 50, n).astype(np.float32) / 8
    f[rng.random(n) < 0.1] = -0.0
    if n > 10:
        f[3] = np.inf
        f[7] = -np.inf
    np.testing.assert_array_equal(host(m.order(cuda(f))), oracle_mod.order(f))


def test_order_config_small_field(m, oracle_mod):
    f = workloads.field_small().numpy().ravel()
    np.testing.assert_array_equal(host(m.order(cuda(f))), oracle_mod.order(f))


def test_order_all_equal_is_identity(m):
    n = 50000
    np.testing.assert_array_equal(host(m.order(torch.zeros(n, device="cuda"))), np.arange(n))


def test_order_nan_sets_status(m):
    f = torch.rand(10000, device="cuda")
    f[777] = float("nan")
    with pytest.raises(m.MSCError) as e:
        m.order(f)
    assert e.value.code == m.ERR_NAN


def test_order_unaligned_input(m, oracle_mod):
    f = np.random.default_rng(1).random(9001, dtype=np.float32)
    t = cuda(np.concatenate([[0.0], f]).astype(np.float32))[1:]  # 4-byte aligned only
    np.testing.assert_array_equal(host(m.order(t)), oracle_mod.order(f))


# ---------------------------------------------------------------------------
# steepest pointers

GRIDS = [(64, 64, 64), (37, 29, 23), (33, 8, 9), (4, 1, 1), (1, 1, 1), (128, 17, 5), (1, 50, 40),
         (40, 1, 33), (32, 8, 8), (36, 10, 10), (96, 24, 16)]


@pytest.mark.parametrize("dims", GRIDS)
def test_steepest_grid(m, oracle_mod, dims):
    n = int(np.prod(dims))
    order = np.random.default_rng(n).permutation(n).astype(np.int32)
    asc, desc = m.steepest_grid(cuda(order), dims)
    oa, od = oracle_mod.steepest_grid(order, dims)
    np.testing.assert_array_equal(host(desc), od)
    np.testing.assert_array_equal(host(asc), oa)


def test_steepest_grid_smooth_order(m, oracle_mod):
    dims = (64, 64, 64)
    order = oracle_mod.order(workloads.field_small().numpy().ravel())
    asc, desc = m.steepest_grid(cuda(order), dims)
    oa, od = oracle_mod.steepest_grid(order, dims)
    np.testing.assert_array_equal(host(desc), od)
    np.testing.assert_array_equal(host(asc), oa)


@pytest.mark.parametrize("edge,frac", [(12, 0.4), (9, 0.0), (7, 1.0)])
def test_steepest_csr(m, oracle_mod, edge, frac):
    row, col = workloads.tet_mesh_csr(edge=edge, delete_frac=frac, seed=3)
    n = row.numel() - 1
    order = np.random.default_rng(edge).permutation(n).astype(np.int32)
    asc, desc = m.steepest_csr(cuda(order), row.cuda(), col.cuda())
    oa, od = oracle_mod.steepest_csr(order, row.numpy(), col.numpy())
    np.testing.assert_array_equal(host(desc), od)
    np.testing.assert_array_equal(host(asc), oa)


def test_steepest_csr_bad_column(m):
    row = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
    col = torch.tensor([1, 5], dtype=torch.int32, device="cuda")
    with pytest.raises(m.MSCError) as e:
        m.steepest_csr(torch.tensor([0, 1], dtype=torch.int32, device="cuda"), row, col)
    assert e.value.code == m.ERR_ARG


# ---------------------------------------------------------------------------
# path compression


def forest(n, rng, roots, span):
    perm = rng.permutation(n)
    ptr = np.empty(n, np.int32)
    ptr[perm[:roots]] = perm[:roots]
    for i in range(roots, n):
        ptr[perm[i]] = perm[rng.integers(max(0, i - span), i)]
    return ptr


@pytest.mark.parametrize("n,roots,span", [(1, 1, 1), (5, 1, 1), (4097, 3, 10), (300001, 5, 2),
                                          (1 << 20, 1, 1)])
def test_compress_forests(m, oracle_mod, n, roots, span):
    ptr = forest(n, np.random.default_rng(n), roots, span)  # span 1: one long chain
    np.testing.assert_array_equal(host(m.compress(cuda(ptr))), oracle_mod.walk_memo(ptr))


def test_compress_active_list_overflow_falls_back(m, oracle_mod):
    """30 % roots and 70 % of the vertices on 70 chains of 10 000: the first
    sweep moves 70 %, which is under 1.5x the list's capacity (n/2), so the
    second sweep builds a list; it moves nearly all of them again, more than
    the list holds, so the third sweep must walk every vertex.  The per-sweep
    counts the call leaves in its workspace show that path was taken."""
    n = 1_000_000
    rng = np.random.default_rng(11)
    perm = rng.permutation(n).astype(np.int32)
    ptr = np.empty(n, np.int32)
    roots = perm[:300_000]
    ptr[roots] = roots
    chains = perm[300_000:].reshape(70, 10_000)
    ptr[chains[:, 0]] = roots[:70]
    ptr[chains[:, 1:]] = chains[:, :-1]
    p = cuda(ptr)
    ws = torch.zeros(m.msc_workspace_bytes(m.OP_COMPRESS, n), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert m.msc_compress(p, n, ws, ws.numel(), st) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    cnt = ws[:256].view(torch.int32).cpu().tolist()
    assert 500_001 < cnt[0] <= 750_001 and cnt[1] > 500_001  # built at sweep 1, overflowed
    np.testing.assert_array_equal(host(p), oracle_mod.walk_memo(ptr))


def test_compress_keeps_inactive(m, oracle_mod):
    rng = np.random.default_rng(5)
    ptr = forest(100003, rng, 50, 100)
    # deactivate whole trees: vertices whose root is odd
    root = oracle_mod.walk_memo(ptr)
    ptr[root % 2 == 1] = -1
    np.testing.assert_array_equal(host(m.compress(cuda(ptr))), oracle_mod.walk(ptr))


def test_compress_cycle_is_reported(m):
    ptr = torch.arange(1, 1001, dtype=torch.int32, device="cuda")
    ptr[-1] = 0  # one big cycle
    with pytest.raises(m.MSCError) as e:
        m.compress(ptr)
    assert e.value.code == m.ERR_NOT_CONVERGED


@pytest.mark.parametrize("cycle", [[1, 0], [1, 2, 0], [0, 2, 3, 1], [1, 2, 3, 4, 5, 6, 7, 0]])
def test_compress_short_cycles_are_reported(m, cycle):
    """In-place jumping can collapse a cycle into a self-loop; still an error."""
    ptr = torch.tensor(cycle, dtype=torch.int32, device="cuda")
    with pytest.raises(m.MSCError) as e:
        m.compress(ptr)
    assert e.value.code == m.ERR_NOT_CONVERGED


def test_compress_bad_pointer_is_reported(m):
    ptr = torch.tensor([0, 0, 7, 2], dtype=torch.int32, device="cuda")
    with pytest.raises(m.MSCError) as e:
        m.compress(ptr)
    assert e.value.code == m.ERR_ARG


# ---------------------------------------------------------------------------
# Morse-Smale ids


@pytest.mark.parametrize("n,nmin,nmax", [(1, 1, 1), (1000, 3, 7), (200003, 40, 900), (65536, 5000, 6000),
                                         # tables past 2^20 slots: ranks by chunks of minimum ids,
                                         # and the sort when a chunk or one minimum has too many pairs
                                         (2_000_003, 300_000, 300_000), (2_000_003, 50, 200_000),
                                         (1_500_007, 3, 1_000_000)])
def test_ms_id(m, oracle_mod, n, nmin, nmax):
    rng = np.random.default_rng(n + nmin)
    ids = rng.permutation(n)
    mins, maxs = ids[:nmin], ids[-nmax:] if nmax <= n - nmin else ids[:nmax]
    asc = rng.choice(mins, n).astype(np.int32)
    desc = rng.choice(maxs, n).astype(np.int32)
    asc[mins] = mins  # labels label themselves
    desc[maxs] = maxs
    ms, k = m.ms_id(cuda(asc), cuda(desc))
    oms, ok = oracle_mod.ms(asc, desc)
    assert k == ok
    np.testing.assert_array_equal(host(ms), oms)


def test_ms_id_rejects_inconsistent_labels(m):
    asc = torch.tensor([1, 2, 0], dtype=torch.int32, device="cuda")  # label 1 does not label itself
    desc = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(m.MSCError) as e:
        m.ms_id(asc, desc)
    assert e.value.code == m.ERR_ARG


# ---------------------------------------------------------------------------
# full segmentation


def check_segment(m, oracle_mod, f, dims):
    o, a, d, ms, k = m.segment(cuda(f), dims)
    oo, oa, od, oms, ok = oracle_mod.segment_grid(f, dims)
    np.testing.assert_array_equal(host(o), oo)
    np.testing.assert_array_equal(host(a), oa)
    np.testing.assert_array_equal(host(d), od)
    assert k == ok
    np.testing.assert_array_equal(host(ms), oms)


def test_segment_small_config(m, oracle_mod):
    """64^3, 8 Gaussians sigma 4..12 + U[0, 1e-3] noise, seed 0."""
    check_segment(m, oracle_mod, workloads.field_small().numpy().ravel(), (64, 64, 64))


@pytest.mark.parametrize("dims", [(37, 29, 23), (1, 1, 1), (5, 1, 7), (64, 40, 33)])
def test_segment_ragged_smooth(m, oracle_mod, dims):
    f = workloads.smooth_field(dims, 6, (2.0, 6.0), seed=sum(dims)).numpy().ravel()
    check_segment(m, oracle_mod, f, dims)


@pytest.mark.parametrize("dims", [(48, 40, 36), (31, 33, 35)])
def test_segment_white_noise_with_ties(m, oracle_mod, dims):
    f = workloads.white_noise(dims, seed=1).numpy().ravel()
    f = np.round(f * 256) / 256  # massive ties: the id decides
    check_segment(m, oracle_mod, f.astype(np.float32), dims)


def test_segment_ramp_is_one_cell(m):
    dims = (40, 24, 16)
    z, y, x = torch.meshgrid(*[torch.arange(s) for s in dims[::-1]], indexing="ij")
    f = (x + 2 * y + 4 * z).float().cuda()
    o, a, d, ms, k = m.segment(f, dims)
    n = f.numel()
    assert k == 1 and bool((a == 0).all()) and bool((d == n - 1).all()) and bool((ms == 0).all())


def test_segment_repeatable(m):
    f = workloads.field_noise(edge=48, seed=3).cuda()
    r1 = m.segment(f, (48, 48, 48))
    r2 = m.segment(f, (48, 48, 48))
    for x, y in zip(r1[:4], r2[:4]):
        assert torch.equal(x, y)
    assert r1[4] == r2[4]


# ---------------------------------------------------------------------------
# connected components


CC_GRIDS = [(64, 8, 8), (70, 19, 13), (1, 1, 1), (3, 100, 2), (128, 16, 24), (65, 9, 9)]


@pytest.mark.parametrize("conn", [6, 14])
@pytest.mark.parametrize("dims", CC_GRIDS)
@pytest.mark.parametrize("density", [0.3, 0.6])
def test_cc_mask_random(m, oracle_mod, conn, dims, density):
    n = int(np.prod(dims))
    mask = (np.random.default_rng(n + conn).random(n) < density).astype(np.uint8)
    got = host(m.cc_mask(cuda(mask), dims, conn))
    np.testing.assert_array_equal(got, oracle_mod.cc_grid(mask, dims, conn))


@pytest.mark.parametrize("conn", [6, 14])
def test_cc_mask_blobs(m, oracle_mod, conn):
    dims = (128, 128, 128)
    mask = workloads.mask_blobs(edge=128, seed=2).numpy().ravel()
    got = host(m.cc_mask(cuda(mask), dims, conn))
    np.testing.assert_array_equal(got, oracle_mod.cc_grid(mask, dims, conn))


def test_cc_mask_closed_forms(m):
    dims = (66, 20, 18)
    n = int(np.prod(dims))
    assert bool((m.cc_mask(torch.ones(n, dtype=torch.uint8, device="cuda"), dims, 6) == 0).all())
    assert bool((m.cc_mask(torch.zeros(n, dtype=torch.uint8, device="cuda"), dims, 14) == -1).all())
    z, y, x = np.meshgrid(*[np.arange(s) for s in dims[::-1]], indexing="ij")
    cb = ((x + y + z) % 2 == 0).astype(np.uint8).ravel()
    lab = host(m.cc_mask(cuda(cb), dims, 6))
    v = np.arange(n)
    assert (lab[cb == 1] == v[cb == 1]).all() and (lab[cb == 0] == -1).all()


def test_cc_mask_spiral(m, oracle_mod):
    """A long snake crossing many tiles: many hooks along one component."""
    dims = (96, 48, 20)
    nx, ny, nz = dims
    mask = np.zeros((nz, ny, nx), np.uint8)
    for z in range(0, nz, 2):
        for y in range(0, ny, 2):
            mask[z, y, :] = 1
            xe = nx - 1 if (y // 2) % 2 == 0 else 0
            if y + 2 < ny:
                mask[z, y + 1, xe] = 1
        if z + 2 < nz:
            mask[z + 1, ny - 2 if (ny // 2) % 2 == 0 else ny - 2, 0] = 1
    mask = mask.ravel()
    got = host(m.cc_mask(cuda(mask), dims, 6))
    np.testing.assert_array_equal(got, oracle_mod.cc_grid(mask, dims, 6))


@pytest.mark.parametrize("edge,frac", [(24, 0.4), (16, 0.8), (9, 0.0), (7, 1.0), (20, 0.65)])
def test_cc_mesh(m, oracle_mod, edge, frac):
    row, col = workloads.tet_mesh_csr(edge=edge, delete_frac=frac, seed=edge)
    got = host(m.cc_mesh(row.cuda(), col.cuda()))
    np.testing.assert_array_equal(got, oracle_mod.cc_csr(row.numpy(), col.numpy()))


def test_cc_mesh_bad_column(m):
    row = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
    col = torch.tensor([1, 9], dtype=torch.int32, device="cuda")
    with pytest.raises(m.MSCError) as e:
        m.cc_mesh(row, col)
    assert e.value.code == m.ERR_ARG


# ---------------------------------------------------------------------------
# Sizes large enough that every persistent kernel's CTAs loop over many tiles
# (the sort takes ~1000 tiles of 4096 keys, the stencil ~2000 tiles, the CC
# kernels ~1000 tiles): state carried from one tile to the next is exercised.


def test_order_many_tiles_per_block(m, oracle_mod):
    rng = np.random.default_rng(11)
    n = 4_000_037
    f = (rng.standard_normal(n) * 3).astype(np.float32).round(2)  # ties
    np.testing.assert_array_equal(host(m.order(cuda(f))), oracle_mod.order(f))


def test_segment_many_tiles_smooth(m, oracle_mod):
    dims = (160, 160, 160)
    f = workloads.smooth_field(dims, 24, (8.0, 24.0), seed=21).numpy().ravel()
    check_segment(m, oracle_mod, f, dims)


def test_segment_many_tiles_noise(m, oracle_mod):
    dims = (168, 150, 144)
    f = workloads.white_noise(dims, seed=22).numpy().ravel()
    check_segment(m, oracle_mod, f, dims)


def test_compress_many_chunks(m, oracle_mod):
    ptr = forest(3_000_017, np.random.default_rng(12), 100, 1000)
    np.testing.assert_array_equal(host(m.compress(cuda(ptr))), oracle_mod.walk_memo(ptr))


@pytest.mark.parametrize("conn", [6, 14])
def test_cc_mask_many_tiles(m, oracle_mod, conn):
    dims = (256, 128, 128)
    mask = workloads.feature_mask(dims, 40, (6.0, 20.0), 0.2, seed=23).numpy().ravel()
    got = host(m.cc_mask(cuda(mask), dims, conn))
    np.testing.assert_array_equal(got, oracle_mod.cc_grid(mask, dims, conn))


def test_cc_mesh_large(m, oracle_mod):
    row, col = workloads.tet_mesh_csr(edge=96, delete_frac=0.55, seed=24)
    got = host(m.cc_mesh(row.cuda(), col.cuda()))
    np.testing.assert_array_equal(got, oracle_mod.cc_csr(row.numpy(), col.numpy()))


# ---------------------------------------------------------------------------
# caller buffers at any 4-byte alignment (views into larger arrays)


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_outputs_at_unaligned_addresses(m, oracle_mod, shift):
    """Every output pointer offset by 1-3 elements from a 16-byte boundary:
    the vector paths must fall back, and the results stay exact."""
    dims = (36, 20, 17)
    n = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(shift)
    f = rng.random(n, dtype=np.float32)
    fbuf = torch.zeros(n + shift, device="cuda")
    fbuf[shift:] = cuda(f)
    bufs = [torch.full((n + shift,), -7, dtype=torch.int32, device="cuda") for _ in range(4)]
    outs = [b[shift:] for b in bufs]
    k = torch.zeros(shift + 1, dtype=torch.int32, device="cuda")[shift:]
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(m.msc_workspace_bytes(m.OP_SEGMENT, n), dtype=torch.uint8, device="cuda")
    assert m.msc_segment(fbuf[shift:], dims, *outs, k, ws, ws.numel(), st) == m.OK
    torch.cuda.synchronize()
    assert int(st.item()) == m.OK
    wo, wa, wd, wm, wk = oracle_mod.segment_grid(f, dims)
    for got, want in zip(outs, (wo, wa, wd, wm)):
        np.testing.assert_array_equal(host(got), want)
    assert int(k.item()) == wk
    # the order alone, into an unaligned view as well
    ows = torch.empty(m.msc_workspace_bytes(m.OP_ORDER, n), dtype=torch.uint8, device="cuda")
    obuf = torch.full((n + shift,), -7, dtype=torch.int32, device="cuda")
    assert m.msc_order(fbuf[shift:], n, obuf[shift:], ows, ows.numel(), st) == m.OK
    np.testing.assert_array_equal(host(obuf[shift:]), wo)
