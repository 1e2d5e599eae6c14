"""Region adjacency on the GPU (msc_adjacency_grid) against the oracle:
random labels on grids that span several 32 x 8 x 4 tiles with ragged
tails, every edge of the grid (labels = vertex ids), the minimum / maximum
labels and cell ids of segmentations computed by the oracle, component
labels, thin grids, truncation at the capacity and the error cases.  At the
full size the result is compared with plain PyTorch set operations over
every edge of the grid."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

POS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


@pytest.fixture(scope="module")
def m():
    import paper_2409_03771_gb300 as msc
    from paper_2409_03771_gb300 import _build

    _build.build()
    msc.load()
    return msc


def gpu_pairs(m, lab, dims, conn, bound=None):
    a, b = m.adjacency_grid(torch.as_tensor(lab).cuda(), dims, conn, label_bound=bound)
    return a.cpu().numpy(), b.cpu().numpy()


def check(m, oracle_mod, lab, dims, conn, bound=None):
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    wa, wb = oracle_mod.adjacency_grid(lab, dims, conn)
    ga, gb = gpu_pairs(m, lab, dims, conn, bound)
    np.testing.assert_array_equal(ga, wa)
    np.testing.assert_array_equal(gb, wb)
    return wa.size


@pytest.mark.parametrize("conn", [6, 14])
@pytest.mark.parametrize("dims", [(70, 19, 11), (33, 9, 5), (31, 7, 3), (96, 40, 9)])
def test_random_labels(m, oracle_mod, dims, conn):
    rng = np.random.default_rng(dims[0] + conn)
    n = dims[0] * dims[1] * dims[2]
    lab = rng.integers(-1, 40, n).astype(np.int32)
    k = check(m, oracle_mod, lab, dims, conn, bound=40)
    assert k > 100
    check(m, oracle_mod, lab, dims, conn)  # loose bound: wider keys, same pairs


@pytest.mark.parametrize("conn", [6, 14])
def test_every_edge_is_a_pair(m, oracle_mod, conn):
    dims = (37, 9, 6)
    n = 37 * 9 * 6
    k = check(m, oracle_mod, np.arange(n, dtype=np.int32), dims, conn)
    edges6 = 3 * n - (9 * 6 + 37 * 6 + 37 * 9)
    assert k == edges6 if conn == 6 else k > 2 * edges6


@pytest.mark.parametrize("dims", [(1, 1, 1), (50, 1, 1), (1, 1, 50), (1, 40, 1), (7, 1, 9), (1, 13, 5), (2, 2, 2)])
def test_thin_grids(m, oracle_mod, dims):
    n = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(n)
    for conn in (6, 14):
        check(m, oracle_mod, rng.integers(-1, 6, n).astype(np.int32), dims, conn, bound=6)
        check(m, oracle_mod, np.arange(n, dtype=np.int32), dims, conn)


def test_constant_and_unlabelled(m):
    dims = (40, 20, 10)
    n = 8000
    for lab in (np.full(n, 5, np.int32), np.full(n, -1, np.int32), np.full(n, -7, np.int32)):
        for conn in (6, 14):
            a, b = gpu_pairs(m, lab, dims, conn)
            assert a.size == 0 and b.size == 0


@pytest.mark.parametrize("kind,edge", [("smooth", 64), ("noise", 40)])
def test_segmentation_labels(m, oracle_mod, kind, edge):
    """The Morse-Smale preview: pairs of minima, of maxima and of cells that
    touch, for labels the oracle computed."""
    dims = (edge, edge + 3, edge - 5)  # ragged against every tile extent
    n = dims[0] * dims[1] * dims[2]
    if kind == "smooth":
        f = workloads.smooth_field(dims, 12, (3.0, 9.0), seed=4).reshape(-1).numpy()
    else:
        f = workloads.white_noise(dims, seed=4).reshape(-1).numpy()
    order, asc, desc, ms, cells = oracle_mod.segment_grid(f, dims)
    for lab, bound in ((asc, n), (desc, n), (ms, cells)):
        for conn in (14, 6):
            k = check(m, oracle_mod, lab, dims, conn, bound=bound)
            assert k > 0


def test_component_labels(m, oracle_mod):
    """Components of one connectivity never touch under it; under the wider
    triangulation link, 6-components can meet across diagonals."""
    dims = (60, 45, 30)
    mask = workloads.feature_mask(dims, 20, (2.0, 5.0), 0.2, seed=9).reshape(-1).numpy()
    lab6 = oracle_mod.cc_grid(mask, dims, 6)
    lab14 = oracle_mod.cc_grid(mask, dims, 14)
    assert check(m, oracle_mod, lab6, dims, 6) == 0
    assert check(m, oracle_mod, lab14, dims, 14) == 0
    check(m, oracle_mod, lab6, dims, 14)


def test_capacity_truncates_and_counts(m, oracle_mod):
    dims = (50, 30, 20)
    n = 30000
    lab = np.random.default_rng(1).integers(0, 300, n).astype(np.int32)
    wa, wb = oracle_mod.adjacency_grid(lab, dims, 14)
    K = wa.size
    d = torch.as_tensor(lab).cuda()
    ws = torch.empty(m.msc_workspace_bytes(m.OP_ADJACENCY, n), dtype=torch.uint8, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    k = torch.empty(1, dtype=torch.int64, device="cuda")
    for cap in (0, 1, K // 3, K, K + 5):
        a = torch.full((cap + 8,), -5, dtype=torch.int32, device="cuda")
        b = torch.full((cap + 8,), -5, dtype=torch.int32, device="cuda")
        assert m.msc_adjacency_grid(d, dims, 14, 300, a, b, cap, k, ws, ws.numel(), st) == m.OK
        torch.cuda.synchronize()
        assert int(st.item()) == m.OK and int(k.item()) == K
        c = min(cap, K)
        np.testing.assert_array_equal(a[:c].cpu().numpy(), wa[:c])
        np.testing.assert_array_equal(b[:c].cpu().numpy(), wb[:c])
        assert bool((a[c:] == -5).all()) and bool((b[c:] == -5).all()), "written past the capacity"
    # the binding grows its buffer when the first capacity is too small
    a, b = m.adjacency_grid(d, dims, 14, label_bound=300, cap=7)
    np.testing.assert_array_equal(a.cpu().numpy(), wa)


def test_label_at_bound_is_an_error(m):
    dims = (20, 10, 10)
    lab = torch.zeros(2000, dtype=torch.int32, device="cuda")
    lab[1234] = 50
    with pytest.raises(m.MSCError) as e:
        m.adjacency_grid(lab, dims, 14, label_bound=50)
    assert e.value.code == m.ERR_ARG
    a, b = m.adjacency_grid(lab, dims, 14, label_bound=51)
    assert a.tolist() == [0] and b.tolist() == [50]


def torch_pairs(lab, dims, conn, shift):
    """Plain PyTorch: every edge's (lo << shift) | hi, de-duplicated and sorted."""
    nx, ny, nz = dims
    L = lab.reshape(nz, ny, nx).long()
    keys = []
    for dx, dy, dz in POS[: 3 if conn == 6 else 7]:
        A = L[: nz - dz, : ny - dy, : nx - dx]
        B = L[dz:, dy:, dx:]
        on = (A >= 0) & (B >= 0) & (A != B)
        lo = torch.minimum(A, B)[on]
        hi = torch.maximum(A, B)[on]
        keys.append((lo << shift) | hi)
        del A, B, on, lo, hi
    return torch.unique(torch.cat(keys))


@pytest.mark.parametrize("kind", ["smooth", "noise"])
def test_full_size_512(m, kind):
    """512^3 segmentations (the benchmarked size): the cell adjacency and the
    maximum adjacency equal the set of pairs over every edge."""
    E = 512
    dims = (E, E, E)
    f = (workloads.field_smooth(edge=E, seed=1, device="cuda") if kind == "smooth"
         else workloads.field_noise(edge=E, seed=1, device="cuda")).reshape(-1)
    order, asc, desc, ms, cells = m.segment(f, dims)
    del order, asc, f
    torch.cuda.empty_cache()
    n = E ** 3
    for lab, bound in ((desc, n), (ms, cells)):
        shift = max(int(bound - 1).bit_length(), 0)
        a, b = m.adjacency_grid(lab, dims, 14, label_bound=bound)
        want = torch_pairs(lab, dims, 14, shift)
        assert a.numel() == want.numel()
        got = (a.long() << shift) | b.long()
        assert torch.equal(got, want)
        del a, b, want, got
        torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# extremum graph: arcs with their saddles (msc_extremum_graph)


def check_graph(m, oracle_mod, lab, order, dims, conn, sense, bound=None):
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    order = np.ascontiguousarray(order, dtype=np.int32)
    wa, wb, ws = oracle_mod.extremum_graph(lab, order, dims, conn, sense)
    a, b, s = m.extremum_graph(torch.as_tensor(lab).cuda(), torch.as_tensor(order).cuda(), dims, sense, conn,
                               label_bound=bound)
    np.testing.assert_array_equal(a.cpu().numpy(), wa)
    np.testing.assert_array_equal(b.cpu().numpy(), wb)
    np.testing.assert_array_equal(s.cpu().numpy(), ws)
    return wa.size


@pytest.mark.parametrize("sense", [1, -1])
@pytest.mark.parametrize("conn", [6, 14])
@pytest.mark.parametrize("dims", [(70, 19, 11), (33, 9, 40), (5, 3, 70)])
def test_graph_random_labels_and_orders(m, oracle_mod, dims, conn, sense):
    rng = np.random.default_rng(dims[2] + conn + sense)
    n = dims[0] * dims[1] * dims[2]
    lab = rng.integers(-1, 30, n).astype(np.int32)
    order = rng.permutation(n).astype(np.int32)
    assert check_graph(m, oracle_mod, lab, order, dims, conn, sense, bound=30) > 50


@pytest.mark.parametrize("kind,edge", [("smooth", 64), ("noise", 40)])
def test_graph_of_segmentations(m, oracle_mod, kind, edge):
    """Maxima joined through their highest boundary crossing and minima
    through their lowest, for the oracle's own segmentations."""
    dims = (edge, edge + 3, edge - 5)
    if kind == "smooth":
        f = workloads.smooth_field(dims, 12, (3.0, 9.0), seed=4).reshape(-1).numpy()
    else:
        f = workloads.white_noise(dims, seed=4).reshape(-1).numpy()
    order, asc, desc, ms, cells = oracle_mod.segment_grid(f, dims)
    for conn in (14, 6):
        assert check_graph(m, oracle_mod, desc, order, dims, conn, 1) > 0
        assert check_graph(m, oracle_mod, asc, order, dims, conn, -1) > 0


def test_graph_on_a_line(m, oracle_mod):
    dims = (1, 1, 300)
    f = np.random.default_rng(5).permutation(300).astype(np.float32)
    order, asc, desc, ms, cells = oracle_mod.segment_grid(f, dims)
    assert check_graph(m, oracle_mod, desc, order, dims, 14, 1) > 10
    assert check_graph(m, oracle_mod, asc, order, dims, 6, -1) > 10


def test_graph_capacity(m, oracle_mod):
    dims = (50, 30, 20)
    n = 30000
    rng = np.random.default_rng(2)
    lab = rng.integers(0, 200, n).astype(np.int32)
    order = rng.permutation(n).astype(np.int32)
    wa, wb, ws = oracle_mod.extremum_graph(lab, order, dims, 14, 1)
    K = wa.size
    d, o = torch.as_tensor(lab).cuda(), torch.as_tensor(order).cuda()
    ws_t = torch.empty(m.msc_workspace_bytes(m.OP_EXTREMUM_GRAPH, n), dtype=torch.uint8, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    k = torch.empty(1, dtype=torch.int64, device="cuda")
    for cap in (0, K // 2, K):
        a, b, s = (torch.full((cap + 4,), -5, dtype=torch.int32, device="cuda") for _ in range(3))
        assert m.msc_extremum_graph(d, o, dims, 14, 200, 1, a, b, s, cap, k, ws_t, ws_t.numel(), st) == m.OK
        torch.cuda.synchronize()
        assert int(st.item()) == m.OK and int(k.item()) == K
        np.testing.assert_array_equal(s[:cap].cpu().numpy(), ws[:cap])
        assert bool((s[cap:] == -5).all())


def torch_graph(lab, order, dims, sense, shift):
    """Plain PyTorch: per pair key, the best crossing (level << 32 | vertex)."""
    nx, ny, nz = dims
    L = lab.reshape(nz, ny, nx).long()
    O = order.reshape(nz, ny, nx).long()
    ids = torch.arange(nx * ny * nz, device=lab.device).reshape(nz, ny, nx)
    keys, vals = [], []
    for dx, dy, dz in POS:
        sl_a = (slice(0, nz - dz), slice(0, ny - dy), slice(0, nx - dx))
        sl_b = (slice(dz, nz), slice(dy, ny), slice(dx, nx))
        A, B = L[sl_a], L[sl_b]
        on = (A >= 0) & (B >= 0) & (A != B)
        oa, ob = O[sl_a][on], O[sl_b][on]
        ia, ib = ids[sl_a][on], ids[sl_b][on]
        pick_a = (oa < ob) if sense > 0 else (oa > ob)
        lev = torch.where(pick_a, oa, ob)
        w = torch.where(pick_a, ia, ib)
        v = (lev << 32) | w
        keys.append((torch.minimum(A, B)[on] << shift) | torch.maximum(A, B)[on])
        vals.append(v if sense > 0 else -v)  # the minimum crossing as a maximum
        del A, B, on, oa, ob, ia, ib, pick_a, lev, w, v
    keys = torch.cat(keys)
    vals = torch.cat(vals)
    uk, inv = torch.unique(keys, return_inverse=True)
    best = torch.full((uk.numel(),), torch.iinfo(torch.int64).min, dtype=torch.int64, device=lab.device)
    best.scatter_reduce_(0, inv, vals, reduce="amax")
    if sense < 0:
        best = -best
    return uk, (best & 0xFFFFFFFF)


def test_graph_full_size_512(m):
    """512^3 smooth and noise fields: maxima arcs and saddles equal plain
    PyTorch group-by over every edge; minima arcs on the smooth field."""
    E = 512
    dims = (E, E, E)
    n = E ** 3
    for kind, senses in (("smooth", (1, -1)), ("noise", (1,))):
        f = (workloads.field_smooth(edge=E, seed=1, device="cuda") if kind == "smooth"
             else workloads.field_noise(edge=E, seed=1, device="cuda")).reshape(-1)
        order, asc, desc, ms, cells = m.segment(f, dims)
        del ms, f
        torch.cuda.empty_cache()
        for sense in senses:
            lab = desc if sense > 0 else asc
            shift = max(int(n - 1).bit_length(), 0)
            a, b, s = m.extremum_graph(lab, order, dims, sense)
            uk, w = torch_graph(lab, order, dims, sense, shift)
            assert a.numel() == uk.numel()
            assert torch.equal((a.long() << shift) | b.long(), uk)
            assert torch.equal(s.long(), w)
            del a, b, s, uk, w
            torch.cuda.empty_cache()
        del order, asc, desc
        torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# explicit meshes (msc_adjacency_csr, msc_extremum_graph_csr)


def random_csr(n, m, rng):
    edges = {(int(min(a, b)), int(max(a, b))) for a, b in rng.integers(0, n, (m, 2)) if a != b}
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    row = np.zeros(n + 1, np.int32)
    for v in range(n):
        row[v + 1] = row[v] + len(adj[v])
    col = np.array([u for v in range(n) for u in sorted(adj[v])], np.int32)
    return row, col


def check_csr(m, oracle_mod, lab, row, col, order=None, sense=1, bound=None):
    lab = np.ascontiguousarray(lab, np.int32)
    want = oracle_mod.adjacency_csr(lab, row, col, order, sense)
    t = lambda x: torch.as_tensor(np.ascontiguousarray(x, np.int32)).cuda()
    if order is None:
        got = m.adjacency_csr(t(lab), t(row), t(col), label_bound=bound)
    else:
        got = m.extremum_graph_csr(t(lab), t(order), t(row), t(col), sense, label_bound=bound)
    assert len(got) == len(want)
    for x, y in zip(got, want):
        np.testing.assert_array_equal(x.cpu().numpy(), y)
    return want[0].size


@pytest.mark.parametrize("seed", range(4))
def test_mesh_random_graphs(m, oracle_mod, seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(1000, 40000))
    row, col = random_csr(n, 4 * n, rng)
    lab = rng.integers(-1, 60, n).astype(np.int32)
    order = rng.permutation(n).astype(np.int32)
    assert check_csr(m, oracle_mod, lab, row, col, bound=60) > 100
    for sense in (1, -1):
        check_csr(m, oracle_mod, lab, row, col, order, sense, bound=60)


def test_mesh_segmentation_labels(m, oracle_mod):
    """A thinned, permuted Kuhn mesh segmented by the oracle: maxima and
    minima arcs with saddles, and cell adjacency."""
    row, col = workloads.tet_mesh_csr(edge=24, delete_frac=0.4, seed=5)
    row, col = row.numpy(), col.numpy()
    n = row.size - 1
    f = np.random.default_rng(6).random(n, dtype=np.float32)
    order = oracle_mod.order(f)
    asc_ptr, desc_ptr = oracle_mod.steepest_csr(order, row, col)
    asc, desc = oracle_mod.walk(asc_ptr), oracle_mod.walk(desc_ptr)
    ms, cells = oracle_mod.ms(asc, desc)
    assert check_csr(m, oracle_mod, desc, row, col, order, 1) > 10
    assert check_csr(m, oracle_mod, asc, row, col, order, -1) > 10
    assert check_csr(m, oracle_mod, ms, row, col, bound=cells) > 10


def test_mesh_edge_cases(m, oracle_mod):
    rng = np.random.default_rng(4)
    # no edges at all, a single vertex, isolated vertices among edges
    for n, mm in ((50, 0), (1, 0), (300, 40)):
        row, col = random_csr(n, mm, rng)
        lab = rng.integers(0, 5, n).astype(np.int32)
        check_csr(m, oracle_mod, lab, row, col, bound=5)
        check_csr(m, oracle_mod, lab, row, col, rng.permutation(n).astype(np.int32), 1, bound=5)
    # a column out of range is an argument error
    row = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
    col = torch.tensor([1, 7], dtype=torch.int32, device="cuda")
    with pytest.raises(m.MSCError) as e:
        m.adjacency_csr(torch.zeros(2, dtype=torch.int32, device="cuda"), row, col)
    assert e.value.code == m.ERR_ARG


def test_mesh_full_size_256(m):
    """The benchmarked mesh (256^3 Kuhn split, 40 % of tetrahedra deleted,
    ids permuted; 16.7M vertices): maxima arcs and saddles of a random field
    equal a plain PyTorch group-by over every CSR entry."""
    row, col = workloads.tet_mesh_csr(edge=256, delete_frac=0.4, seed=3, device="cuda")
    n = row.numel() - 1
    g = torch.Generator(device="cuda").manual_seed(11)
    f = torch.rand(n, device="cuda", generator=g)
    order = m.order(f)
    asc_ptr, desc_ptr = m.steepest_csr(order, row, col)
    desc = m.compress(desc_ptr)
    a, b, s = m.extremum_graph_csr(desc, order, row, col, 1)
    deg = (row[1:] - row[:-1]).long()
    src = torch.repeat_interleave(torch.arange(n, device="cuda"), deg)
    dst = col.long()
    keep = dst > src
    src, dst = src[keep], dst[keep]
    la, lb = desc.long()[src], desc.long()[dst]
    on = la != lb
    src, dst, la, lb = src[on], dst[on], la[on], lb[on]
    shift = max(int(n - 1).bit_length(), 0)
    keys = (torch.minimum(la, lb) << shift) | torch.maximum(la, lb)
    o = order.long()
    w = torch.where(o[src] < o[dst], src, dst)
    vals = (o[w] << 32) | w
    uk, inv = torch.unique(keys, return_inverse=True)
    best = torch.full((uk.numel(),), -1, dtype=torch.int64, device="cuda")
    best.scatter_reduce_(0, inv, vals, reduce="amax")
    assert a.numel() == uk.numel()
    assert torch.equal((a.long() << shift) | b.long(), uk)
    assert torch.equal(s.long(), best & 0xFFFFFFFF)
