"""Batched segmentation (msc_batch_*) vs the CPU oracle, instance by instance.

A batch packs many grids into one vertex space; every output is
instance-local, so each instance must equal the oracle's segmentation of
that grid alone -- bit for bit, through plain launches, through a replayed
CUDA graph, and under every tuning the autotuner may pick.
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


def field_for(dims, seed, kind):
    n = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(seed)
    if kind == "ties":  # few distinct values: the id tie-break decides
        return (rng.integers(-3, 4, n) / 2).astype(np.float32)
    if kind == "noise":
        return rng.random(n, dtype=np.float32)
    centres, sigmas, amps, _ = workloads.gaussian_params(dims, 4, (1.5, 6.0), None, rng=rng)
    return workloads.gaussian_sum(dims, centres, sigmas, amps).numpy().ravel()


# anisotropic, degenerate (1 x 1 x 1, lines, planes), ragged against every
# tile shape, several sort tiles per instance, nx % 4 == 0 and != 0
DIMS = [(1, 1, 1), (17, 3, 5), (64, 8, 8), (1, 40, 1), (33, 1, 29), (5, 6, 7), (40, 36, 12), (2, 2, 2),
        (70, 61, 9), (16, 16, 16), (1, 1, 300), (9, 50, 23)]
KINDS = ["smooth", "ties", "noise"]


@pytest.fixture(scope="module")
def mixed(m):
    fields = [field_for(d, 100 + i, KINDS[i % 3]) for i, d in enumerate(DIMS)]
    want = [workloads_oracle(f, d) for f, d in zip(fields, DIMS)]
    return fields, want


def workloads_oracle(f, dims):
    import oracle

    return oracle.segment_grid(f, dims)


def fill(b, fields):
    b.f.copy_(torch.from_numpy(np.concatenate(fields)).cuda())
    for t in (b.order, b.asc, b.desc, b.ms, b.num_cells):
        t.fill_(-7)  # stale values must not survive


def check(b, want):
    cells = b.num_cells.cpu().numpy()
    for i, (o, a, d, s) in enumerate(zip(*(b.split(t[: b.total]) for t in (b.order, b.asc, b.desc, b.ms)))):
        wo, wa, wd, ws, wk = want[i]
        np.testing.assert_array_equal(o.cpu().numpy(), wo, err_msg=f"order, instance {i} {b.dims[i]}")
        np.testing.assert_array_equal(a.cpu().numpy(), wa, err_msg=f"asc, instance {i} {b.dims[i]}")
        np.testing.assert_array_equal(d.cpu().numpy(), wd, err_msg=f"desc, instance {i} {b.dims[i]}")
        np.testing.assert_array_equal(s.cpu().numpy(), ws, err_msg=f"ms, instance {i} {b.dims[i]}")
        assert cells[i] == wk, (i, b.dims[i])


def test_batch_plain_launches_match_oracle(m, mixed):
    fields, want = mixed
    b = m.Batch(DIMS)
    fill(b, fields)
    b.run()
    check(b, want)


def test_batch_graph_replay_matches_oracle(m, mixed):
    fields, want = mixed
    b = m.Batch(DIMS)
    kernels = b.plan()
    assert kernels > 10
    for rep in range(2):  # replays reset every piece of state they use
        fill(b, fields)
        before = m.msc_launch_count()
        b.launch()
        assert m.msc_launch_count() - before == kernels
        check(b, want)
    b.close()


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("shift", [1, 3, 6])
def test_batch_every_tuning_gives_the_same_result(m, mixed, shape, shift):
    fields, want = mixed
    b = m.Batch(DIMS)
    fill(b, fields)
    b.run(tune=(shape, shift))
    check(b, want)


def test_batch_autotune_picks_a_tuning_and_keeps_results(m, mixed):
    fields, want = mixed
    b = m.Batch(DIMS)
    fill(b, fields)
    (shape, shift), ms = b.autotune(reps=1)
    assert 0 <= shape < 4 and 1 <= shift <= 30 and ms > 0
    fill(b, fields)
    b.run()  # tune=None: the remembered choice
    check(b, want)


def test_batch_single_instance_equals_segment(m):
    dims = (48, 40, 36)
    f = field_for(dims, 7, "smooth")
    b = m.Batch([dims])
    fill(b, [f])
    b.run()
    check(b, [workloads_oracle(f, dims)])


def test_batch_nan_sets_status(m):
    dims_list = [(8, 8, 8), (9, 9, 9)]
    b = m.Batch(dims_list)
    f = np.zeros(b.total, np.float32)
    f[600] = np.nan  # inside the second instance
    b.f.copy_(torch.from_numpy(f).cuda())
    with pytest.raises(m.MSCError) as e:
        b.run()
    assert e.value.code == m.ERR_NAN


def test_batch_rejects_bad_grids(m):
    assert m.msc_batch_workspace_bytes([(4, 0, 4)]) == 0
    assert m.msc_batch_workspace_bytes([(1 << 11, 1 << 11, 1 << 10)]) == 0  # 2^32 vertices
    assert m.msc_batch_workspace_bytes([]) == 0


def test_batch_many_instances_with_long_paths(m):
    """64 smooth instances of the batched workload's shape family (edges
    scaled down to 8..40): every one equals its oracle segmentation."""
    dims_list, fields, want = [], [], []
    for i in range(64):
        dims, rng = workloads.batch_dims(1000 + i)
        dims = tuple(max(1, d // 6) for d in dims)
        centres, sigmas, amps, _ = workloads.gaussian_params(dims, 8, (2.0, 6.0), None, rng=rng)
        f = workloads.gaussian_sum(dims, centres, sigmas, amps).numpy().ravel()
        dims_list.append(dims)
        fields.append(f)
        want.append(workloads_oracle(f, dims))
    b = m.Batch(dims_list)
    fill(b, fields)
    b.plan()
    b.launch()
    check(b, want)
    b.close()


def test_batch_full_size_512_instances(m):
    """The batched workload at full size: 512 anisotropic instances (seeds
    100..611, edges 16..256 per axis, ~330M vertices) in one graph launch.
    Every instance equals msc_segment on that grid alone, bit for bit; the
    oracle checks the six smallest instances and two of median size."""
    import oracle

    dims_list, fields = [], []
    for i in range(512):
        dims, f = workloads.batch_instance(100 + i, device="cuda")
        dims_list.append(dims)
        fields.append(f.reshape(-1))
    b = m.Batch(dims_list)
    torch.cat(fields, out=b.f)
    del fields
    b.plan()
    b.launch()
    ws = torch.empty(m.msc_workspace_bytes(m.OP_SEGMENT, max(b.sizes)), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    k = torch.zeros(1, dtype=torch.int32, device="cuda")
    outs = [torch.empty(max(b.sizes), dtype=torch.int32, device="cuda") for _ in range(4)]
    batch_views = [b.split(t[: b.total]) for t in (b.order, b.asc, b.desc, b.ms)]
    cells = b.num_cells.cpu().tolist()
    for i, d in enumerate(dims_list):
        n = b.sizes[i]
        a, z = b.offsets[i], b.offsets[i + 1]
        assert m.msc_segment(b.f[a:z], d, *(o[:n] for o in outs), k, ws, ws.numel(), st) == m.OK
        for j in range(4):
            assert torch.equal(outs[j][:n], batch_views[j][i]), (i, d, j)
        assert int(k.item()) == cells[i] and int(st.item()) == m.OK
    by_size = sorted(range(512), key=lambda i: b.sizes[i])
    for i in by_size[:6] + by_size[255:257]:
        f = b.f[b.offsets[i]:b.offsets[i + 1]].cpu().numpy()
        wo, wa, wd, wm, wk = oracle.segment_grid(f, dims_list[i])
        for got, want in zip((batch_views[j][i] for j in range(4)), (wo, wa, wd, wm)):
            np.testing.assert_array_equal(got.cpu().numpy(), want)
        assert cells[i] == wk
    b.close()
