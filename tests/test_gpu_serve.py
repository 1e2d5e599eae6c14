"""Served requests (msc_server_*): every result equals the single-request
entry point on the same input, alone and in a mix that the server runs with
continuous batching; small requests also equal the CPU oracle.  Admission
respects the HBM budget and never skips ahead."""
import time

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

GiB = 1 << 30


@pytest.fixture(scope="module")
def m():
    import paper_2409_03771_gb300 as msc
    from paper_2409_03771_gb300 import _build

    _build.build()
    msc.load()
    return msc


def seg_field(dims, seed):
    rng = np.random.default_rng(seed)
    g = max(dims) / 64.0
    centres, sigmas, amps, _ = workloads.gaussian_params(dims, 8, (4.0 * g, 12.0 * g), None, rng=rng)
    return workloads.gaussian_sum(dims, centres, sigmas, amps, device="cuda").reshape(-1)


def cc_mask(dims, seed):
    return (seg_field(dims, seed) > 0.3).to(torch.uint8)


# small segmentations (grouped into batched launches), large ones, CC masks
MIX = [("seg", (20, 20, 20)), ("seg", (24, 16, 30)), ("cc", (48, 48, 48)), ("seg", (33, 33, 33)),
       ("seg", (96, 96, 96)), ("seg", (17, 5, 40)), ("cc", (100, 90, 80)), ("seg", (128, 128, 128)),
       ("seg", (31, 32, 33)), ("cc", (64, 80, 50)), ("seg", (40, 40, 40)), ("seg", (8, 8, 8)), ("cc", (33, 33, 33))]


@pytest.fixture(scope="module")
def inputs(m):
    return [(kind, dims, seg_field(dims, 10 + i) if kind == "seg" else cc_mask(dims, 10 + i))
            for i, (kind, dims) in enumerate(MIX)]


def solo(m, kind, dims, t):
    if kind == "seg":
        o, a, d, s, k = m.segment(t, dims)
        return {"order": o, "asc": a, "desc": d, "ms": s, "num_cells": k}
    return {"label": m.cc_mask(t, dims, 6)}


def same(x, y):
    assert x.keys() == y.keys()
    for k in x:
        if isinstance(x[k], int):
            assert x[k] == y[k], k
        else:
            assert torch.equal(x[k], y[k]), k


def submit(srv, kind, dims, t):
    return srv.submit_segment(t, dims) if kind == "seg" else srv.submit_cc(t, dims, 6)


def test_mix_equals_each_request_alone(m, inputs):
    want = [solo(m, *x) for x in inputs]
    srv = m.Server(8 * GiB, slots=4, group_max_vertices=1 << 16)
    tickets = [submit(srv, *x) for x in inputs]  # all at once: the server batches and overlaps them
    groups = []
    for t, w in zip(tickets, want):
        r = srv.wait(t)
        assert r.status == m.OK
        assert r.t_submit <= r.t_start <= r.t_done
        groups.append(r.group_size)
        same(srv.outputs(t), w)
        srv.release(t)
    assert max(groups) > 1, "small segmentations should have shared a launch"
    assert srv.stats()["arena_used"] == 0
    # one at a time through the same server: the same bytes again
    for x, w in zip(inputs, want):
        t = submit(srv, *x)
        same(srv.outputs(t), w)
        srv.release(t)
    srv.close()


def test_small_served_requests_match_the_oracle(m, inputs):
    import oracle

    srv = m.Server(2 * GiB, slots=2, group_max_vertices=1 << 16)
    picked = [x for x in inputs if x[1][0] * x[1][1] * x[1][2] <= 50_000]
    tickets = [submit(srv, *x) for x in picked]
    for (kind, dims, t), tk in zip(picked, tickets):
        out = srv.outputs(tk)
        if kind == "seg":
            wo, wa, wd, wm, wk = oracle.segment_grid(t.cpu().numpy(), dims)
            for key, want in zip(("order", "asc", "desc", "ms"), (wo, wa, wd, wm)):
                np.testing.assert_array_equal(out[key].cpu().numpy(), want)
            assert out["num_cells"] == wk
        else:
            np.testing.assert_array_equal(out["label"].cpu().numpy(), oracle.cc_grid(t.cpu().numpy(), dims, 6))
        srv.release(tk)
    srv.close()


def test_small_segmentations_group_past_a_large_request(m):
    """With the only slot busy, the queue holds small, large, small, small,
    CC: the small segmentations run as one launch, the large request keeps
    its place behind the head, and every output equals the request alone."""
    srv = m.Server(8 * GiB, slots=1, group_max_vertices=1 << 16)
    blocker = seg_field((160, 160, 160), 80)
    queue = [("seg", (20, 20, 20), seg_field((20, 20, 20), 81)),
             ("seg", (100, 100, 100), seg_field((100, 100, 100), 82)),
             ("seg", (24, 18, 22), seg_field((24, 18, 22), 83)),
             ("seg", (16, 16, 16), seg_field((16, 16, 16), 84)),
             ("cc", (40, 40, 40), cc_mask((40, 40, 40), 85))]
    tb = srv.submit_segment(blocker, (160, 160, 160))
    tickets = [submit(srv, *x) for x in queue]
    res = [srv.wait(t) for t in tickets]
    assert all(r.status == m.OK for r in res)
    assert [r.group_size for r in res] == [3, 1, 3, 3, 1]
    assert res[1].t_start >= res[0].t_start  # the large request was not overtaken by its own group's head
    for t, x in zip(tickets, queue):
        same(srv.outputs(t), solo(m, *x))
        srv.release(t)
    srv.release(tb)
    srv.close()


def test_budget_admission_waits_for_release(m):
    dims = (96, 96, 96)
    f1, f2 = seg_field(dims, 1), seg_field(dims, 2)
    n = 96 ** 3
    one = m.msc_workspace_bytes(m.OP_SEGMENT, n) + 16 * n + (1 << 20)
    srv = m.Server(int(one * 1.5), slots=4, group_max_vertices=0)
    t1 = srv.submit_segment(f1, dims)
    t2 = srv.submit_segment(f2, dims)
    assert srv.wait(t1).status == m.OK
    # the second request cannot fit while the first result is held
    r2 = srv.wait(t2, timeout_ms=300)
    assert r2.status == m.PENDING and srv.stats()["queued"] == 1
    srv.release(t1)
    assert srv.wait(t2, timeout_ms=30_000).status == m.OK
    o = srv.outputs(t2)
    want = m.segment(f2, dims)
    assert torch.equal(o["ms"], want[3]) and o["num_cells"] == want[4]
    srv.release(t2)
    # a request that could never fit is refused at once
    big = torch.zeros(200 ** 3, device="cuda")
    with pytest.raises(m.MSCError) as e:
        srv.submit_segment(big, (200, 200, 200))
    assert e.value.code == m.ERR_BUDGET
    srv.close()


def test_error_in_a_batched_group_stays_with_its_request(m):
    srv = m.Server(2 * GiB, slots=1, group_max_vertices=1 << 16)
    dims = (16, 16, 16)
    good = [seg_field(dims, 40 + i) for i in range(4)]
    bad = seg_field(dims, 50).clone()
    bad[123] = float("nan")
    order = good[:2] + [bad] + good[2:]
    blocker = seg_field((160, 160, 160), 51)  # holds the only slot: the next five queue up together
    tb = srv.submit_segment(blocker, (160, 160, 160))
    tickets = [srv.submit_segment(t, dims) for t in order]
    res = [srv.wait(t) for t in tickets]
    assert [r.status for r in res] == [m.OK, m.OK, m.ERR_NAN, m.OK, m.OK]
    assert srv.wait(tb).status == m.OK
    srv.release(tb)
    for t, f, r in zip(tickets, order, res):
        if r.status == m.OK:
            assert torch.equal(srv.outputs(t)["ms"], m.segment(f, dims)[3])
        srv.release(t)
    srv.close()


def test_requests_arriving_while_others_run_are_admitted(m):
    """A stream of arrivals spread over time: later requests are admitted
    while earlier ones are still on the GPU (their run intervals overlap).
    The first request is just below the size that runs without newcomers."""
    srv = m.Server(16 * GiB, slots=4, group_max_vertices=1 << 16)
    dims_big = (255, 255, 255)
    big = seg_field(dims_big, 3)
    small = [seg_field((24, 24, 24), 60 + i) for i in range(6)]
    t_big = srv.submit_segment(big, dims_big)
    time.sleep(0.001)
    ts = [srv.submit_segment(f, (24, 24, 24)) for f in small]
    rb = srv.wait(t_big)
    rs = [srv.wait(t) for t in ts]
    assert rb.status == m.OK and all(r.status == m.OK for r in rs)
    # at least one small request started before the big one finished
    assert min(r.t_start for r in rs) < rb.t_done
    for t, f in zip(ts, small):
        assert torch.equal(srv.outputs(t)["asc"], m.segment(f, (24, 24, 24))[1])
        srv.release(t)
    srv.release(t_big)
    srv.close()


def test_a_large_request_runs_without_newcomers_under_light_load(m):
    """A request of >= 2^24 vertices on the GPU and a short queue: a small
    request that arrives meanwhile starts only after the large one is done."""
    srv = m.Server(16 * GiB, slots=4, group_max_vertices=1 << 16)
    dims_big = (256, 256, 256)  # 2^24 vertices
    big = seg_field(dims_big, 4)
    small = seg_field((24, 24, 24), 90)
    t_big = srv.submit_segment(big, dims_big)
    t_small = srv.submit_segment(small, (24, 24, 24))
    rb, rs = srv.wait(t_big), srv.wait(t_small)
    assert rb.status == m.OK and rs.status == m.OK
    assert rs.t_start >= rb.t_done
    assert torch.equal(srv.outputs(t_small)["ms"], m.segment(small, (24, 24, 24))[3])
    srv.release(t_small)
    srv.release(t_big)
    srv.close()


def test_destroy_with_queued_requests(m):
    srv = m.Server(1 * GiB, slots=1, group_max_vertices=0)
    fs = [seg_field((64, 64, 64), 70 + i) for i in range(4)]
    for f in fs:
        srv.submit_segment(f, (64, 64, 64))
    srv.close()  # waits for the running request, cancels the queued ones
