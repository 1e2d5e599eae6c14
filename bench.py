#!/usr/bin/env python3
"""Throughput of the Morse-Smale segmentation + connected-components hot path
on one GB300 (replicas on N GPUs), in vertices per second.

One step = the whole hot path over one batch of synthetic input:
  * msc_segment on a 512^3 sum of 64 Gaussians (order, steepest pointers,
    path compression of both, Morse-Smale ids),
  * msc_segment on a 512^3 white-noise field (heavy ties, ~46M cells),
  * msc_cc_mask on a 512^3 feature mask (6-connectivity),
  * msc_cc_mesh on a thinned, permuted 256^3 Kuhn tetrahedral mesh.
value = vertices processed per second (all four calls) over all ranks.

--impl reference times the plain CPU oracle (the only other implementation
of the method: the paper's code is CPU C++ inside TTK and not available) on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vertices/s and % HBM roofline for MS segmentation + CC at 512^3; batched/served p50/p99"
EDGE = 512
MESH_EDGE = 256


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--edge", type=int, default=EDGE, help="grid edge (512 is the benchmarked size)")
    ap.add_argument("--mesh-edge", type=int, default=MESH_EDGE)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-instance batched measurement")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--no-serve", action="store_true", help="skip the served-request rate sweep")
    ap.add_argument("--serve-requests", type=int, default=1000, help="requests per arrival rate")
    ap.add_argument("--no-density", action="store_true", help="skip the 1024^3 mask-density sweep")
    ap.add_argument("--no-adjacency", action="store_true", help="skip the region-adjacency measurement")
    ap.add_argument("--copy-streams", type=int, default=1, help="copy streams per direction in the e2e leg")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# helpers


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_throughput(ms_local, units_per_rank, world, device):
    """Whole-job throughput of `world` independent replicas (one per GPU,
    no data-path collective): the step time is the maximum over the ranks
    (one all-reduce of the timing only), and every rank processes
    units_per_rank units per step.  Returns (max ms per step, units/s)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms_local)], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * units_per_rank / (ms_max / 1e3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.out = out
        return False

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "out", "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def sources_sha(names):
    """Hash of the kernel source files `names` (in the package's csrc) and of
    every device header there (a kernel's own header, the radix and TMA
    helpers; the public header only declares entry points and is left out)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2409_03771_gb300", "csrc")
    files = sorted(f for f in os.listdir(csrc) if f.endswith(".cuh")) + sorted(names)
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def committed_traffic(label):
    """DRAM bytes per vertex of a kernel from a committed ncu summary, if the
    kernel's source file has not changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        t = json.load(fh)
    e = t.get("kernels", {}).get(label)
    if e is None or e.get("sha") != sources_sha([e["source"]]):
        return None
    return float(e["dram_bytes_per_vertex"])


def jump_activity(msc, fields, dims, dev):
    """Vertices the pointer-jumping sweeps of one step process: for each
    field and each pointer array, sum over the sweeps of |A_s| (all n in the
    first sweep, then the vertices the previous sweep moved -- the others
    already point at their extremum).  Read from the per-sweep counters that
    msc_compress leaves at the start of its workspace (cnt[64], uint32),
    on pointers made by the same order and stencil calls."""
    import torch

    total = 0
    for f in fields:
        n = f.numel()
        asc, desc = msc.steepest_grid(msc.order(f), dims)
        ws = torch.zeros(msc.msc_workspace_bytes(msc.OP_COMPRESS, n), dtype=torch.uint8, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        for p in (asc, desc):
            assert msc.msc_compress(p, n, ws, ws.numel(), st) == 0
            torch.cuda.synchronize()
            cnt = ws[:256].view(torch.int32).cpu().tolist()
            total += n + sum(c for c in cnt if c > 0)
        del asc, desc, ws
    return total


def link_probe(dev, nbytes=1 << 30, reps=3):
    """Pinned host <-> device copy bandwidth (GB/s) over the host link: each
    direction alone, and both at once on two streams (the end-to-end leg
    runs both directions together)."""
    import torch

    h_a = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h_b = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d_a = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d_b = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed(jobs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            for st, fn in jobs:
                with torch.cuda.stream(st):
                    fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    up = lambda: d_a.copy_(h_a, non_blocking=True)
    down = lambda: h_b.copy_(d_b, non_blocking=True)
    timed([(s1, up), (s2, down)])  # warm-up
    t_up = timed([(s1, up)])
    t_down = timed([(s2, down)])
    t_both = timed([(s1, up), (s2, down)])
    gb = reps * nbytes / 1e9
    return {"h2d_alone": round(gb / t_up, 1), "d2h_alone": round(gb / t_down, 1),
            "both_total": round(2 * gb / t_both, 1)}


# Algorithmic bytes per launch of each traced kernel, as functions of the
# step's sizes (n = grid vertices, nm / nnz = mesh vertices / CSR entries).
def algorithmic_bytes(label, n, nm, nnz):
    table = {
        "order.up": 4 * n,               # read the pass's keys (or f)
        "order.down_first": 12 * n,      # read f, write (key, id)
        "order.down": 16 * n,            # read and write (key, id)
        "order.down_last": 16 * n,       # read (key, id), write (id, position) pairs
        "order.split": 16 * n,           # read the pairs, write them by sub-bucket of 2^15 ids
        "order.scatter": 12 * n,         # read the pairs, write order
        "steepest.grid": 12 * n,         # read order, write asc + desc
        "msid.insert": 12 * n,           # read asc + desc, write slot
        "msid.lookup": 8 * n,            # read slot, write id
        "cc.local": 5 * n,               # read mask, write label
        "cc.flatten": 8 * n,             # read label, write label
        "mesh.init": 4 * nm,             # write label = v
        "mesh.link": 24 * nm,            # read row[v], row[v+1], two columns, write two hooks
        "mesh.flatten": 8 * nm,          # read and write every label
        # order.scan, the MS-id table passes (occupancy, chunk ranks) and
        # mesh.hook move data-dependent amounts: no fixed algorithmic figure
    }
    return table.get(label)


# Stages of the step: a stage's achieved bandwidth is the sum of its
# kernels' algorithmic bytes over the sum of their device times.
STAGES = {
    "order": "order.",
    "steepest": "steepest.",
    "compress": "compress.",
    "msid": "msid.",
    "cc.mask": "cc.",
    "cc.mesh": "mesh.",
}


# ---------------------------------------------------------------------------
# our implementation


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2409_03771_gb300 as msc
    import workloads

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    msc.load()

    E, ME = args.edge, args.mesh_edge
    dims = (E, E, E)
    n = E ** 3
    t0 = time.time()
    f_smooth = workloads.field_smooth(edge=E, seed=1, device=dev).reshape(-1)
    f_noise = workloads.field_noise(edge=E, seed=1, device=dev).reshape(-1)
    mask = workloads.mask_blobs(edge=E, seed=2, device=dev).reshape(-1)
    row, col = workloads.tet_mesh_csr(edge=ME, delete_frac=0.4, seed=3, device=dev)
    nm, nnz = row.numel() - 1, col.numel()
    torch.cuda.synchronize()
    gen_s = time.time() - t0

    i32 = dict(dtype=torch.int32, device=dev)
    seg_out = [[torch.empty(n, **i32) for _ in range(4)] for _ in range(2)]
    cells = torch.zeros(2, **i32)
    lab = torch.empty(n, **i32)
    mlab = torch.empty(nm, **i32)
    ws = torch.empty(msc.msc_workspace_bytes(msc.OP_SEGMENT, n), dtype=torch.uint8, device=dev)
    small_ws = torch.empty(256, dtype=torch.uint8, device=dev)
    mesh_ws = torch.empty(msc.msc_workspace_bytes(msc.OP_CC_MESH, nm, nnz), dtype=torch.uint8, device=dev)
    status = torch.zeros(4, **i32)
    stream = torch.cuda.current_stream(dev)

    def step(fs, fn, mk, rw, cl, out=None, st=None):
        # out: (seg_out, cells, lab, mlab) to write to; st: the stream (default: the timed ones)
        so, ce, la, ml = out or (seg_out, cells, lab, mlab)
        st = st or stream
        for j, f in enumerate((fs, fn)):
            o = so[j]
            r = msc.msc_segment(f, dims, o[0], o[1], o[2], o[3], ce[j:j + 1], ws, ws.numel(),
                                status[j:j + 1], st)
            assert r == 0, msc.msc_status_string(r)
        r = msc.msc_cc_mask(mk, dims, 6, la, small_ws, small_ws.numel(), status[2:3], st)
        assert r == 0, msc.msc_status_string(r)
        r = msc.msc_cc_mesh(rw, cl, nm, ml, mesh_ws, mesh_ws.numel(), status[3:4], st)
        assert r == 0, msc.msc_status_string(r)

    def check_status(where):
        s = status.cpu().tolist()
        if any(s):
            raise RuntimeError(f"{where}: device status {s}")

    verts = 3 * n + nm
    for _ in range(args.warmup):
        step(f_smooth, f_noise, mask, row, col)
    torch.cuda.synchronize()
    check_status("warm-up")

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- timed region (device) ----
    msc.msc_trace_reset()
    msc.msc_trace_enable(True)
    launches0 = msc.msc_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.25)  # let the sampler start before the timed region
        ev0.record(stream)
        for _ in range(args.steps):
            step(f_smooth, f_noise, mask, row, col)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    launches = msc.msc_launch_count() - launches0
    msc.msc_trace_enable(False)
    trace = msc.msc_trace_collect()
    check_status("timed region")
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max, value = replica_throughput(ms, verts, world, dev)

    # ---- end to end: pinned host inputs in, every output back to host ----
    # Pipelined as a user of the streams API would run it: the inputs of a
    # step go in on copy streams, the step computes on its own stream, its
    # outputs come back on other copy streams; inputs and outputs are
    # double-buffered, so the copies of neighbouring steps overlap the
    # compute.  With one copy stream per direction each array is one copy;
    # with --copy-streams > 1 the copies are cut into pieces of at most 64 MiB
    # dealt round-robin over the streams, so that several copy engines work
    # at once.  Every step still copies all its inputs in and all its
    # outputs out.
    e2e = None
    if not args.no_e2e:
        srcs = (f_smooth, f_noise, mask, row, col)
        h_in = [x.cpu().pin_memory() for x in srcs]
        d_in = [[torch.empty_like(x) for x in srcs] for _ in range(2)]
        d_out = [(seg_out, cells, lab, mlab),
                 ([[torch.empty(n, **i32) for _ in range(4)] for _ in range(2)], torch.zeros(2, **i32),
                  torch.empty(n, **i32), torch.empty(nm, **i32))]

        def flat(o):
            return o[0][0] + o[0][1] + [o[1], o[2], o[3]]

        h_out = [[torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in flat(d_out[0])] for _ in range(2)]
        h2d = sum(x.numel() * x.element_size() for x in h_in)
        d2h = sum(x.numel() * x.element_size() for x in h_out[0])
        ncs = max(1, args.copy_streams)
        s_in = [torch.cuda.Stream(dev) for _ in range(ncs)]
        s_out = [torch.cuda.Stream(dev) for _ in range(ncs)]
        ev_in = [[torch.cuda.Event() for _ in range(ncs)] for _ in range(2)]
        # per timed step: first / last copy of each direction (timing events)
        dir_ev = []
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [[torch.cuda.Event() for _ in range(ncs)] for _ in range(2)]
        for e in ev_done + [x for xs in ev_out for x in xs]:
            e.record(stream)

        # one copy per array on a single copy stream (fewer host calls per
        # step); pieces of 64 MiB when several streams share the arrays
        piece_bytes = (64 << 20) if ncs > 1 else (1 << 40)

        def pieces(dsts, srcs_):
            """(dst, src) views of at most piece_bytes covering every pair."""
            out = []
            for d, h in zip(dsts, srcs_):
                d1, h1 = d.view(-1), h.view(-1)
                step_elems = max(1, piece_bytes // d1.element_size())
                for a in range(0, d1.numel(), step_elems):
                    out.append((d1[a:a + step_elems], h1[a:a + step_elems]))
            return out

        def e2e_step(i, timing=False):
            b = i % 2
            te = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if timing else None
            for j in range(ncs):
                s_in[j].wait_event(ev_done[b])  # step i-2 no longer reads d_in[b]
            if timing:
                te[0].record(s_in[0])
            for j, (d, h) in enumerate(pieces(d_in[b], h_in)):
                with torch.cuda.stream(s_in[j % ncs]):
                    d.copy_(h, non_blocking=True)
            if timing:
                te[1].record(s_in[0])
            for j in range(ncs):
                ev_in[b][j].record(s_in[j])
                stream.wait_event(ev_in[b][j])
                stream.wait_event(ev_out[b][j])  # step i-2's outputs in d_out[b] have left
            step(*d_in[b], out=d_out[b], st=stream)
            ev_done[b].record(stream)
            for j in range(ncs):
                s_out[j].wait_event(ev_done[b])
            if timing:
                te[2].record(s_out[0])
            for j, (h, d) in enumerate(pieces(h_out[b], flat(d_out[b]))):
                with torch.cuda.stream(s_out[j % ncs]):
                    h.copy_(d, non_blocking=True)
            if timing:
                te[3].record(s_out[0])
                dir_ev.append(te)
            for j in range(ncs):
                ev_out[b][j].record(s_out[j])

        for i in range(4):  # untimed: the copy path and both buffer sets warm up
            e2e_step(i)
        torch.cuda.synchronize()
        ee = max(2, args.steps)
        barrier()
        torch.cuda.synchronize()
        gc.disable()  # no collector pause while the host enqueues the steps
        try:
            ev0.record(stream)
            for j in range(ncs):
                s_in[j].wait_event(ev0)
            for i in range(ee):
                e2e_step(i, timing=(ncs == 1))
        finally:
            gc.enable()
        for b in range(2):
            for j in range(ncs):
                stream.wait_event(ev_out[b][j])
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        check_status("e2e")
        e_ms, e_value = replica_throughput(ev0.elapsed_time(ev1) / ee, verts, world, dev)
        # achieved rate of each direction's copies within the steps (one
        # copy stream per direction: first to last piece on that stream)
        dirs = {}
        if dir_ev:
            up = sorted(e[0].elapsed_time(e[1]) for e in dir_ev)
            down = sorted(e[2].elapsed_time(e[3]) for e in dir_ev)
            # step to step: the start of one step's input copies to the next one's
            gaps = sorted(a[0].elapsed_time(b[0]) for a, b in zip(dir_ev, dir_ev[1:]))
            dirs = {"h2d_ms_median": round(up[len(up) // 2], 2), "d2h_ms_median": round(down[len(down) // 2], 2),
                    "h2d_gbs": round(h2d / (up[len(up) // 2] / 1e3) / 1e9, 1),
                    "d2h_gbs": round(d2h / (down[len(down) // 2] / 1e3) / 1e9, 1),
                    "h2d_ms_max": round(up[-1], 2), "d2h_ms_max": round(down[-1], 2),
                    "step_ms_min": round(gaps[0], 2) if gaps else None,
                    "step_ms_median": round(gaps[len(gaps) // 2], 2) if gaps else None,
                    "step_ms_max": round(gaps[-1], 2) if gaps else None}
        e2e = {"value": e_value, "unit": "vertices/s", "ms_per_step": e_ms, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "copy_streams_per_direction": ncs, "within_steps": dirs,
               "link_probe": link_probe(dev),
               "pipelined": (("inputs and outputs one copy per array on one copy stream per direction, " if ncs == 1 else
                              f"inputs and outputs in pieces of <= 64 MiB over {ncs} copy streams per direction, ") +
                             "compute on its own stream, double-buffered; every step copies all inputs and outputs")}
        del d_in, d_out, h_out

    # ---- rooflines (live trace over the timed region) ----
    peak, peak_kind = measured_peaks()
    stages = {k: round(v[1] / args.steps, 4) for k, v in sorted(trace.items(), key=lambda kv: -kv[1][1])}
    # pointer jumping: 12 B per active vertex per sweep (read d[v], gather d[d[v]], write d[v])
    jump_bytes_per_step = 12 * jump_activity(msc, (f_smooth, f_noise), dims, dev)

    def per_launch_bytes(label, cnt):
        if label == "compress.jump":
            return jump_bytes_per_step * args.steps / cnt  # an average over the step's sweeps
        return algorithmic_bytes(label, n, nm, nnz)

    rooflines = {}
    for label, (cnt, tot) in sorted(trace.items(), key=lambda kv: -kv[1][1]):
        b = per_launch_bytes(label, cnt)
        if b is None:
            continue
        achieved = b / (tot / cnt / 1e3) / 1e9
        tb = committed_traffic(label)
        rooflines[label] = {
            "bound": "hbm", "kernel": label, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
            "traffic": None if tb is None else tb * (nm if label.startswith("mesh") else n),
            "algorithmic_bytes": round(b), "avg_launch_ms": round(tot / cnt, 4),
            "share_of_step": round(tot / args.steps / ms, 4)}
    roofline = dict(next(iter(rooflines.values()))) if rooflines else None  # the kernel with the largest share
    # every stage with its share of the step; the spec kernels
    # (stencil, pointer jumping) by name
    stage_list = []
    for name, prefix in STAGES.items():
        labels = [k for k in trace if k.startswith(prefix)]
        t = sum(trace[k][1] for k in labels) / args.steps
        known = [k for k in labels if per_launch_bytes(k, trace[k][0]) is not None]
        b = sum(per_launch_bytes(k, trace[k][0]) * trace[k][0] for k in known) / args.steps
        tk = sum(trace[k][1] for k in known) / args.steps
        e = {"stage": name, "ms_per_step": round(t, 4), "share_of_step": round(t / ms, 4),
             "kernels": sorted(labels, key=lambda k: -trace[k][1])}
        if tk > 0:
            e.update({"achieved": round(b / (tk / 1e3) / 1e9, 1), "frac": round(b / (tk / 1e3) / 1e9 / peak, 4),
                      "bytes_counted_ms": round(tk, 4)})
        stage_list.append(e)
    stage_list.sort(key=lambda e: -e["share_of_step"])
    if roofline:
        roofline["stages"] = stage_list
        roofline["stencil_and_jumping"] = {k: {kk: rooflines[k][kk] for kk in ("achieved", "frac", "avg_launch_ms")}
                                          for k in ("steepest.grid", "compress.jump") if k in rooflines}

    out = {
        "metric": METRIC, "value": value, "unit": "vertices/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i32", "data": "synthetic",
        "config": {
            "workload": (f"segment {E}^3 Gaussian sum (64, seed 1) + segment {E}^3 white noise (seed 1) + "
                         f"6-conn CC of a {E}^3 mask (256 Gaussians > 0.3, seed 2) + CC of a {ME}^3 Kuhn "
                         f"mesh (40% tets deleted, permuted, seed 3)"),
            "vertices_per_step": verts, "mesh_vertices": nm, "mesh_nnz": nnz,
            "cells": [int(c) for c in cells.cpu().tolist()],
            "mask_fraction": round(float(mask.float().mean().item()), 4),
            "l2": "inputs larger than L2 (512 MiB fields, 128 MiB mask, 0.9 GiB CSR); no flush",
            "parallelism": f"replicas x{world}", "input_gen_s": round(gen_s, 1),
        },
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": roofline,
        "kernel_rooflines": {k: {kk: v[kk] for kk in ("achieved", "frac", "avg_launch_ms", "share_of_step")}
                             for k, v in rooflines.items()},
        "stages_ms_per_step": stages,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(f_smooth, f_noise, mask, E, row, col, (seg_out, cells, lab, mlab))
    if not args.no_adjacency:
        out["adjacency"] = adjacency_bench(dev, dims, [
            ("smooth", "desc", seg_out[0][2], n, None, 0), ("smooth", "ms", seg_out[0][3], int(cells[0].item()), None, 0),
            ("noise", "desc", seg_out[1][2], n, None, 0), ("noise", "ms", seg_out[1][3], int(cells[1].item()), None, 0),
            # the extremum graph: maxima / minima arcs with their saddles
            ("smooth", "desc", seg_out[0][2], n, seg_out[0][0], 1), ("smooth", "asc", seg_out[0][1], n, seg_out[0][0], -1),
            ("noise", "desc", seg_out[1][2], n, seg_out[1][0], 1)])
        out["adjacency"]["mesh"] = mesh_graph_bench(dev, row, col)
    if not args.no_batch:
        del f_smooth, f_noise, mask, row, col, seg_out, lab, mlab, ws
        torch.cuda.empty_cache()
        out["batch"] = batch_bench(dev, count=args.batch_count)
    if not args.no_serve:
        torch.cuda.empty_cache()
        out["serve"] = serve_bench(dev, args.serve_requests)
    if not args.no_density:
        torch.cuda.empty_cache()
        out["cc_density"] = density_bench(dev)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batched segmentation: 512 anisotropic instances in one graph launch vs one
# msc_segment launch sequence per instance


BATCH_SEED0 = 100


def batch_bench(dev, count=512, reps=5):
    import torch

    import paper_2409_03771_gb300 as msc
    import workloads

    t0 = time.time()
    dims_list, fields = [], []
    for i in range(count):
        dims, f = workloads.batch_instance(BATCH_SEED0 + i, device=dev)
        dims_list.append(dims)
        fields.append(f.reshape(-1))
    b = msc.Batch(dims_list, device=dev)
    torch.cat(fields, out=b.f)
    del fields
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    stream = torch.cuda.current_stream(dev)
    (shape, shift), tuned_ms = b.autotune(reps=1)
    kernels = b.plan()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        b.launch(sync=False)
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        time.sleep(0.2)
        ev0.record(stream)
        for _ in range(reps):
            b.launch(sync=False)
        ev1.record(stream)
        torch.cuda.synchronize()
    graph_ms = ev0.elapsed_time(ev1) / reps
    batch_status = int(b.status.item())
    # the plain path: one msc_segment per instance, outputs in the same packed layout
    nmax = max(b.sizes)
    ws = torch.empty(msc.msc_workspace_bytes(msc.OP_SEGMENT, nmax), dtype=torch.uint8, device=dev)
    outs = [torch.empty_like(t) for t in (b.order, b.asc, b.desc, b.ms)]
    cells = torch.empty(count, dtype=torch.int32, device=dev)
    st = torch.zeros(count, dtype=torch.int32, device=dev)

    def plain():
        for i, d in enumerate(dims_list):
            a, z = b.offsets[i], b.offsets[i + 1]
            r = msc.msc_segment(b.f[a:z], d, outs[0][a:z], outs[1][a:z], outs[2][a:z], outs[3][a:z],
                                cells[i:i + 1], ws, ws.numel(), st[i:i + 1], stream)
            assert r == 0, msc.msc_status_string(r)

    plain()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(2):
        plain()
    ev1.record(stream)
    torch.cuda.synchronize()
    plain_ms = ev0.elapsed_time(ev1) / 2
    if batch_status != 0 or int(st.abs().sum().item()) != 0:
        raise RuntimeError("batched or plain segmentation reported a device error")
    same = all(torch.equal(x[: b.total], y[: b.total]) for x, y in zip((b.order, b.asc, b.desc, b.ms), outs))
    same = same and torch.equal(cells, b.num_cells)
    out = {
        "workload": (f"{count} instances (seeds {BATCH_SEED0}..{BATCH_SEED0 + count - 1}), edges "
                     f"log-uniform in [16, 256] per axis, 8 Gaussians each; MS segmentation per instance"),
        "vertices": b.total, "graph_ms": round(graph_ms, 3), "plain_ms": round(plain_ms, 3),
        "graph_vertices_per_s": b.total / (graph_ms / 1e3), "plain_vertices_per_s": b.total / (plain_ms / 1e3),
        "speedup_vs_plain": round(plain_ms / graph_ms, 3), "identical_to_plain": bool(same),
        "kernels_per_graph": kernels, "plain_launches": None,
        "tune": {"steepest_shape": shape, "build_shift": shift, "autotuned_ms": round(tuned_ms, 3)},
        "cells_total": int(b.num_cells.sum().item()), "input_gen_s": round(gen_s, 1), "clocks": clk.summary(),
    }
    launches0 = msc.msc_launch_count()
    plain()
    torch.cuda.synchronize()
    out["plain_launches"] = int(msc.msc_launch_count() - launches0)
    b.close()
    return out


# ---------------------------------------------------------------------------
# serving: Poisson arrivals of mixed segmentation / mask-CC requests


SERVE_RATES = (100, 300, 1000, 3000, 10000)
SERVE_SEED0 = 5000       # request i at rate index r has seed SERVE_SEED0 + 100000 * r + i
SERVE_BUDGET = 120 << 30


def serve_inputs(count, seed0, dev):
    """The requests of one rate, each with the input made from its own seed
    (about 63 MB per request on average)."""
    import torch

    import workloads

    jobs = [workloads.serve_job(seed0 + i, device=dev) for i in range(count)]
    torch.cuda.synchronize()
    return jobs


def serve_run(msc, jobs, rate, slots, group_max):
    """Poisson arrivals at `rate` of the prepared requests; a waiter thread
    takes the results in submission order and releases them at once, so
    that finished results do not fill the arena."""
    import collections
    import threading

    import numpy as np

    srv = msc.Server(SERVE_BUDGET, slots=slots, group_max_vertices=group_max)
    rng = np.random.default_rng(rate)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(jobs)))
    pending = collections.deque()
    cv = threading.Condition()
    results, state = [], {"done": False}

    def waiter():
        while True:
            with cv:
                cv.wait_for(lambda: pending or state["done"])
                if not pending:
                    return
                tk = pending[0]
            r = srv.wait(tk)
            results.append((r.status, r.t_submit, r.t_start, r.t_done, r.group_size))
            srv.release(tk)
            with cv:
                pending.popleft()

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    verts, late = 0, 0
    t0 = time.perf_counter()
    for i, (kind, dims, t) in enumerate(jobs):
        delay = t0 + arrivals[i] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        elif delay < -1e-3:
            late += 1
        tk = srv.submit_segment(t, dims) if kind == "segment" else srv.submit_cc(t, dims, 6)
        verts += dims[0] * dims[1] * dims[2]
        with cv:
            pending.append(tk)
            cv.notify_all()
    with cv:
        state["done"] = True
        cv.notify_all()
    th.join()
    srv.close()
    if any(r[0] != msc.OK for r in results):
        raise RuntimeError(f"served request failed: {[r[0] for r in results if r[0]]}")
    lat = np.array([(r[3] - r[1]) * 1e3 for r in results])
    span = max(r[3] for r in results) - min(r[1] for r in results)
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "vertices_per_s": verts / span, "requests_per_s": len(jobs) / span,
            "mean_group": round(float(np.mean([r[4] for r in results])), 2),
            "submitted_late": late}


def serve_bench(dev, count):
    import torch

    import paper_2409_03771_gb300 as msc

    warm = serve_inputs(16, SERVE_SEED0 + 900000, dev)
    serve_run(msc, warm, 1000, 4, 1 << 21)  # warm-up: library state, allocator
    del warm
    rates, gen_s = [], 0.0
    with ClockSampler(dev.index) as clk:
        for ri, rate in enumerate(SERVE_RATES):
            t0 = time.time()
            jobs = serve_inputs(count, SERVE_SEED0 + 100000 * ri, dev)
            gen_s += time.time() - t0
            row = {"rate": rate, "input_gb": round(sum(t.numel() * t.element_size() for _, _, t in jobs) / 2**30, 1)}
            row.update(serve_run(msc, jobs, rate, 4, 1 << 21))
            row["plain"] = serve_run(msc, jobs, rate, 1, 0)
            rates.append(row)
            del jobs
            torch.cuda.empty_cache()
    return {
        "workload": (f"Poisson arrivals, {count} requests per rate, each with its own seeded input (made before "
                     "the rate's run): 70% MS segmentation of a cube with edge log-uniform in [32, 512], 30% "
                     "6-conn mask CC with edge log-uniform in [64, 768]; the same requests for the server and for "
                     "the plain path"),
        "budget_gb": SERVE_BUDGET >> 30,
        "server": ("4 slots, each a high-priority stream (requests >= 2^24 vertices) and a low-priority one; "
                   "segmentations <= 2^21 vertices batched, drawn from the next 64 waiting requests"),
        "plain": "1 slot, one request per launch sequence, no batching",
        "latency": "host submit to completion seen by the server (completion callback)",
        "rates": rates, "input_gen_s": round(gen_s, 1), "clocks": clk.summary(),
    }


# ---------------------------------------------------------------------------
# region adjacency (the Morse-Smale connectivity preview) of the step's own
# segmentation outputs: pairs of maxima whose manifolds touch and pairs of
# cells that share a boundary, 14-neighbour triangulation


def adjacency_bench(dev, dims, cases, reps=3):
    import torch

    import paper_2409_03771_gb300 as msc

    n = dims[0] * dims[1] * dims[2]
    ws = torch.empty(msc.msc_workspace_bytes(msc.OP_EXTREMUM_GRAPH, n), dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    k = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    peak, peak_kind = measured_peaks()
    rows = []
    for field, labels, lab, bound, order, sense in cases:
        cap = 7 * n  # room for every pair: nothing is cut
        a = torch.empty(cap, dtype=torch.int32, device=dev)
        b = torch.empty(cap, dtype=torch.int32, device=dev)
        sad = torch.empty(cap if order is not None else 1, dtype=torch.int32, device=dev)

        def run():
            if order is None:
                r = msc.msc_adjacency_grid(lab, dims, 14, bound, a, b, cap, k, ws, ws.numel(), st, stream)
            else:
                r = msc.msc_extremum_graph(lab, order, dims, 14, bound, sense, a, b, sad, cap, k, ws, ws.numel(), st,
                                           stream)
            assert r == 0, msc.msc_status_string(r)

        run()
        torch.cuda.synchronize()
        msc.msc_trace_reset()
        msc.msc_trace_enable(True)
        ev0.record(stream)
        for _ in range(reps):
            run()
        ev1.record(stream)
        torch.cuda.synchronize()
        msc.msc_trace_enable(False)
        trace = msc.msc_trace_collect()
        if int(st.item()) != 0:
            raise RuntimeError(f"adjacency of {field} {labels}: device status {int(st.item())}")
        ms = ev0.elapsed_time(ev1) / reps
        cnt, tot = trace.get("adjacency.emit", (1, 0.0))
        emit_ms = tot / max(cnt, 1)
        # the emit kernel's algorithmic traffic: every label read once (the
        # tile de-duplicated keys it writes are data-dependent and excluded)
        emit_gbs = 4 * n / (emit_ms / 1e3) / 1e9 if emit_ms > 0 else None
        rows.append({
            "field": field, "labels": labels, "op": "adjacency" if order is None else f"extremum graph ({'+' if sense > 0 else '-'})",
            "label_bound": bound, "pairs": int(k.item()), "ms": round(ms, 3),
            "vertices_per_s": n / (ms / 1e3),
            "kernels_ms": {lbl: round(t / c, 4) for lbl, (c, t) in sorted(trace.items(), key=lambda kv: -kv[1][1])},
            "emit_roofline": {"bound": "hbm", "achieved": None if emit_gbs is None else round(emit_gbs, 1),
                              "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
                              "frac": None if emit_gbs is None else round(emit_gbs / peak, 4)}})
        del a, b, sad
    return {"workload": (f"adjacency of the step's {dims[0]}^3 maximum labels and cell ids, and the extremum graph "
                         f"(arcs + saddles) of its maximum and minimum labels; 14-neighbour link"),
            "rows": rows}


def mesh_graph_bench(dev, row, col, reps=3):
    """Extremum graph over the step's explicit mesh: maxima of a seeded
    uniform field on its vertices (order, steepest pointers over the CSR and
    pointer jumping by the library), arcs and saddles over its edges."""
    import torch

    import paper_2409_03771_gb300 as msc

    n, nnz = row.numel() - 1, col.numel()
    g = torch.Generator(device=dev).manual_seed(11)
    f = torch.rand(n, device=dev, generator=g)
    order = msc.order(f)
    _, desc_ptr = msc.steepest_csr(order, row, col)
    desc = msc.compress(desc_ptr)
    del f, desc_ptr
    ws = torch.empty(msc.msc_workspace_bytes(msc.OP_EXTREMUM_GRAPH_CSR, n, nnz), dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    k = torch.zeros(1, dtype=torch.int64, device=dev)
    cap = max(nnz, 1)
    a, b, sad = (torch.empty(cap, dtype=torch.int32, device=dev) for _ in range(3))
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run():
        r = msc.msc_extremum_graph_csr(desc, order, row, col, n, nnz, n, 1, a, b, sad, cap, k, ws, ws.numel(), st,
                                       stream)
        assert r == 0, msc.msc_status_string(r)

    run()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        run()
    ev1.record(stream)
    torch.cuda.synchronize()
    if int(st.item()) != 0:
        raise RuntimeError(f"mesh extremum graph: device status {int(st.item())}")
    ms = ev0.elapsed_time(ev1) / reps
    return {"workload": f"extremum graph (maxima, saddles) of a uniform field on the step's mesh ({n} vertices, "
                        f"{nnz} CSR entries)", "arcs": int(k.item()), "ms": round(ms, 3),
            "vertices_per_s": n / (ms / 1e3)}


# ---------------------------------------------------------------------------
# connected components across mask densities (the paper's top 10 / 50 / 90 %
# sweep at 1024^3), with 6 and with the triangulation's 14 neighbours


def density_bench(dev, edge=1024, reps=3):
    import torch

    import paper_2409_03771_gb300 as msc
    import workloads

    n = edge ** 3
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.empty(256, dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for top in (0.1, 0.5, 0.9):
        mask = workloads.mask_top(edge=edge, seed=2, top=top, device=dev).reshape(-1)
        frac = float(mask.float().mean().item())
        for conn in (6, 14):
            for _ in range(2):
                assert msc.msc_cc_mask(mask, (edge,) * 3, conn, lab, ws, 256, st, stream) == 0
            ev0.record(stream)
            for _ in range(reps):
                assert msc.msc_cc_mask(mask, (edge,) * 3, conn, lab, ws, 256, st, stream) == 0
            ev1.record(stream)
            torch.cuda.synchronize()
            if int(st.item()) != 0:
                raise RuntimeError(f"cc_mask at top {top}, conn {conn}: device status {int(st.item())}")
            ms = ev0.elapsed_time(ev1) / reps
            rows.append({"top": top, "mask_fraction": round(frac, 4), "conn": conn, "ms": round(ms, 3),
                         "vertices_per_s": n / (ms / 1e3)})
        del mask
    return {"workload": f"CC of the top 10/50/90 % of a {edge}^3 field of 256 Gaussians (seed 2)",
            "rows": rows}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)


# (field z-planes, mask z-planes, mesh edge) of the oracle samples: the CPU
# baseline takes ~10 s of single-core work, a reference-arm step ~1 s
BASELINE_SAMPLE = (96, 192, 128)
STEP_SAMPLE = (8, 16, 96)


def oracle_sample(f_smooth, f_noise, mask, E, size=STEP_SAMPLE):
    """Host copies of a bounded sample of the step's workload: the first zs
    z-planes of each field, zm z-planes of the mask, and a mesh of the same
    recipe with the given edge."""
    import workloads

    zs, zm, me = size
    zs, zm = min(zs, E), min(zm, E)
    fs = f_smooth.reshape(E, E, E)[:zs].contiguous().cpu().numpy().ravel()
    fn = f_noise.reshape(E, E, E)[:zs].contiguous().cpu().numpy().ravel()
    mk = mask.reshape(E, E, E)[:zm].contiguous().cpu().numpy().ravel()
    row, col = workloads.tet_mesh_csr(edge=me, delete_frac=0.4, seed=3, device=f_smooth.device)
    return {"fs": (fs, (E, E, zs)), "fn": (fn, (E, E, zs)), "mk": (mk, (E, E, zm)),
            "mesh": (row.cpu().numpy(), col.cpu().numpy()),
            "desc": f"segment of {E}x{E}x{zs} slabs of both fields, 6-conn CC of a {E}x{E}x{zm} mask slab, "
                    f"CC of a {me}^3 mesh of the same recipe ({row.numel() - 1} vertices)"}


def oracle_step(sample):
    import oracle

    verts = 0
    for key in ("fs", "fn"):
        f, d = sample[key]
        oracle.segment_grid(f, d)
        verts += f.size
    m, d = sample["mk"]
    oracle.cc_grid(m, d, 6)
    verts += m.size
    row, col = sample["mesh"]
    oracle.cc_csr(row, col)
    verts += row.size - 1
    return verts


def paper_omp_step(f_smooth, f_noise, mask, E, row, col, gpu_out=None):
    """The paper's shared-memory method (Alg. 1 / Alg. 3, OpenMP, all host
    cores) on the full step: both fields, the mask, the mesh.  With the GPU's
    outputs of the same step, also whether every output is identical."""
    import numpy as np

    from oracle import paper_omp

    paper_omp.build()
    dims = (E, E, E)
    host = [f_smooth.cpu().numpy(), f_noise.cpu().numpy(), mask.cpu().numpy(), row.cpu().numpy(),
            col.cpu().numpy()]
    stage = [0.0] * 4
    t0 = time.perf_counter()
    segs = []
    for f in host[:2]:
        r = paper_omp.segment_grid(f, dims)
        stage = [a + b for a, b in zip(stage, r[5])]
        segs.append(r)
    t1 = time.perf_counter()
    lab = paper_omp.cc_grid(host[2], dims, 6)
    t2 = time.perf_counter()
    mlab = paper_omp.cc_csr(host[3], host[4])
    t3 = time.perf_counter()
    out = {"value": (3 * E ** 3 + host[3].size - 1) / (t3 - t0), "unit": "vertices/s",
           "cores": paper_omp.threads(), "kind": "paper method: Alg. 1 and Alg. 3, OpenMP",
           "sample": "the full step: both 512^3 segmentations (with the order and cell ids), the 512^3 mask CC, "
                     "the 256^3 mesh CC",
           "seconds": round(t3 - t0, 2),
           "stage_seconds": {"order": round(stage[0], 3), "steepest": round(stage[1], 3),
                             "path_compression": round(stage[2], 3), "cell_ids": round(stage[3], 3),
                             "cc_mask": round(t2 - t1, 3), "cc_mesh": round(t3 - t2, 3)}}
    if gpu_out is not None:
        so, cells, glab, gmlab = gpu_out
        same = all(np.array_equal(segs[j][i], so[j][i].cpu().numpy()) for j in range(2) for i in range(4))
        same &= [s_[4] for s_ in segs] == [int(c) for c in cells.cpu().tolist()]
        same &= np.array_equal(lab, glab.cpu().numpy()) and np.array_equal(mlab, gmlab.cpu().numpy())
        out["identical_to_gpu"] = bool(same)
    return out


def cpu_baseline(f_smooth, f_noise, mask, E, row=None, col=None, gpu_out=None):
    import oracle

    oracle.build()
    sample = oracle_sample(f_smooth, f_noise, mask, E, BASELINE_SAMPLE)
    t0 = time.perf_counter()
    verts = oracle_step(sample)
    dt = time.perf_counter() - t0
    out = {"value": verts / dt, "unit": "vertices/s", "cores": 1, "kind": "oracle",
           "sample": sample["desc"], "seconds": round(dt, 2)}
    if row is not None:
        out["paper_omp"] = paper_omp_step(f_smooth, f_noise, mask, E, row, col, gpu_out)
    return out


def run_reference(args):
    import torch

    import oracle
    import workloads

    rank, world, local = dist_info()
    if rank != 0:  # the oracle runs once, on rank 0
        return
    oracle.build()
    E, ME = args.edge, args.mesh_edge
    dev = torch.device("cuda", local) if torch.cuda.is_available() else torch.device("cpu")
    f_smooth = workloads.field_smooth(edge=E, seed=1, device=dev).reshape(-1)
    f_noise = workloads.field_noise(edge=E, seed=1, device=dev).reshape(-1)
    mask = workloads.mask_blobs(edge=E, seed=2, device=dev).reshape(-1)
    sample = oracle_sample(f_smooth, f_noise, mask, E)
    del f_smooth, f_noise, mask
    for _ in range(args.warmup):
        oracle_step(sample)
    t0 = time.perf_counter()
    verts = 0
    for _ in range(args.steps):
        verts += oracle_step(sample)
    dt = time.perf_counter() - t0
    value = verts / dt
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "vertices/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
        "config": {"workload": "CPU oracle on a bounded sample of the same workload", "sample": sample["desc"],
                   "vertices_per_step": verts // max(1, args.steps)},
        "cpu_baseline": {"value": value, "unit": "vertices/s", "cores": 1, "kind": "oracle",
                         "sample": sample["desc"]},
        "e2e": {"value": value, "unit": "vertices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
