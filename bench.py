#!/usr/bin/env python
"""Per-frame dynamic-mesh update benchmark (fixed-topology physics path).

Workload (synthetic, seeded): a 400 x 250 grid torus (R = 1.0, r = 0.35;
100k vertices / 200k faces) deformed every frame by 4-bone linear-blend
skinning (rotations <= 30 deg); 1M particles uniform in the rest-pose box
grown by 0.2 run contact queries with cutoff 0.05; 600k Gaussians (3 per face
at seeded barycentres).  One step = one frame:

  a1+a5  refit:    vertex-buffer update from frame k, BVH refit (fixed topology)
  a6     contact:  1M closest-point queries with cutoff 0.05
  a7     rebind:   600k face-bound Gaussians (centre, rotation, scale)
  a2-a5  rebuild:  full LBVH build of the same frame (the varying-topology path)
  a8     chamfer:  Chamfer distance, 10k samples on the deformed mesh vs 10k on
                   the rest pose (the paper's CD sample count)

value = point-to-mesh queries per second (1M contact + 20k Chamfer queries per
frame) over graph-replayed frames, inputs resident in HBM, L2 flushed (a 512 MB
write) between frames outside the timed events.  Stage times, the dominant
kernel's roofline and the refit-vs-rebuild comparison come from the five
stages captured as separate graphs and replayed back to back with events
between them.  `e2e` repeats the frame through the public API
from pinned host buffers (frame vertices and particles in, contact face and
distance out).  `--impl reference` times the CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads.meshes import torus, TorusSkinning  # noqa: E402
from workloads.sampling import osada_barycentrics, points_from, sample_surface, uniform_box  # noqa: E402

METRIC = "point-to-mesh queries/s; ms/frame update (refit vs LBVH rebuild); % of roofline"
WORKLOAD = "fixed-topology physics frame: torus 100k V / 200k F, 4-bone LBS, 1M particles " \
           "(cutoff 0.05), 600k Gaussians, refit vs LBVH rebuild, 10k+10k-sample Chamfer"
NU, NV_, CUTOFF, N_PART, G_PER_FACE, N_CD = 400, 250, 0.05, 1 << 20, 3, 10000
SEED = 3000
CONTACT_BYTES = 12 + 4 + 12 + 12 + 4      # query xyz in; face, bary, point, dist2 out
NODE_BYTES = 64                            # one node visit reads both 32-byte child boxes
WIDE_BYTES = 128                           # one 4-wide record (traversal variant 13): 4 boxes, links
TRI_BYTES = 48                             # one triangle test reads a packed triangle
ROOF_FRAME = 30                            # skinned pose of the roofline launch and its ncu record
REFIT_BYTES = 150                          # per face: 16 B index + ~8 B vertex share + 32 B leaf
                                           # box + internal (2 x 32 B read + 32 B write)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="meshgs", choices=["meshgs", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="physics",
                    choices=["physics", "batch", "sequence", "fit", "tracking", "contact", "render"],
                    help="physics: the default frame; batch: 64 scenes batched vs per scene; "
                         "sequence: varying-topology conversion; fit: differentiable template fit; "
                         "contact: the contact kernel and the refit alone (profiling); "
                         "render: the frame's Gaussian render alone (profiling)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="contact workload: one-thread traversal variant (-1: the autotuner's)")
    ap.add_argument("--leaf", type=int, default=1, help="contact workload: leaf size (with --variant)")
    ap.add_argument("--block", type=int, default=128, help="contact workload: threads per block (with --variant)")
    ap.add_argument("--no-extras", action="store_true",
                    help="physics workload: skip the batched, template-fit and 2.4M-face refit "
                         "measurements that follow the frame")
    return ap.parse_args()


class Workload:
    """Host-side inputs (generated once, seeded)."""

    def __init__(self, n_frames: int):
        self.V0, self.F = torus(NU, NV_)
        self.skin = TorusSkinning(self.V0, seed=SEED)
        self.frames = [self.skin.frame(t) for t in range(n_frames)]
        lo, hi = self.V0.min(0) - 0.2, self.V0.max(0) + 0.2
        self.P = uniform_box(N_PART, lo, hi, seed=SEED + 2)
        rng = np.random.default_rng(SEED + 3)
        self.gface = np.repeat(np.arange(self.F.shape[0], dtype=np.int32), G_PER_FACE)
        self.gbary = osada_barycentrics(rng, self.gface.shape[0]).astype(np.float32)
        self.cd_face, self.cd_bary = sample_surface(self.V0, self.F, N_CD, seed=SEED + 4)
        rf, rb = sample_surface(self.V0, self.F, N_CD, seed=SEED + 5)
        self.rest_samples = points_from(self.V0, self.F, rf, rb)

    @property
    def queries_per_frame(self):
        return N_PART + 2 * N_CD


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) == 6 and p[0].isdigit():
                rows.append(p)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [int(r[0]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": int(rows[0][1]),
                "samples": len(rows), "reasons": reasons}


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time per step (the replicas' aggregate rate divides the work
    of all ranks by it); identity for one process."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def render_camera():
    """The render's view of the torus (world -> camera rotation and translation)."""
    eye, tgt = np.array([0.4, -2.6, 1.5]), np.zeros(3)
    zc = (tgt - eye) / np.linalg.norm(tgt - eye)
    xc = np.cross(zc, [0, 0, 1.0])
    xc /= np.linalg.norm(xc)
    Rc = np.stack([xc, np.cross(zc, xc), zc])
    return Rc, -Rc @ eye


def render_appearance(n):
    """Seeded opacities and colours of the n rendered Gaussians."""
    rng = np.random.default_rng(SEED + 6)
    return (rng.uniform(0.4, 0.9, n).astype(np.float32), rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32))


def bench_render(args):
    """The frame's Gaussian-splatting render alone (profiling): the 600k face-bound
    Gaussians of the skinned torus (frame 1) from the frame's camera at 1280 x 720,
    rendered warmup + steps times; one JSON line with the per-render times."""
    import torch
    from paper_2606_00444_gb300 import MeshBVH, Workspace, gs_render
    dev = torch.device("cuda")
    W = Workload(2)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    fixed = MeshBVH(W.V0.shape[0], W.F.shape[0], dev).build(t(W.V0), t(W.F), method="ploc")
    fixed.refit(t(W.frames[1]))
    mu, quat, scale = fixed.bind_gaussians(t(W.gface), t(W.gbary))
    g_op, g_col = (t(a) for a in render_appearance(W.gface.shape[0]))
    Rc, tc = render_camera()
    ws, out, ms = Workspace(dev), None, []
    for k in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = gs_render(mu, quat, scale, g_op, g_col, Rc, tc, 1100.0, 1100.0, 640, 360, 1280, 720, ws=ws, out=out)
        b.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            ms.append(a.elapsed_time(b))
    print(json.dumps({"metric": "Gaussian render alone", "workload": "render", "gaussians": int(W.gface.shape[0]),
                      "steps": args.steps, "warmup": args.warmup, "render_ms": ms,
                      "median_ms": float(np.median(ms))}))


def replicas_value(queries_per_frame: int, world: int, ms: float) -> float:
    """Whole-job queries per second: every rank runs the same frame on its own GPU."""
    return world * queries_per_frame / (ms * 1e-3)


def gpu_arm(args, rank, world, local_rank):
    import torch
    from paper_2606_00444_gb300 import MeshBVH, Workspace, chamfer, chamfer_step, launch_count, morton_order

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    nfr = max(args.warmup + args.steps, 2)
    W = Workload(min(nfr, 64))
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    frames = torch.stack([t(f) for f in W.frames])           # resident in HBM
    F = t(W.F)
    # The particle set persists across frames, so it is stored once in Morton
    # order (mesh_morton_order), as a physics engine keeps its particles; the
    # same is done for the Chamfer samples.  Unsorted contact time is reported too.
    P_unsorted = t(W.P)
    P = P_unsorted[morton_order(P_unsorted).long()].contiguous()
    gface, gbary = t(W.gface), t(W.gbary)
    cd_rest_pos = t(points_from(W.V0, W.F, W.cd_face, W.cd_bary))
    o = morton_order(cd_rest_pos).long()
    cdf, cdb = t(W.cd_face)[o].contiguous(), t(W.cd_bary)[o].contiguous()
    rest_S = t(W.rest_samples)
    rest_S = rest_S[morton_order(rest_S).long()].contiguous()
    nV, nF = W.V0.shape[0], W.F.shape[0]

    # the fixed-topology trees are built once from the rest pose (mesh_build_ploc, an
    # agglomerative tree with fewer node visits per query) and refit every frame; the
    # varying-topology baseline rebuilds an LBVH every frame
    fixed = MeshBVH(nV, nF, dev)
    torch.cuda.synchronize()
    t_once = time.perf_counter()
    fixed.build(t(W.V0), F, method="ploc")
    torch.cuda.synchronize()
    ploc_build_ms = (time.perf_counter() - t_once) * 1e3
    rebuilt = MeshBVH(nV, nF, dev)
    rest = MeshBVH(nV, nF, dev).build(t(W.V0), F, method="ploc")
    # traversal variant for the contact queries, chosen by timing on this workload
    from paper_2606_00444_gb300.tune import tune_contact
    fixed.refit(t(W.frames[0]))
    # the contact step itself is tuned (warm start and work order included), stepping
    # through the first frames of the motion as the simulation does
    tuned = tune_contact(fixed, P, CUTOFF, frames=[frames[k] for k in range(min(4, frames.shape[0]))])
    rebuilt.set_query_config(tuned["lanes"], tuned["variant"], tuned["block"])   # same traversal
    rebuilt.set_leaf_size(tuned["leaf"], refit=False)               # on the LBVH, from its builds
    # lanes per sample of the Chamfer, chosen by timing the frame's form of it (the
    # ordered, warm-started step) on this frame's samples
    from paper_2606_00444_gb300.tune import tune_chamfer
    S0 = fixed.interpolate(cdf, cdb)
    tuned_cd = tune_chamfer(fixed, S0, rest, rest_S, step=True)
    Vin = torch.empty(nV, 3, device=dev)
    # the contact step's workspace carries each particle's work class to the next frame
    ct_ws = Workspace(dev)
    # contact faces persist from frame to frame: each frame's contact step (mesh_contact)
    # is warm-started with the previous frame's faces and runs the particles in the
    # order of the previous frame's work classes (the same answers up to near ties
    # whose kept face depends on the order faces are met)
    contact = dict(face=torch.full((N_PART,), -1, dtype=torch.int32, device=dev),
                   bary=torch.empty(N_PART, 3, device=dev), point=torch.empty(N_PART, 3, device=dev),
                   dist2=torch.empty(N_PART, device=dev))
    gout = (torch.empty(gface.shape[0], 3, device=dev), torch.empty(gface.shape[0], 4, device=dev),
            torch.empty(gface.shape[0], 3, device=dev))
    S_def = torch.empty(N_CD, 3, device=dev)
    cd_out = torch.empty(2, dtype=torch.float64, device=dev)
    # The frame's Chamfer runs as a step of the sequence (mesh_chamfer_step): warm-started
    # from the previous frame's per-sample faces, each side's samples run heaviest first
    # by the costs the previous frame left in its workspace (per-sample results those of
    # mesh_chamfer, bit for bit); the plain call is timed beside it
    cd_ps = dict(faceA=torch.full((N_CD,), -1, dtype=torch.int32, device=dev),
                 baryA=torch.empty(N_CD, 3, device=dev), dist2A=torch.empty(N_CD, device=dev),
                 faceB=torch.full((N_CD,), -1, dtype=torch.int32, device=dev),
                 baryB=torch.empty(N_CD, 3, device=dev), dist2B=torch.empty(N_CD, device=dev))
    cd_ws = Workspace(dev)
    cd_step_ws = Workspace(dev)
    flush = torch.empty(128 << 20, dtype=torch.float32, device=dev)   # 512 MB > L2

    # The frame as a fork-join graph, as an engine would schedule it: the full
    # rebuild of the frame (the varying-topology path) only reads the frame's
    # vertices and forks at the frame start; the refit and the rebind of the
    # Gaussians run as one pass (mesh_refit_bind, the Gaussians grouped by face,
    # G_PER_FACE each), after which the contact queries (main stream) and the
    # Chamfer branch (side stream) run concurrently.  The branches share no
    # workspace.  Per-stage device times are measured separately below, one stage
    # at a time (refit and rebind also as the two separate calls).
    gstart = torch.arange(0, G_PER_FACE * nF + 1, G_PER_FACE, dtype=torch.int32, device=dev)
    side_a = torch.cuda.Stream(device=dev)
    side_b = torch.cuda.Stream(device=dev)

    def stages():
        main = torch.cuda.current_stream()
        side_b.wait_stream(main)
        with torch.cuda.stream(side_b):
            rebuilt.build(Vin, F)                                # a1 + a2..a5
        fixed.refit_bind(Vin, gstart, gbary, out=gout)           # a1 + a5 + a7
        side_a.wait_stream(main)
        with torch.cuda.stream(side_a):
            fixed.interpolate(cdf, cdb, out=S_def)               # a8
            chamfer_step(fixed, S_def, rest, rest_S, cd_ps, cd_step_ws, out=cd_out)
        fixed.contact(P, CUTOFF, contact, ws=ct_ws)              # a6 (warm start, work order)
        main.wait_stream(side_a)
        main.wait_stream(side_b)

    def load_frame(k):
        Vin.copy_(frames[k % frames.shape[0]], non_blocking=True)

    # eager warm-up, and launches per frame
    for k in range(max(args.warmup, 3)):
        load_frame(k)
        stages()
    torch.cuda.synchronize()
    n0 = launch_count()
    stages()
    torch.cuda.synchronize()
    launches_per_frame = launch_count() - n0
    bits, _ = fixed.status()
    if bits & ~0x4:
        raise RuntimeError(f"device status bits {bits:#x} after warm-up")

    # capture one frame as a CUDA graph (static buffers)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        stages()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        stages()
    torch.cuda.synchronize()

    def timed_graph(nsteps, warm):
        for k in range(warm):
            load_frame(k)
            g.replay()
        times = []
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
        for k in range(nsteps):
            flush.fill_(float(k))
            starts[k].record()
            load_frame(warm + k)
            g.replay()
            ends[k].record()
        torch.cuda.synchronize()
        for k in range(nsteps):
            times.append(starts[k].elapsed_time(ends[k]))
        return times

    import torch.distributed as dist
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank)
    time.sleep(0.3)
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")          # lets a profiler keep to the timed frames
    step_ms = timed_graph(args.steps, args.warmup)
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = max_over_ranks(float(np.mean(step_ms)), world, dev)

    # per-stage device times: each stage captured as its own graph and the five
    # replayed back to back with events between them (no host gaps inside a
    # stage), after an L2 flush and the frame load, as in the timed frames
    stage_fns = [lambda: fixed.refit(Vin),
                 lambda: fixed.contact(P, CUTOFF, contact, ws=ct_ws),
                 lambda: fixed.bind_gaussians(gface, gbary, out=gout),
                 lambda: rebuilt.build(Vin, F),
                 lambda: (fixed.interpolate(cdf, cdb, out=S_def),
                          chamfer_step(fixed, S_def, rest, rest_S, cd_ps, cd_step_ws, out=cd_out))]
    contact_nh = {k: torch.empty_like(v) for k, v in contact.items()}
    stage_fns.append(lambda: fixed.closest_point(P, CUTOFF, out=contact_nh))   # no warm start
    contact_pt = {k: v.clone() for k, v in contact.items()}
    stage_fns.append(lambda: fixed.closest_point(P, CUTOFF, out=contact_pt,   # hinted, Morton order
                                                 hint=contact_pt["face"]))
    signed_out = {k: torch.empty_like(v) for k, v in contact.items() if k != "dist2"}
    signed_out["sdist"] = torch.empty_like(contact["dist2"])
    fixed.signed_distance(P, CUTOFF, out=signed_out)       # face adjacency, once per topology
    stage_fns.append(lambda: fixed.signed_distance(P, CUTOFF, out=signed_out))
    # the same contact step on the rebuilt LBVH (warm start from its own previous faces --
    # face ids survive a rebuild of the same topology -- and its own work classes), so the
    # refit and rebuild paths are compared with the same query
    contact_rb = {k: v.clone() for k, v in contact.items()}
    ct_ws_rb = Workspace(dev)
    stage_fns.append(lambda: rebuilt.contact(P, CUTOFF, contact_rb, ws=ct_ws_rb))
    cd_out_h = torch.empty_like(cd_out)
    stage_fns.append(lambda: chamfer(fixed, S_def, rest, rest_S, ws=cd_ws, out=cd_out_h))
    # refit and rebind in one pass, as the frame runs them (the two calls above give
    # the same boxes and Gaussians, bit for bit)
    gout_f = tuple(torch.empty_like(x) for x in gout)
    stage_fns.append(lambda: fixed.refit_bind(Vin, gstart, gbary, out=gout_f))
    stage_graphs = []
    for fn in stage_fns:
        gs = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gs):
            fn()
        stage_graphs.append(gs)
    torch.cuda.synchronize()
    nst = min(args.steps, 100)
    ns = len(stage_graphs)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(ns + 1)] for _ in range(nst)]
    torch.cuda.nvtx.range_push("stages")         # lets a profiler pick one stage's kernel
    for k in range(nst):
        flush.fill_(float(k))
        load_frame(k)
        for i, gs in enumerate(stage_graphs):
            evs[k][i].record()
            gs.replay()
        evs[k][ns].record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    names = ["refit", "contact", "rebind", "rebuild", "chamfer", "contact_without_warm_start",
             "contact_hinted_unordered", "contact_signed", "contact_on_rebuilt_lbvh", "chamfer_plain",
             "refit_and_rebind_fused"]
    st = {n: float(np.mean([e[i].elapsed_time(e[i + 1]) for e in evs])) for i, n in enumerate(names)}

    # the concurrent frame graph computes what the stages compute one at a time
    # (both from the same warm-start faces, so the inputs are identical)
    def frame_outputs():
        arr = rebuilt.arrays()                                   # the rebuilt tree, as bits
        tree = [arr[k].clone() for k in ("keys", "perm", "parent", "nodes_i")] + \
               [arr["tris"].view(torch.int32).clone()]
        return [v.clone() for v in contact.values()] + [x.clone() for x in gout] + [cd_out.clone()] + \
            [v.clone() for v in cd_ps.values()] + tree
    hint0 = contact["face"].clone()
    cd_state0 = [cd_ps["faceA"].clone(), cd_ps["faceB"].clone(), cd_step_ws.buf.clone()]
    load_frame(7)
    g.replay()
    conc = frame_outputs()
    contact["face"].copy_(hint0)
    for x, y in zip((cd_ps["faceA"], cd_ps["faceB"], cd_step_ws.buf), cd_state0):
        x.copy_(y)
    load_frame(7)
    for gs in stage_graphs[:5]:
        gs.replay()
    seq = frame_outputs()
    torch.cuda.synchronize()
    bad = [i for i, (x, y) in enumerate(zip(conc, seq)) if not torch.equal(x, y)]
    if bad:
        raise RuntimeError(f"the concurrent frame graph differs from the stages run one at a "
                           f"time in outputs {bad}")
    # the fused refit + rebind gives the boxes and Gaussians of the two calls, bit for bit
    nodes_seq = fixed.arrays()["nodes_i"].clone()
    load_frame(7)
    stage_graphs[names.index("refit_and_rebind_fused")].replay()
    torch.cuda.synchronize()
    fused_equal = all(torch.equal(x, y) for x, y in zip(gout_f, gout)) and \
        torch.equal(nodes_seq, fixed.arrays()["nodes_i"])
    un_ms = []
    contact_un = {k: torch.empty_like(v) for k, v in contact.items()}
    for k in range(min(nst, 20)):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fixed.closest_point(P_unsorted, CUTOFF, out=contact_un)
        b.record()
        torch.cuda.synchronize()
        un_ms.append(a.elapsed_time(b))
    st["contact_unsorted_particles"] = float(np.mean(un_ms))

    # Gaussian-splatting render of the frame's 600k rebound Gaussians, 1280 x 720
    # (synchronous call: it reads the tile-instance count; host time included)
    from paper_2606_00444_gb300 import gs_render
    g_op, g_col = (t(a) for a in render_appearance(gface.shape[0]))
    Rc, tc = render_camera()
    r_ws, r_out = Workspace(dev), None
    r_ms = []
    for k in range(13):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r_out = gs_render(gout[0], gout[1], gout[2], g_op, g_col, Rc, tc, 1100.0, 1100.0, 640, 360, 1280, 720,
                          ws=r_ws, out=r_out)
        b.record()
        torch.cuda.synchronize()
        if k >= 3:
            r_ms.append(a.elapsed_time(b))
    st["render_600k_gaussians_1280x720"] = float(np.mean(r_ms))
    # the same render with a fixed instance capacity (no host read), captured in a graph
    from paper_2606_00444_gb300 import gs_render_capacity
    r_cnt = torch.zeros(2, dtype=torch.int32, device=dev)
    gs_render_capacity(gout[0], gout[1], gout[2], g_op, g_col, Rc, tc, 1100.0, 1100.0, 640, 360, 1280, 720,
                       1 << 22, ws=r_ws, out=r_out, counts=r_cnt)
    torch.cuda.synchronize()
    r_cap = int(int(r_cnt[1].item()) * 1.25) + 1024
    r_graph = _capture(lambda: gs_render_capacity(gout[0], gout[1], gout[2], g_op, g_col, Rc, tc, 1100.0,
                                                  1100.0, 640, 360, 1280, 720, r_cap, ws=r_ws, out=r_out,
                                                  counts=r_cnt))
    st["render_600k_gaussians_1280x720_graph"] = _time_graph(r_graph, 10, 3, flush)
    if int(r_cnt[0].item()) != 0:
        raise RuntimeError("render capacity overflowed")

    # end to end through the public API from pinned host buffers, the frame run as
    # above in four graphs (refit + rebind; contact; Chamfer; rebuild) with the
    # copies on a further stream beside the kernels: the particle upload beside
    # the refit, the download of the contact results beside the rest of the frame
    # (events order them)
    gA, gB, gC, gD = (torch.cuda.CUDAGraph() for _ in range(4))
    with torch.cuda.graph(gA):
        fixed.refit_bind(Vin, gstart, gbary, out=gout)           # refit + rebind
    with torch.cuda.graph(gB):
        stage_fns[1]()                                            # contact
    with torch.cuda.graph(gC):
        stage_fns[4]()                                            # Chamfer
    with torch.cuda.graph(gD):
        stage_fns[3]()                                            # rebuild
    torch.cuda.synchronize()
    main, cs = torch.cuda.current_stream(), torch.cuda.Stream(device=dev)
    e2e_steps = min(args.steps, 50)
    hV = [torch.from_numpy(np.ascontiguousarray(W.frames[k % len(W.frames)])).pin_memory()
          for k in range(min(e2e_steps, len(W.frames)))]
    # the host keeps its particles in the same (Morton) order as the device copy, as a
    # physics engine that owns the particle order would
    hP = P.cpu().pin_memory()
    h_face = torch.empty(N_PART, dtype=torch.int32).pin_memory()
    h_d2 = torch.empty(N_PART).pin_memory()
    h_cd = torch.empty(2, dtype=torch.float64).pin_memory()
    e_ms = []
    for k in range(e2e_steps + 3):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev_p, ev_c, ev_d = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
        a.record(main)
        cs.wait_event(a)
        with torch.cuda.stream(cs):
            P.copy_(hP, non_blocking=True)                        # particles in
            ev_p.record(cs)
        Vin.copy_(hV[k % len(hV)], non_blocking=True)             # frame vertices in
        side_b.wait_stream(main)
        with torch.cuda.stream(side_b):
            gD.replay()
        gA.replay()
        side_a.wait_stream(main)
        with torch.cuda.stream(side_a):
            gC.replay()
            h_cd.copy_(cd_out, non_blocking=True)                 # Chamfer out
        main.wait_event(ev_p)
        gB.replay()
        ev_c.record(main)
        cs.wait_event(ev_c)
        with torch.cuda.stream(cs):
            h_face.copy_(contact["face"], non_blocking=True)      # contact results out
            h_d2.copy_(contact["dist2"], non_blocking=True)
            ev_d.record(cs)
        main.wait_event(ev_d)
        main.wait_stream(side_a)
        main.wait_stream(side_b)
        b.record(main)
        b.synchronize()
        if k >= 3:
            e_ms.append(a.elapsed_time(b))
    if not (torch.equal(h_face, contact["face"].cpu()) and torch.equal(h_cd, cd_out.cpu())):
        raise RuntimeError("end-to-end results read back differ from the device's")
    h2d = nV * 12 + N_PART * 12
    d2h = N_PART * 8 + 16

    # The roofline launch: the contact query without warm start on one fixed pose
    # (frame ROOF_FRAME of the skinning cycle), the launch the committed ncu counters
    # were captured from (bench.py --workload contact), with the counting kernel's
    # node visits and triangle tests for the same pose and the median of 20 launches.
    from paper_2606_00444_gb300 import l2_read_bandwidth
    fixed.refit(t(W.skin.frame(ROOF_FRAME)))
    stats = fixed.closest_point_stats(P, CUTOFF)
    roof_ms = []
    for k in range(23):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fixed.closest_point(P, CUTOFF, out=contact_nh)
        b.record()
        torch.cuda.synchronize()
        if k >= 3:
            roof_ms.append(a.elapsed_time(b))
    l2 = l2_read_bandwidth()
    out = dict(ms=ms, wall=wall, step_ms=step_ms, stages=st, clocks=ck, e2e_ms=float(np.mean(e_ms)),
               ploc_build_ms=ploc_build_ms,
               tuned=tuned, tuned_chamfer=tuned_cd, stats=stats, l2_read_gbs=l2,
               roof_ms=float(np.median(roof_ms)),
               h2d=h2d, d2h=d2h, launches=launches_per_frame * args.steps, fused_equal=fused_equal,
               contact_hits=int((contact["face"] >= 0).sum().item()),
               chamfer=[float(x) for x in cd_out.cpu()])
    return out, W


def node_bytes(cfg: dict) -> int:
    """Bytes one counted visit reads: a 64-byte node record, or a 128-byte 4-wide record
    with the one-thread traversal variant 13."""
    return WIDE_BYTES if (cfg.get("variant") == 13 and cfg.get("lanes", 1) == 1) else NODE_BYTES


def traversal_label(cfg: dict) -> str:
    """Key of a contact-kernel configuration: leaf size, variant, threads per block."""
    return f"L{cfg.get('leaf', 1)}/v{cfg['variant']}/b{cfg.get('block', 128)}"


def contact_traffic(cfg):
    """Counters per launch of the contact kernel in this configuration (a traversal_label
    or a tuned dict) from the committed ncu capture (dram_bytes, lts_bytes, fma pipe and
    issue figures), if the kernel source is still the one that was captured (else None)."""
    key = cfg if isinstance(cfg, str) else traversal_label(cfg)
    import hashlib
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    m = hashlib.sha256()
    for f in d.get("source_files", []):
        m.update(open(os.path.join(ROOT, f), "rb").read())
    if m.hexdigest()[:16] != d.get("source_hash"):
        return None
    return d.get("by_config", {}).get(key)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle (the reported baseline and the reference arm)
# ---------------------------------------------------------------------------
def host_cpu():
    """(model name, logical cores) of the host, from /proc/cpuinfo or lscpu."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return model or "unknown", os.cpu_count() or 1


def oracle_frame_sample(W, frame, nq, ng, ncd, rng, parallel=False):
    """Time the oracle on one frame: full serial LBVH build, nq contact queries,
    ng Gaussians, ncd Chamfer samples per side (the brute-force parts over every
    host core when parallel); returns the extrapolated time of a full frame (1M
    queries, 600k Gaussians, 10k + 10k Chamfer samples) and the time spent."""
    import oracle
    V = W.frames[frame % len(W.frames)]
    t0 = time.perf_counter()
    oracle.build_lbvh(V, W.F)
    t1 = time.perf_counter()
    qi = rng.choice(N_PART, nq, replace=False)
    oracle.closest_point(V, W.F, W.P[qi], CUTOFF, parallel=parallel)
    t2 = time.perf_counter()
    gi = rng.choice(W.gface.shape[0], ng, replace=False)
    oracle.bind_gaussians(V, W.F, W.gface[gi], W.gbary[gi], parallel=parallel)
    t3 = time.perf_counter()
    ci = rng.choice(N_CD, ncd, replace=False)
    SA = oracle.interpolate(V.astype(np.float64), W.F, W.cd_face[ci], W.cd_bary[ci])
    oracle.chamfer(V, W.F, SA, W.V0, W.F, W.rest_samples[ci], parallel=parallel)
    t4 = time.perf_counter()
    full = ((t1 - t0) + (t2 - t1) * N_PART / nq + (t3 - t2) * W.gface.shape[0] / ng
            + (t4 - t3) * N_CD / ncd)
    return full, t4 - t0


def cpu_baseline(W):
    """The oracle as it stands on this host: every core (the brute-force parts over
    OpenMP threads; the serial LBVH build on one), and one thread, each on a bounded
    sample of one frame extrapolated to the whole frame."""
    import oracle
    model, ncpu = host_cpu()
    nthr = oracle.num_threads()
    rng = np.random.default_rng(7)
    nq1 = 2048
    full1, spent1 = oracle_frame_sample(W, 1, nq1, 30000, 128, rng)
    nqa = 2048 * max(1, min(nthr, 16))
    fulla, spenta = oracle_frame_sample(W, 1, nqa, 30000 * max(1, min(nthr, 16)), 1024, rng, parallel=True)
    q = W.queries_per_frame
    return {"value": q / fulla, "unit": "queries/s", "cores": nthr, "kind": "oracle",
            "sample": f"one frame on {nthr} threads: full serial LBVH build of 200k faces, {nqa} of "
                      f"1M contact queries (brute force, OpenMP over queries), "
                      f"{30000 * max(1, min(nthr, 16))} of 600k Gaussians, 1024 of 10k Chamfer "
                      f"samples per side; extrapolated linearly to the full frame ({spenta:.1f} s "
                      f"of wall time)",
            "single_thread": {"value": q / full1, "cores": 1,
                              "sample": f"{nq1} contact queries, 30000 Gaussians, 128 Chamfer samples "
                                        f"per side, serial LBVH build; extrapolated ({spent1:.1f} s)"},
            "host": {"cpu_model": model, "nproc": ncpu}}


def reference_arm(args, rank, world):
    """The oracle, as it stands, on this host's cores (its brute-force parts over OpenMP
    threads, the LBVH build serial), each step one bounded sample of the physics frame
    extrapolated linearly to the whole frame (a full frame is ~2e11 point-triangle tests)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    W = Workload(4)
    nthr = oracle.num_threads()
    model, ncpu = host_cpu()
    total = args.steps + args.warmup
    budget = 150.0 / max(total, 1)                     # seconds per step, whole run ~ minutes
    nq = int(max(16, min(4096 * max(1, min(nthr, 16)), (budget - 0.35) * 250 * max(1, min(nthr, 16)))))
    rng = np.random.default_rng(11)
    for _ in range(args.warmup):
        oracle_frame_sample(W, 0, nq, 4096, 16, rng, parallel=True)
    fulls = []
    t0 = time.perf_counter()
    for k in range(args.steps):
        full, _ = oracle_frame_sample(W, k, nq, 4096, 16, rng, parallel=True)
        fulls.append(full)
    spent = time.perf_counter() - t0
    val = W.queries_per_frame / float(np.mean(fulls))
    line = {"metric": METRIC, "value": val, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(fulls)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "queries_per_frame": W.queries_per_frame,
                       "faces": NU * NV_ * 2, "gaussians": NU * NV_ * 2 * G_PER_FACE,
                       "parallelism": f"host, {nthr} threads", "frames": args.steps},
            "timing": "ms_per_step is the full frame extrapolated from each step's sample; "
                      f"the {args.steps} sampled steps took {spent:.1f} s of wall time",
            "cpu_baseline": {"value": val, "unit": "queries/s", "cores": nthr, "kind": "oracle",
                             "sample": f"per step: full serial LBVH build, {nq} contact queries, "
                                       f"4096 Gaussians, 16 Chamfer samples per side (brute force "
                                       f"over {nthr} threads), extrapolated to the full frame "
                                       f"({spent:.1f} s total)",
                             "host": {"cpu_model": model, "nproc": ncpu}},
            "e2e": {"value": val, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# Other workloads (measurements for the design notes; one JSON line each)
# ---------------------------------------------------------------------------
def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _time_graph(g, steps, warm, flush, pre=None):
    import torch
    for k in range(warm):
        if pre:
            pre(k)
        g.replay()
    st, en = _events(steps), _events(steps)
    for k in range(steps):
        flush.fill_(float(k))
        st[k].record()
        if pre:
            pre(warm + k)
        g.replay()
        en[k].record()
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in zip(st, en)]))


def _capture(fn):
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g


def bench_contact(args):
    """The contact kernel and the refit alone, for profiling and the roofline counters:
    the physics frame's agglomerative tree built once from the rest pose and refit to
    one skinned pose (frame 30), 1M Morton-ordered particles, cutoff 0.05.  Each step
    (L2 flushed first) is one refit and one plain contact query (no warm start, the
    launch the roofline is computed for) in the given traversal variant (--variant;
    -1 = the autotuner's choice).  The traversal counters run before the steps, so a
    profiler can take the k-th contact launch as the k-th step's."""
    import torch
    from paper_2606_00444_gb300 import MeshBVH, l2_read_bandwidth, morton_order
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    V0, F = torus(NU, NV_)
    sk = TorusSkinning(V0, seed=SEED)
    lo, hi = V0.min(0) - 0.2, V0.max(0) + 0.2
    P = t(uniform_box(N_PART, lo, hi, seed=SEED + 2))
    P = P[morton_order(P).long()].contiguous()
    fixed = MeshBVH(V0.shape[0], F.shape[0], dev).build(t(V0), t(F), method="ploc")
    V1 = t(sk.frame(ROOF_FRAME))
    fixed.refit(V1)
    if args.variant >= 0:
        fixed.set_leaf_size(args.leaf)
        fixed.set_query_config(1, args.variant, args.block)
        tuned = {"leaf": args.leaf, "lanes": 1, "variant": args.variant, "block": args.block}
    else:
        from paper_2606_00444_gb300.tune import tune_closest_point
        tuned = tune_closest_point(fixed, P, CUTOFF)
    stats = fixed.closest_point_stats(P, CUTOFF)
    out = dict(face=torch.empty(N_PART, dtype=torch.int32, device=dev),
               bary=torch.empty(N_PART, 3, device=dev), point=torch.empty(N_PART, 3, device=dev),
               dist2=torch.empty(N_PART, device=dev))
    flush = torch.empty(128 << 20, dtype=torch.float32, device=dev)
    tc, tr = [], []
    for k in range(args.warmup + args.steps):
        flush.fill_(float(k))
        e = _events(3)
        e[0].record()
        fixed.refit(V1)
        e[1].record()
        fixed.closest_point(P, CUTOFF, out=out)
        e[2].record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            tr.append(e[0].elapsed_time(e[1]))
            tc.append(e[1].elapsed_time(e[2]))
    l2 = l2_read_bandwidth()
    vis, tst = stats["visits"] / N_PART, stats["tests"] / N_PART
    bpq = CONTACT_BYTES + node_bytes(tuned) * vis + TRI_BYTES * tst
    line = {"metric": "contact kernel and refit alone", "workload": "contact", "steps": args.steps,
            "warmup": args.warmup, "tuned": tuned,
            "contact_ms": {"median": float(np.median(tc)), "mean": float(np.mean(tc)),
                           "min": float(np.min(tc)), "max": float(np.max(tc))},
            "refit_ms": {"median": float(np.median(tr)), "mean": float(np.mean(tr))},
            "per_query": {"node_visits": vis, "triangle_tests": tst, "algorithmic_bytes": bpq},
            "hits": stats["hits"], "l2_read_gbs": l2}
    print(json.dumps(line))


def batch_measure(steps, warmup):
    """64 scenes (log-uniform 1k-200k faces): per frame every scene is rebuilt, queried
    (4 x its vertex count, uniform in its box grown by 10%) and its Gaussians (one per
    face at the centroid) updated.  Batched: one launch per phase for all scenes.
    Per scene: the same calls 64 times.  Both captured as one CUDA graph; the batched
    outputs are checked equal, bit for bit, to the per-scene ones (the same accuracy).
    Also times the batched refit of all scenes' trees (2.9M faces)."""
    import torch
    from paper_2606_00444_gb300 import MeshBatch, MeshBVH, launch_count, set_query_group
    from workloads.meshes import batch_scenes
    dev = torch.device("cuda")
    S = batch_scenes(64, seed=4000)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    V, vo, F, fo = MeshBatch.concat(S, dev)
    from paper_2606_00444_gb300 import morton_order
    Qs, Qu, qn = [], [], []
    for i, (v, f) in enumerate(S):
        lo, hi = v.min(0), v.max(0)
        pad = 0.1 * (hi - lo)
        q = uniform_box(4 * len(v), lo - pad, hi + pad, seed=4100 + i)
        Qu.append(q)
        Qs.append(q[morton_order(t(q)).cpu().numpy()])     # each scene's queries in Morton order
        qn.append(4 * len(v))
    Q = t(np.concatenate(Qs))
    qoff = t(np.concatenate([[0], np.cumsum(qn)]).astype(np.int32))
    gface = torch.cat([torch.arange(len(f), dtype=torch.int32) for _, f in S]).to(dev)
    goff = fo
    gbary = torch.full((gface.shape[0], 3), 1.0 / 3.0, device=dev)
    nQ = Q.shape[0]
    batch = MeshBatch(64, V.shape[0], F.shape[0], dev)
    out = dict(face=torch.empty(nQ, dtype=torch.int32, device=dev), bary=torch.empty(nQ, 3, device=dev),
               point=torch.empty(nQ, 3, device=dev), dist2=torch.empty(nQ, device=dev))
    gout = (torch.empty(gface.shape[0], 3, device=dev), torch.empty(gface.shape[0], 4, device=dev),
            torch.empty(gface.shape[0], 3, device=dev))

    def batched():
        batch.build(V, vo, F, fo)
        batch.closest_point(Q, qoff, out=out)
        batch.bind_gaussians(gface, goff, gbary, out=gout)

    singles = [MeshBVH(len(v), len(f), dev) for v, f in S]
    Vs = [t(v) for v, _ in S]
    Fs = [t(f) for _, f in S]
    Qd = [t(q) for q in Qs]
    outs = [dict(face=torch.empty(len(q), dtype=torch.int32, device=dev),
                 bary=torch.empty(len(q), 3, device=dev), point=torch.empty(len(q), 3, device=dev),
                 dist2=torch.empty(len(q), device=dev)) for q in Qs]
    gfs = [torch.arange(len(f), dtype=torch.int32, device=dev) for _, f in S]
    gbs = [torch.full((len(f), 3), 1.0 / 3.0, device=dev) for _, f in S]
    gos = [(torch.empty(len(f), 3, device=dev), torch.empty(len(f), 4, device=dev),
            torch.empty(len(f), 3, device=dev)) for _, f in S]

    def plain():
        for i in range(64):
            singles[i].build(Vs[i], Fs[i])
            singles[i].closest_point(Qd[i], out=outs[i])
            singles[i].bind_gaussians(gfs[i], gbs[i], out=gos[i])

    # the per-scene calls also in the queries' sampling order: a per-scene launch is often
    # a single wave of blocks, which Morton order can leave waiting on the few blocks that
    # hold the deepest searches (the batched launch takes its work dynamically)
    Qdu = [t(q) for q in Qu]

    def plain_unsorted():
        for i in range(64):
            singles[i].build(Vs[i], Fs[i])
            singles[i].closest_point(Qdu[i], out=outs[i])
            singles[i].bind_gaussians(gfs[i], gbs[i], out=gos[i])

    flush = torch.empty(128 << 20, dtype=torch.float32, device=dev)
    set_query_group(1)
    try:
        n0 = launch_count(); batched(); torch.cuda.synchronize(); lb = launch_count() - n0
        n0 = launch_count(); plain(); torch.cuda.synchronize(); lp = launch_count() - n0
        gb, gp, gpu_ = _capture(batched), _capture(plain), _capture(plain_unsorted)
        ms_b = _time_graph(gb, steps, warmup, flush)
        ms_p = _time_graph(gp, steps, warmup, flush)
        ms_pu = _time_graph(gpu_, steps, warmup, flush)
        st, en = _events(5), _events(5)
        for k in range(5):
            flush.fill_(1.0); st[k].record(); plain(); en[k].record()
        torch.cuda.synchronize()
        ms_e = float(np.mean([a.elapsed_time(b) for a, b in zip(st, en)]))
        # the same accuracy: batched and per-scene outputs of the last replays, bit for bit
        gb.replay()
        gp.replay()
        torch.cuda.synchronize()
        same = all(torch.equal(out[k], torch.cat([o[k] for o in outs])) for k in out) and \
            all(torch.equal(gout[i], torch.cat([g[i] for g in gos])) for i in range(3))
        if not same:
            raise RuntimeError("batched outputs differ from the per-scene outputs")
        # batched refit of every scene's tree from the same vertices
        gr = _capture(lambda: batch.refit(V))
        ms_r = _time_graph(gr, steps, warmup, flush)
    finally:
        set_query_group(0)
    return {"faces": int(F.shape[0]), "queries": int(nQ), "scenes": 64,
            "ms_per_frame": {"batched_graph": ms_b, "per_scene_graph": ms_p,
                             "per_scene_graph_sampling_order": ms_pu, "per_scene_eager": ms_e},
            "launches_per_frame": {"batched": lb, "per_scene": lp},
            "outputs_equal_per_scene": same,
            "batched_refit_ms": ms_r,
            "batched_refit_frac_hbm": REFIT_BYTES * int(F.shape[0]) / (ms_r * 1e-3) / 1e9 / peaks()[0]}


def bench_batch(args):
    r = batch_measure(args.steps, args.warmup)
    ms_b = r["ms_per_frame"]["batched_graph"]
    line = {"metric": METRIC, "value": r["queries"] / (ms_b * 1e-3), "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 scenes, faces log-uniform 1k-200k (tori / icospheres, "
                                   "sinusoidal displacement), queries 4 x vertices per scene; per "
                                   "frame: LBVH build + closest point + one Gaussian per face",
                       "faces": r["faces"], "queries": r["queries"]}}
    line.update({k: v for k, v in r.items() if k not in ("faces", "queries")})
    print(json.dumps(line))


def bench_sequence(args):
    """Varying-topology conversion (template projection, Eq. 2): per frame the extracted
    target is rebuilt, the 10242 template vertices projected onto it, the template refit
    and its 20480 Gaussians updated, and the Chamfer distance (10k + 10k samples) taken."""
    r = sequence_measure(args.steps, args.warmup)
    line = {"metric": METRIC, "value": r["queries_per_frame"] / (r["ms_per_frame"] * 1e-3), "unit": "queries/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_frame"],
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "varying-topology sequence: marching cubes 128^3 of a 4-sphere "
                                   "smooth union, template icosphere 10242 V / 20480 F projected per "
                                   "frame", "frames": r["frames"], "target_faces": r["target_faces"]},
            "stages_ms": r["stages_ms"], "chamfer_last": r["chamfer_last"]}
    print(json.dumps(line))


def sequence_measure(steps, warmup):
    """The varying-topology frame of bench_sequence, timed over `steps` frames (events
    around each stage, L2 flushed before each frame)."""
    import torch
    from paper_2606_00444_gb300 import MeshBVH, Workspace, chamfer, morton_order
    from workloads.isosurface import BlobSequence
    from workloads.meshes import icosphere
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    mo = lambda P: P[morton_order(P).long()].contiguous()   # samples stored in Morton order
    nfr = min(120, max(steps + warmup, 8))
    seq = BlobSequence(2000)
    frames = [seq.mesh(k) for k in range(nfr)]
    tg = [(t(v), t(f), mo(t(points_from(v, f, *sample_surface(v, f, N_CD, seed=2100 + k)))))
          for k, (v, f) in enumerate(frames)]
    VT, FT = icosphere(5)
    VTd, FTd = t(VT), t(FT)
    maxF = max(len(f) for _, f in frames)
    maxV = max(len(v) for v, _ in frames)
    target = MeshBVH(maxV, maxF, dev)
    tmpl = MeshBVH.from_mesh(VTd, FTd, method="ploc")   # fixed topology: built once, refit
    gface = torch.arange(len(FT), dtype=torch.int32, device=dev)
    gbary = torch.full((len(FT), 3), 1.0 / 3.0, device=dev)
    sf, sb = sample_surface(VT, FT, N_CD, seed=2200)
    sf, sb = t(sf), t(sb)
    o = morton_order(t(points_from(VT, FT, sf.cpu().numpy(), sb.cpu().numpy()))).long()
    sf, sb = sf[o].contiguous(), sb[o].contiguous()
    ws = Workspace(dev)
    cd_out = torch.empty(2, dtype=torch.float64, device=dev)
    flush = torch.empty(128 << 20, dtype=torch.float32, device=dev)
    proj = dict(point=torch.empty(len(VT), 3, device=dev), dist2=torch.empty(len(VT), device=dev))
    ev = []

    def frame(k):
        V, F, SB = tg[k % nfr]
        e = _events(6)
        e[0].record()
        target.build(V, F)                                     # rebuild (varying topology)
        e[1].record()
        target.closest_point(VTd, want=("point", "dist2"), out=proj)   # Eq. 2 projection
        e[2].record()
        tmpl.refit(proj["point"])                              # fixed-topology vertex update
        e[3].record()
        tmpl.bind_gaussians(gface, gbary)
        e[4].record()
        SA = tmpl.interpolate(sf, sb)
        chamfer(tmpl, SA, target, SB, ws=ws, out=cd_out)
        e[5].record()
        return e

    for k in range(warmup):
        frame(k)
    torch.cuda.synchronize()
    for k in range(steps):
        flush.fill_(float(k))
        ev.append(frame(warmup + k))
    torch.cuda.synchronize()
    names = ["rebuild", "project", "refit", "rebind", "chamfer"]
    st = {n: float(np.mean([e[i].elapsed_time(e[i + 1]) for e in ev])) for i, n in enumerate(names)}
    ms = float(np.mean([e[0].elapsed_time(e[5]) for e in ev]))
    return {"ms_per_frame": ms, "stages_ms": st, "frames": nfr, "queries_per_frame": len(VT) + 2 * N_CD,
            "target_faces": [int(min(len(f) for _, f in frames)), int(maxF)],
            "chamfer_last": [float(x) for x in cd_out.cpu()]}


def bench_tracking(args):
    """Topology conversion over a 200-frame varying-topology sequence (Sec. 3.3): Strategy 1
    (temporal tracking, Eq. 1: k = 4 weighted projection of the tracked template onto each
    rebuilt frame, re-anchored 80/20 to the template projection every 50 frames) and
    Strategy 2 (template projection, Eq. 2), timed per frame; the drift of each is the
    Chamfer distance (10k + 10k samples) between the converted mesh and the frame."""
    import torch
    from paper_2606_00444_gb300 import MeshBVH, TemporalTracker, Workspace, chamfer, project_template
    from workloads.isosurface import BlobSequence
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    nfr, N = 200, 96
    seq = BlobSequence(2000)
    frames = [seq.mesh(k, N=N) for k in range(nfr + 1)]
    V0, F0 = frames[0]
    from paper_2606_00444_gb300 import morton_order
    tg = [(t(v), t(f), (lambda P: P[morton_order(P).long()].contiguous())(
               t(points_from(v, f, *sample_surface(v, f, N_CD, seed=2300 + k)))))
          for k, (v, f) in enumerate(frames)]
    maxV = max(len(v) for v, _ in frames)
    maxF = max(len(f) for _, f in frames)
    V0d, F0d = t(V0), t(F0)
    tracker = TemporalTracker(V0d, maxV, maxF, k=4, reanchor_every=50, keep=0.8)
    target2 = MeshBVH(maxV, maxF, dev)
    proj = torch.empty_like(V0d)
    conv = MeshBVH.from_mesh(V0d, F0d, method="ploc")   # the converted (fixed-topology) mesh
    sf, sb = sample_surface(V0, F0, N_CD, seed=2400)
    sf, sb = t(sf), t(sb)
    ws = Workspace(dev)
    cd = torch.empty(2, dtype=torch.float64, device=dev)
    ev1, ev2, drift1, drift2 = [], [], [], []
    for k in range(1, nfr + 1):
        V, F, SB = tg[k]
        e = _events(2)
        e[0].record()
        tracked = tracker.step(V, F)                   # rebuild + Eq. 1 (+ re-anchor)
        e[1].record()
        ev1.append(e)
        conv.refit(tracked)
        chamfer(conv, conv.interpolate(sf, sb), tracker.target, SB, ws=ws, out=cd)
        drift1.append(float(cd.sum().item()))
        e = _events(2)
        e[0].record()
        target2.build(V, F)                            # rebuild + Eq. 2
        project_template(target2, V0d, out=proj)
        e[1].record()
        ev2.append(e)
        conv.refit(proj)
        chamfer(conv, conv.interpolate(sf, sb), target2, SB, ws=ws, out=cd)
        drift2.append(float(cd.sum().item()))
    torch.cuda.synchronize()
    skip = min(5, nfr - 1)                             # first frames include one-time set-up
    ms1 = float(np.mean([e[0].elapsed_time(e[1]) for e in ev1[skip:]]))
    ms2 = float(np.mean([e[0].elapsed_time(e[1]) for e in ev2[skip:]]))
    at = [1, 25, 49, 50, 51, 100, 150, 200]
    line = {"metric": "topology conversion: ms/frame (rebuild + projection) and Chamfer drift",
            "value": ms1, "unit": "ms/frame", "n_gpus": 1, "steps": nfr, "warmup": skip,
            "ms_per_step": ms1, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"varying-topology sequence: marching cubes {N}^3 of a 4-sphere smooth "
                                   f"union, {nfr} frames; template = frame 0 ({len(V0)} V / {len(F0)} F)",
                       "k": 4, "reanchor_every": 50, "keep": 0.8,
                       "target_faces": [int(min(len(f) for _, f in frames)), int(maxF)]},
            "strategy1_tracking_ms_per_frame": ms1, "strategy2_projection_ms_per_frame": ms2,
            "chamfer_strategy1": {str(a): drift1[a - 1] for a in at},
            "chamfer_strategy2": {str(a): drift2[a - 1] for a in at},
            "chamfer_mean": {"strategy1": float(np.mean(drift1)), "strategy2": float(np.mean(drift2))}}
    print(json.dumps(line))


def fit_measure(n_steps):
    """Differentiable template fit: icosphere 40962 V / 81920 F fitted to the extracted
    target at tau = pi (frame 60) by Adam (lr 1e-3) on symmetric Chamfer over 1M samples
    per side plus the mean squared point-to-mesh distance of the template vertices;
    every forward and backward step runs in the library's kernels.  Beside it, the plain
    form: the same loss evaluated forward only (no autograd, no gradient kernels) on the
    same template, whose value must equal the differentiable forward's bit for bit."""
    import torch
    from paper_2606_00444_gb300 import MeshBVH, chamfer_step, morton_order, set_query_group
    from paper_2606_00444_gb300.autograd import Chamfer, Interpolate, PointMeshDistance, chamfer_state
    from workloads.isosurface import BlobSequence
    set_query_group(0)            # lanes per sample from the sample count (not the frame's tuning)
    from workloads.meshes import icosphere
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    VG, FG = BlobSequence(2000).mesh(60)
    VT, FT = icosphere(6, radius=0.9)
    ns = 1 << 20
    ft, bt = sample_surface(VT, FT, ns, seed=5001)
    SG = t(points_from(VG, FG, *sample_surface(VG, FG, ns, seed=5002)))
    tmpl = MeshBVH.from_mesh(t(VT), t(FT), method="ploc")   # built once, refit every step
    targ = MeshBVH.from_mesh(t(VG), t(FG), method="ploc")   # static target
    VGd = t(VG)
    ft, bt = t(ft), t(bt)
    # both sample sets persist over the fit, so they are stored once in the Morton order
    # of their starting positions (neighbouring threads then search neighbouring nodes)
    o = morton_order(t(points_from(VT, FT, ft.cpu().numpy(), bt.cpu().numpy()))).long()
    ft, bt = ft[o].contiguous(), bt[o].contiguous()
    SG = SG[morton_order(SG).long()].contiguous()
    V = t(VT).requires_grad_(True)
    opt = torch.optim.Adam([V], lr=1e-3)
    # the Chamfer of each step is a step of the sequence (mesh_chamfer_step): warm-started
    # from the previous step's faces, samples heaviest first by the previous step's costs
    state = chamfer_state(ns, ns, dev)

    def loss_of(Vx, grad):
        if grad:
            ST = Interpolate.apply(Vx, tmpl, ft, bt)
            cd = Chamfer.apply(ST, Vx, tmpl, SG, VGd, targ, state)
            d2v, _ = PointMeshDistance.apply(Vx, VGd, targ)
            return cd[0] + cd[1] + d2v.mean()
        tmpl.refit(Vx)                                   # the plain per-frame form
        ST = tmpl.interpolate(ft, bt)
        cd = chamfer_step(tmpl, ST, targ, SG, state["ps"], state["ws"])
        d2v = targ.closest_point(Vx, want=("dist2",))["dist2"]
        return cd[0] + cd[1] + d2v.mean()

    def step():
        opt.zero_grad(set_to_none=True)
        loss = loss_of(V, True)
        loss.backward()
        opt.step()
        return loss

    l0 = float(step().item())
    torch.cuda.synchronize()
    st, en = _events(n_steps), _events(n_steps)
    losses = []
    torch.cuda.nvtx.range_push("timed")          # lets a profiler keep to the timed steps
    for k in range(n_steps):
        st[k].record()
        loss = step()
        en[k].record()
        losses.append(loss)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in zip(st, en)]))
    # the plain forward on the current template, against the differentiable forward
    with torch.no_grad():
        Vc = V.detach().clone()
    fwd = []
    for k in range(max(3, min(n_steps, 20)) + 2):
        a, b = _events(2)
        a.record()
        lp = loss_of(Vc, False)
        b.record()
        torch.cuda.synchronize()
        if k >= 2:
            fwd.append(a.elapsed_time(b))
    # both forms from the same state (faces and sample order), so the sums match bit for bit
    snap = [v.clone() for v in state["ps"].values()] + [state["ws"].buf.clone()]
    lp = loss_of(Vc, False)
    for x, y in zip(list(state["ps"].values()) + [state["ws"].buf], snap):
        x.copy_(y)
    ld = loss_of(Vc.clone().requires_grad_(True), True)
    torch.cuda.synchronize()
    if not torch.equal(lp.detach(), ld.detach()):
        raise RuntimeError(f"plain forward loss {lp.item()!r} differs from the differentiable "
                           f"forward's {ld.item()!r}")
    return {"steps": n_steps, "ms_per_adam_step": ms, "ms_plain_forward": float(np.mean(fwd)),
            "loss_first": l0, "loss_last": float(losses[-1].item()),
            "forward_loss_equal_plain": True, "samples_per_side": ns,
            "template": [int(len(VT)), int(len(FT))], "target_faces": int(len(FG))}


def bench_fit(args):
    n_steps = 300 if args.steps >= 100 else args.steps
    r = fit_measure(n_steps)
    line = {"metric": METRIC, "value": (2 * r["samples_per_side"] + r["template"][0]) / (r["ms_per_adam_step"] * 1e-3),
            "unit": "queries/s", "n_gpus": 1, "steps": n_steps, "warmup": 1,
            "ms_per_step": r["ms_per_adam_step"], "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "template fit: icosphere 40962 V to the extracted target at "
                                   "tau = pi, Chamfer 1M + 1M samples + vertex point-to-mesh, Adam "
                                   "lr 1e-3", "target_faces": r["target_faces"]}}
    line.update(r)
    print(json.dumps(line))


def refit_large_measure(steps, warmup):
    """Refit of a 2.4M-face torus (1200 x 1000 grid) to a skinned pose, vertex update
    included, as the 200k-face frame's refit (graph replay, L2 flushed): where the
    refit's bytes, not its latency, set its time."""
    import torch
    from paper_2606_00444_gb300 import MeshBVH
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    V0, F = torus(1200, 1000)
    sk = TorusSkinning(V0, seed=SEED)
    b = MeshBVH(V0.shape[0], F.shape[0], dev).build(t(V0), t(F), method="ploc")
    Vs = [t(sk.frame(k)) for k in (10, 40)]
    Vin = torch.empty_like(Vs[0])
    flush = torch.empty(128 << 20, dtype=torch.float32, device=dev)
    g = _capture(lambda: b.refit(Vin))
    ms = _time_graph(g, steps, warmup, flush, pre=lambda k: Vin.copy_(Vs[k % 2]))
    copy = _time_graph(_capture(lambda: None), steps, warmup, flush, pre=lambda k: Vin.copy_(Vs[k % 2]))
    ms = max(ms - copy, 1e-6)                        # the frame load is not the refit's
    nF = int(F.shape[0])
    return {"faces": nF, "ms": ms, "algorithmic_bytes": REFIT_BYTES * nF,
            "frac_hbm": REFIT_BYTES * nF / (ms * 1e-3) / 1e9 / peaks()[0]}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload != "physics":
        return {"batch": bench_batch, "sequence": bench_sequence, "fit": bench_fit,
                "tracking": bench_tracking, "contact": bench_contact, "render": bench_render}[args.workload](args)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res, W = gpu_arm(args, rank, world, local_rank)
    if rank != 0:
        return
    q = W.queries_per_frame
    ms = res["ms"]
    hbm, src = peaks()
    l2 = res["l2_read_gbs"]
    # The roofline of the dominant kernel, the contact query.  Its tree (40 MB) and
    # particles stay in L2, so its bytes are bounded by L2, not HBM, bandwidth: the
    # headline fraction is its algorithmic bytes (44 B of query I/O, 64 B per node
    # visit = both children's 32-byte boxes, or 128 B per 4-wide record with
    # traversal variant 13, 48 B per triangle test, counted by the
    # counting form of the same traversal) over the L2 read bandwidth measured in
    # this run.  Beside it, from the committed ncu capture of the same launch: DRAM
    # bytes over the measured HBM peak, L2 bytes over the L2 peak, and the FP32 pipe.
    # Counters, time and ncu record all belong to the same launch: the search without
    # a warm start on frame ROOF_FRAME.
    t_contact = res["roof_ms"] * 1e-3
    vis = res["stats"]["visits"] / N_PART
    tst = res["stats"]["tests"] / N_PART
    # (with the 4-wide traversal the counting form counts its 128-byte records)
    nb = node_bytes(res["tuned"])
    per_query = CONTACT_BYTES + nb * vis + TRI_BYTES * tst
    achieved = per_query * N_PART / t_contact / 1e9
    rec = contact_traffic(res["tuned"]) if res["tuned"]["lanes"] == 1 else None
    rec = rec or {}
    dram, lts = rec.get("dram_bytes"), rec.get("lts_bytes")
    roof = {"kernel": f"k_closest_point {traversal_label(res['tuned'])} (contact, 1M queries, "
                      f"no warm start, frame {ROOF_FRAME})",
            "ms": res["roof_ms"],
            "bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s", "frac": achieved / l2,
            "peak_source": "measured in this run: k_l2_read (mesh_probe_l2_read) over a 48 MB "
                           "L2-resident buffer, best of 20",
            "traffic": dram,
            "bytes_per_query": per_query,
            "per_query": {"io": CONTACT_BYTES, "node_visits": vis, "triangle_tests": tst,
                          "node_bytes": nb, "triangle_bytes": TRI_BYTES},
            "algorithmic_over_hbm_peak": achieved / hbm,
            "hbm": {"bytes_per_launch": dram, "achieved": dram / t_contact / 1e9 if dram else None,
                    "peak": hbm, "peak_source": src,
                    "frac": dram / t_contact / 1e9 / hbm if dram else None},
            "l2": {"bytes_per_launch": lts, "achieved": lts / t_contact / 1e9 if lts else None,
                   "peak": l2, "frac": lts / t_contact / 1e9 / l2 if lts else None},
            "sm": {k: rec[k] for k in ("fma_pipe_pct", "alu_pipe_pct", "issue_active_pct",
                                       "lanes_per_inst", "warps_active_pct") if k in rec},
            "counters_source": "profiles/roofline_traffic.json (ncu, same launch; null when the "
                               "kernel source changed since)"}
    st = dict(res["stages"])
    un = st.pop("contact_unsorted_particles")
    refit_frac = REFIT_BYTES * NU * NV_ * 2 / (st["refit"] * 1e-3) / 1e9 / hbm
    line = {
        "metric": METRIC,
        "value": replicas_value(q, world, ms),
        "unit": "queries/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "queries_per_frame": q, "faces": NU * NV_ * 2,
                   "gaussians": NU * NV_ * 2 * G_PER_FACE, "parallelism": f"replicas{world}",
                   "l2": "flushed between frames (512 MB write, outside the timed events)",
                   "graph": "one CUDA graph per frame"},
        "step_ms_stats": {"mean": float(np.mean(res["step_ms"])), "median": float(np.median(res["step_ms"])),
                          "min": float(np.min(res["step_ms"])), "max": float(np.max(res["step_ms"]))},
        "stages_ms": st,
        "refit_and_rebind": {"two_calls_ms": st["refit"] + st["rebind"], "fused_ms": st["refit_and_rebind_fused"],
                             "outputs_equal": res["fused_equal"]},
        "ms_per_frame": {"refit_path": st["refit"] + st["contact"] + st["rebind"],
                         "rebuild_path": st["rebuild"] + st["contact_on_rebuilt_lbvh"] + st["rebind"],
                         "refit": st["refit"], "rebuild": st["rebuild"]},
        "refit_roofline": {"faces": NU * NV_ * 2, "ms": st["refit"], "bytes_per_face": REFIT_BYTES,
                           "frac_hbm": refit_frac},
        "fixed_topology_tree": {"build": "agglomerative (mesh_build_ploc), once from the rest pose",
                                "build_ms_once": res["ploc_build_ms"]},
        "roofline": roof,
        "clocks": res["clocks"],
        "e2e": {"value": world * q / (res["e2e_ms"] * 1e-3), "unit": "queries/s",
                "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"]},
        "gpu_launches": res["launches"],
        "contact_hits_per_frame": res["contact_hits"],
        "contact_ms_unsorted_particles": un,
        "tuned_contact": {k: res["tuned"][k] for k in ("leaf", "lanes", "variant", "block", "tried")},
        "tuned_chamfer": {k: res["tuned_chamfer"][k] for k in ("lanes", "tried")},
    }
    if not args.no_extras and world == 1:
        # the other configurations: batched vs per-scene launches (same outputs, 5
        # frames), the template fit's 300 Adam steps vs the plain forward (same loss),
        # the varying-topology sequence (12 frames of rebuild, projection, refit, rebind
        # and Chamfer), and the refit of a 2.4M-face mesh
        import torch
        torch.cuda.empty_cache()
        line["batched_64_scenes"] = batch_measure(5, 3)
        torch.cuda.empty_cache()
        line["template_fit"] = fit_measure(300)
        line["varying_topology_sequence"] = sequence_measure(12, 4)
        torch.cuda.empty_cache()
        line["refit_2_4M_faces"] = refit_large_measure(10, 3)
    if not args.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        line["cpu_baseline"] = cpu_baseline(W)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
