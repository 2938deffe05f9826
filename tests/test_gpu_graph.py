"""A whole fixed-topology frame (vertex update, refit, contact queries, Gaussian
rebind, full rebuild, Chamfer) captured in one CUDA graph and replayed gives the
same bits as the same frame run eagerly, for several frames in a row; and the
same frame run as a fork-join over three streams (the branches that only read
the refit mesh, and the rebuild, concurrently), eagerly or captured, gives the
same bits as the calls run one after another."""
import numpy as np
import pytest
import torch

from paper_2606_00444_gb300 import MeshBVH, Workspace, chamfer
from parity import dev
from workloads.meshes import torus, TorusSkinning
from workloads.sampling import osada_barycentrics, sample_surface, uniform_box

pytestmark = pytest.mark.gpu


def _frame_setup():
    V0, F = torus(80, 50)
    sk = TorusSkinning(V0, seed=77)
    frames = [dev(sk.frame(t)) for t in range(4)]
    Fd = dev(F)
    P = dev(uniform_box(50000, V0.min(0) - 0.2, V0.max(0) + 0.2, seed=78))
    rng = np.random.default_rng(79)
    gface = dev(np.repeat(np.arange(len(F), dtype=np.int32), 2))
    gbary = dev(osada_barycentrics(rng, 2 * len(F)).astype(np.float32))
    sf, sb = (dev(a) for a in sample_surface(V0, F, 3000, seed=80))
    fixed = MeshBVH.from_mesh(dev(V0), Fd)
    rebuilt = MeshBVH(len(V0), len(F))
    rest = MeshBVH.from_mesh(dev(V0), Fd)
    Vin = torch.empty_like(frames[0])
    outs = dict(face=torch.empty(50000, dtype=torch.int32, device="cuda"),
                dist2=torch.empty(50000, device="cuda"), bary=torch.empty(50000, 3, device="cuda"),
                point=torch.empty(50000, 3, device="cuda"))
    g3 = (torch.empty(len(gface), 3, device="cuda"), torch.empty(len(gface), 4, device="cuda"),
          torch.empty(len(gface), 3, device="cuda"))
    S = torch.empty(3000, 3, device="cuda")
    cd = torch.empty(2, dtype=torch.float64, device="cuda")
    ws = Workspace(torch.device("cuda"))

    def frame():
        fixed.refit(Vin)
        fixed.closest_point(P, 0.05, out=outs)
        fixed.bind_gaussians(gface, gbary, out=g3)
        rebuilt.build(Vin, Fd)
        fixed.interpolate(sf, sb, out=S)
        chamfer(fixed, S, rest, S, ws=ws, out=cd)

    def snapshot():
        # every output and every array of both BVHs (scratch lists excluded:
        # only their first entries per block are defined)
        torch.cuda.synchronize()
        arrs = [v for b in (rebuilt, fixed) for v in b.arrays().values()]
        return [t.contiguous().clone().view(-1).view(torch.uint8) for t in (*outs.values(), *g3, S, cd, *arrs)]

    side_a, side_b = torch.cuda.Stream(), torch.cuda.Stream()

    def frame_fork_join():
        main = torch.cuda.current_stream()
        side_b.wait_stream(main)
        with torch.cuda.stream(side_b):
            rebuilt.build(Vin, Fd)
        fixed.refit(Vin)
        side_a.wait_stream(main)
        with torch.cuda.stream(side_a):
            fixed.bind_gaussians(gface, gbary, out=g3)
            fixed.interpolate(sf, sb, out=S)
            chamfer(fixed, S, rest, S, ws=ws, out=cd)
        fixed.closest_point(P, 0.05, out=outs)
        main.wait_stream(side_a)
        main.wait_stream(side_b)

    return frames, Vin, frame, frame_fork_join, snapshot


def _capture(fn):
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def test_graph_replayed_frame_equals_eager_frame():
    frames, Vin, frame, _, snapshot = _frame_setup()
    eager = []
    for f in frames:
        Vin.copy_(f)
        frame()
        eager.append(snapshot())
    Vin.copy_(frames[0])
    g = _capture(frame)
    for f, ref in zip(frames, eager):
        Vin.copy_(f)
        g.replay()
        got = snapshot()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)


def test_fork_join_frame_on_three_streams_equals_sequential():
    frames, Vin, frame, frame_fork_join, snapshot = _frame_setup()
    seq = []
    for f in frames:
        Vin.copy_(f)
        frame()
        seq.append(snapshot())
    for f, ref in zip(frames, seq):                     # eager, three streams
        Vin.copy_(f)
        frame_fork_join()
        for a, b in zip(snapshot(), ref):
            assert torch.equal(a, b)
    Vin.copy_(frames[0])
    g = _capture(frame_fork_join)                      # captured fork-join graph
    for f, ref in zip(frames, seq):
        Vin.copy_(f)
        g.replay()
        for a, b in zip(snapshot(), ref):
            assert torch.equal(a, b)
