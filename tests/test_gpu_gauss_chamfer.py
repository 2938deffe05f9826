"""GPU face-bound Gaussian update, Chamfer distance and gradients against the
oracle (Gaussian parameters 1e-5 absolute; Chamfer 1e-5 relative; gradients
1e-4 relative, component by component, to the oracle's analytic gradient,
itself pinned by float64 central differences)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_00444_gb300 import MeshBVH, chamfer
from paper_2606_00444_gb300.autograd import BindGaussians, Chamfer, Interpolate, PointMeshDistance
from parity import (assert_grad_close, assert_identical, check_gaussians, dev, host, point_grad_atol,
                    vertex_weight_sums)
from workloads.meshes import displaced_icosphere, icosphere, torus, TorusSkinning
from workloads.sampling import osada_barycentrics, points_from, sample_surface, uniform_box

pytestmark = pytest.mark.gpu


def test_rebind_centroid_single_frame():
    VT, FT = icosphere(3)
    G = FT.shape[0]
    gface = np.arange(G, dtype=np.int32)
    gbary = np.full((G, 3), 1 / 3, np.float32)
    bvh = MeshBVH.from_mesh(dev(VT), dev(FT))
    got = bvh.bind_gaussians(dev(gface), dev(gbary))
    check_gaussians(got, oracle.bind_gaussians(VT, FT, gface, gbary))


def test_rebind_random_anchors_offsets_and_degenerate_faces():
    V, F = displaced_icosphere(3, 0.1, 2.0)
    F = F.copy()
    F[::11, 1] = F[::11, 0]
    rng = np.random.default_rng(5)
    G = 5000
    gface = rng.integers(0, F.shape[0], G).astype(np.int32)
    gbary = osada_barycentrics(rng, G).astype(np.float32)
    goff = rng.normal(scale=0.02, size=G).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    got = bvh.bind_gaussians(dev(gface), dev(gbary), dev(goff))
    ref = oracle.bind_gaussians(V, F, gface, gbary, goff)
    check_gaussians(got, ref)
    bits, ndeg = bvh.status()
    assert ndeg == ref["n_degenerate"] > 0 and bits == 0x4


def test_rebind_full_size_600k_after_refit():
    V0, F = torus(400, 250)
    V1 = TorusSkinning(V0, seed=3000).frame(88)
    rng = np.random.default_rng(3003)
    gface = np.repeat(np.arange(F.shape[0], dtype=np.int32), 3)
    gbary = osada_barycentrics(rng, gface.shape[0]).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V0), dev(F))
    bvh.refit(dev(V1))
    mu, quat, scale = bvh.bind_gaussians(dev(gface), dev(gbary))
    pick = rng.choice(gface.shape[0], 20000, replace=False)
    ref = oracle.bind_gaussians(V1, F, gface[pick], gbary[pick])
    idx = dev(pick.astype(np.int64))
    check_gaussians((mu[idx], quat[idx], scale[idx]), ref)


def test_rebind_bad_index_sets_status():
    V, F = icosphere(1)
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    gface = np.array([0, 5, 999], np.int32)
    gbary = np.full((3, 3), 1 / 3, np.float32)
    mu, quat, scale = bvh.bind_gaussians(dev(gface), dev(gbary))
    bits, _ = bvh.status()
    assert bits & 0x1
    assert np.array_equal(host(quat)[2], [1, 0, 0, 0])


@pytest.fixture(scope="module")
def pair():
    VA, FA = icosphere(3)
    VB, FB = displaced_icosphere(4, 0.1, 0.4)
    fa, ba = sample_surface(VA, FA, 3000, seed=6)
    fb, bb = sample_surface(VB, FB, 2500, seed=7)
    SA, SB = points_from(VA, FA, fa, ba), points_from(VB, FB, fb, bb)
    return VA, FA, SA, VB, FB, SB


def test_chamfer_matches_oracle_and_is_reproducible(pair):
    VA, FA, SA, VB, FB, SB = pair
    A = MeshBVH.from_mesh(dev(VA), dev(FA))
    B = MeshBVH.from_mesh(dev(VB), dev(FB))
    out, ps = chamfer(A, dev(SA), B, dev(SB), per_sample=True)
    ref, dA, dB = oracle.chamfer(VA, FA, SA, VB, FB, SB)
    np.testing.assert_allclose(host(out), ref, rtol=1e-5)
    np.testing.assert_allclose(np.sqrt(host(ps["dist2A"])), np.sqrt(dA), rtol=1e-5, atol=1e-8)
    again = chamfer(A, dev(SA), B, dev(SB))
    assert torch.equal(out, again)
    same = chamfer(A, dev(SA), A, dev(SA))
    assert host(same).max() < 1e-12
    empty = chamfer(A, dev(SA[:0]), B, dev(SB[:5]))
    assert host(empty)[0] == 0


def test_closest_point_backward_matches_oracle():
    V, F = displaced_icosphere(3, 0.1, 0.9)
    Q = uniform_box(3000, [-1.4] * 3, [1.4] * 3, seed=8)
    g = np.random.default_rng(9).normal(size=3000).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    out = bvh.closest_point(dev(Q))
    gQ = torch.empty(3000, 3, device="cuda")
    gV = torch.zeros(V.shape[0], 3, device="cuda")
    bvh.closest_point_backward(dev(Q), out["face"], out["bary"], dev(g), gQ, gV)
    rgQ, rgV = oracle.closest_point_backward(V, F, Q, host(out["face"]),
                                             host(out["bary"]).astype(np.float64), g)
    assert_grad_close(host(gQ), rgQ, 1e-4, "dL/dQ")
    assert_grad_close(host(gV), rgV, 1e-4, "dL/dV")


def test_rebind_backward_matches_oracle():
    V, F = displaced_icosphere(2, 0.1, 0.3)
    rng = np.random.default_rng(10)
    G = 2000
    gface = rng.integers(0, F.shape[0], G).astype(np.int32)
    gbary = osada_barycentrics(rng, G).astype(np.float32)
    goff = rng.normal(scale=0.05, size=G).astype(np.float32)
    wm = rng.normal(size=(G, 3)).astype(np.float32)
    wq = rng.normal(size=(G, 4)).astype(np.float32)
    ws = rng.normal(size=(G, 3)).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    gV = torch.zeros(V.shape[0], 3, device="cuda")
    bvh.bind_gaussians_backward(dev(gface), dev(gbary), dev(goff), dev(wm), dev(wq), dev(ws), gV)
    ref = oracle.bind_gaussians_backward(V, F, gface, gbary, wm, wq, ws, goff)
    assert_grad_close(host(gV), ref, 1e-4)


def test_autograd_template_fit_gradient_matches_oracle():
    """L = mean d(S_T(V), target)^2 + mean d(S_G, template(V))^2 + mean d(V, target)^2
    on a 162-vertex template: autograd through the CUDA kernels vs the oracle."""
    VT, FT = icosphere(2, radius=0.95)
    VG, FG = displaced_icosphere(3, 0.1, 0.4)
    ft, bt = sample_surface(VT, FT, 4000, seed=11)
    fg, bg = sample_surface(VG, FG, 4000, seed=12)
    SG = points_from(VG, FG, fg, bg)
    tmpl = MeshBVH.from_mesh(dev(VT), dev(FT))
    targ = MeshBVH.from_mesh(dev(VG), dev(FG))
    V = dev(VT).requires_grad_(True)
    VGd = dev(VG)
    ST = Interpolate.apply(V, tmpl, dev(ft), dev(bt))
    cd = Chamfer.apply(ST, V, tmpl, dev(SG), VGd, targ)
    d2v, _ = PointMeshDistance.apply(V, VGd, targ)
    loss = cd[0] + cd[1] + d2v.mean()
    loss.backward()
    # oracle gradient of the same loss
    VT64 = VT.astype(np.float64)
    S = oracle.interpolate(VT64, FT, ft, bt)
    oA = oracle.closest_point(VG, FG, S)
    oB = oracle.closest_point(VT64, FT, SG)
    oV = oracle.closest_point(VG, FG, VT64)
    gS, _ = oracle.closest_point_backward(VG, FG, S, oA["face"], oA["bary"],
                                          np.full(S.shape[0], 1 / S.shape[0]))
    ref = oracle.interpolate_backward(VT.shape[0], FT, ft, bt, gS)
    ref += oracle.closest_point_backward(VT64, FT, SG, oB["face"], oB["bary"],
                                         np.full(SG.shape[0], 1 / SG.shape[0]))[1]
    ref += oracle.closest_point_backward(VG, FG, VT64, oV["face"], oV["bary"],
                                         np.full(VT.shape[0], 1 / VT.shape[0]))[0]
    lref = oA["d2"].mean() + oB["d2"].mean() + oV["d2"].mean()
    assert loss.item() == pytest.approx(lref, rel=1e-5)
    assert_grad_close(host(V.grad), ref, 1e-4)


def test_autograd_chamfer_with_sequence_state_gives_the_same_gradients():
    """Chamfer.apply with a chamfer_state (the ordered, warm-started step) over a few
    optimisation steps: the same per-step loss (up to the float64 sum order) and the same
    gradient as the stateless form on the same vertices (the same faces and weights; the
    vertex gradients are accumulated with float atomics, so up to their order)."""
    from paper_2606_00444_gb300.autograd import chamfer_state
    VT, FT = icosphere(3, radius=0.95)
    VG, FG = displaced_icosphere(3, 0.1, 0.4)
    ft, bt = sample_surface(VT, FT, 6000, seed=21)
    SG = dev(points_from(VG, FG, *sample_surface(VG, FG, 5000, seed=22)))
    tmpl = MeshBVH.from_mesh(dev(VT), dev(FT))
    targ = MeshBVH.from_mesh(dev(VG), dev(FG))
    VGd = dev(VG)
    state = chamfer_state(6000, 5000)
    rng = np.random.default_rng(23)
    Vk = VT.copy()
    for step in range(4):
        grads, losses = [], []
        for st in (None, state):
            V = dev(Vk).requires_grad_(True)
            ST = Interpolate.apply(V, tmpl, dev(ft), dev(bt))
            cd = Chamfer.apply(ST, V, tmpl, SG, VGd, targ, st)
            loss = cd[0] + cd[1]
            loss.backward()
            grads.append(V.grad.clone())
            losses.append(loss.item())
        torch.testing.assert_close(grads[1], grads[0], rtol=1e-5, atol=1e-6 * float(grads[0].abs().max()))
        assert losses[1] == pytest.approx(losses[0], rel=1e-12)
        Vk = (Vk + 0.004 * rng.normal(size=Vk.shape)).astype(np.float32)


def test_autograd_bind_gaussians_matches_oracle_backward():
    V, F = displaced_icosphere(2, 0.1, 0.8)
    rng = np.random.default_rng(13)
    G = 1500
    gface = rng.integers(0, F.shape[0], G).astype(np.int32)
    gbary = osada_barycentrics(rng, G).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    Vd = dev(V).requires_grad_(True)
    mu, quat, scale = BindGaussians.apply(Vd, bvh, dev(gface), dev(gbary))
    wm, wq, ws = (rng.normal(size=s).astype(np.float32) for s in ((G, 3), (G, 4), (G, 3)))
    ((mu * dev(wm)).sum() + (quat * dev(wq)).sum() + (scale * dev(ws)).sum()).backward()
    ref = oracle.bind_gaussians_backward(V, F, gface, gbary, wm, wq, ws)
    assert_grad_close(host(Vd.grad), ref, 1e-4)


@pytest.mark.parametrize("lanes", [1, 4, 32])
def test_chamfer_every_group_width(pair, lanes):
    from paper_2606_00444_gb300 import set_query_group
    VA, FA, SA, VB, FB, SB = pair
    A = MeshBVH.from_mesh(dev(VA), dev(FA))
    B = MeshBVH.from_mesh(dev(VB), dev(FB))
    try:
        set_query_group(lanes)
        out = chamfer(A, dev(SA), B, dev(SB))
    finally:
        set_query_group(0)
    ref, _, _ = oracle.chamfer(VA, FA, SA, VB, FB, SB)
    np.testing.assert_allclose(host(out), ref, rtol=1e-5)


@pytest.mark.parametrize("lanes", [1, 4, 16])
def test_chamfer_warm_start_hints_give_identical_results(pair, lanes):
    """mesh_chamfer_hinted with exact, random, -1 and out-of-range hints, and
    hints aliasing the face outputs, gives the unhinted per-sample results bit for
    bit (one thread or a cooperative group per sample), and the unhinted sums bit
    for bit."""
    from paper_2606_00444_gb300 import set_query_group
    VA, FA, SA, VB, FB, SB = pair
    A = MeshBVH.from_mesh(dev(VA), dev(FA))
    B = MeshBVH.from_mesh(dev(VB), dev(FB))
    rng = np.random.default_rng(21)
    try:
        set_query_group(lanes)
        ref, rps = chamfer(A, dev(SA), B, dev(SB), per_sample=True)
        nA, nB = SA.shape[0], SB.shape[0]
        cases = [(rps["faceA"].clone(), rps["faceB"].clone()),
                 (dev(rng.integers(0, FB.shape[0], nA).astype(np.int32)),
                  dev(rng.integers(0, FA.shape[0], nB).astype(np.int32))),
                 (dev(np.full(nA, -1, np.int32)), None),
                 (None, dev(rng.integers(-3, 3 * FA.shape[0], nB).astype(np.int32)))]
        def same(out, ps):
            assert_identical(ps, rps, "faceA")
            assert_identical(ps, rps, "faceB")
            assert torch.equal(out, ref)

        for hints in cases:
            out, ps = chamfer(A, dev(SA), B, dev(SB), per_sample=True, hints=hints)
            same(out, ps)
        ps = {k: v.clone() for k, v in rps.items()}
        ps["faceA"] = dev(rng.integers(0, FB.shape[0], nA).astype(np.int32))
        ps["faceB"] = dev(rng.integers(0, FA.shape[0], nB).astype(np.int32))
        out, _ = chamfer(A, dev(SA), B, dev(SB), per_sample=True, ps=ps, hints=(ps["faceA"], ps["faceB"]))
        same(out, ps)
    finally:
        set_query_group(0)


@pytest.mark.parametrize("lanes,garbage", [(1, False), (16, False), (16, True), (4, True)])
def test_chamfer_step_over_frames_equals_plain_chamfer(lanes, garbage):
    """mesh_chamfer_step over a skinned sequence (warm start from the previous frame's
    faces, samples run heaviest first by the costs the previous call left in the
    workspace) gives mesh_chamfer's per-sample results bit for bit every frame, and
    its means up to the order of the float64 sums; a workspace of random bytes only
    changes the first frame's order."""
    from paper_2606_00444_gb300 import Workspace, chamfer_step, set_query_group
    V0, F = torus(120, 60)
    skin = TorusSkinning(V0, seed=12)
    fs, bs = sample_surface(V0, F, 3000, seed=5)
    rf, rb = sample_surface(V0, F, 2500, seed=6)
    SB = dev(points_from(V0, F, rf, rb))
    rest = MeshBVH.from_mesh(dev(V0), dev(F), method="ploc")
    A = MeshBVH.from_mesh(dev(V0), dev(F), method="ploc")
    nA, nB = fs.shape[0], SB.shape[0]
    ws = Workspace(torch.device("cuda"))
    if garbage:
        from paper_2606_00444_gb300 import lib
        buf = ws.get(lib().mesh_chamfer_step_workspace_bytes(nA, nB))
        buf.copy_(torch.randint(0, 256, buf.shape, dtype=torch.uint8, device="cuda"))
    ps = dict(faceA=dev(np.full(nA, -1, np.int32)), baryA=torch.empty(nA, 3, device="cuda"),
              dist2A=torch.empty(nA, device="cuda"), faceB=dev(np.full(nB, -1, np.int32)),
              baryB=torch.empty(nB, 3, device="cuda"), dist2B=torch.empty(nB, device="cuda"))
    try:
        set_query_group(lanes)
        for t in range(0, 40, 8):
            A.refit(dev(skin.frame(t)))
            SA = A.interpolate(dev(fs), dev(bs))
            ref, rps = chamfer(A, SA, rest, SB, per_sample=True)
            out = chamfer_step(A, SA, rest, SB, ps, ws)
            for k in rps:
                assert torch.equal(ps[k], rps[k]), (t, k)
            torch.testing.assert_close(out, ref, rtol=1e-12, atol=0)
        assert A.status()[0] == 0 and rest.status()[0] == 0
    finally:
        set_query_group(0)


@pytest.mark.parametrize("lanes", [2, 8, 32])
def test_closest_point_hints_in_cooperative_groups(pair, lanes):
    from paper_2606_00444_gb300 import set_query_group
    VA, FA, SA, VB, FB, SB = pair
    B = MeshBVH.from_mesh(dev(VB), dev(FB))
    rng = np.random.default_rng(22)
    Q = dev(uniform_box(3000, [-1.5] * 3, [1.5] * 3, seed=23))
    try:
        set_query_group(lanes)
        for cut in (np.inf, 0.05):
            ref = B.closest_point(Q, cut)
            for hint in (ref["face"].clone(), dev(rng.integers(-2, FB.shape[0] + 5, 3000).astype(np.int32))):
                got = B.closest_point(Q, cut, hint=hint)
                assert_identical(got, ref)
    finally:
        set_query_group(0)


@pytest.mark.parametrize("mesh", ["ico3", "torus_200k"])
def test_refit_bind_equals_refit_then_bind(mesh):
    """mesh_refit_bind (refit and rebind in one pass, Gaussians grouped by face)
    gives the boxes of mesh_refit and the Gaussians of mesh_bind_gaussians bit for bit
    (the same face and centre arithmetic); 0 to 4 Gaussians per face with normal
    offsets, and the Gaussians also match the oracle."""
    if mesh == "ico3":
        V0, F = icosphere(3)
        V1 = (V0 * 1.1 + 0.05 * np.sin(3 * V0[:, [1, 2, 0]])).astype(np.float32)
    else:
        V0, F = torus(400, 250)
        V1 = TorusSkinning(V0, seed=3000).frame(30)
    rng = np.random.default_rng(31)
    counts = rng.integers(0, 5, F.shape[0])
    gstart = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    G = int(gstart[-1])
    gface = np.repeat(np.arange(F.shape[0], dtype=np.int32), counts)
    gbary = osada_barycentrics(rng, G).astype(np.float32)
    goff = rng.normal(scale=0.01, size=G).astype(np.float32)
    a = MeshBVH.from_mesh(dev(V0), dev(F))
    b = MeshBVH.from_mesh(dev(V0), dev(F))
    for t in range(2):
        Vt = V1 if t == 0 else V0
        a.refit(dev(Vt))
        ref = a.bind_gaussians(dev(gface), dev(gbary), dev(goff))
        got = b.refit_bind(dev(Vt), dev(gstart), dev(gbary), dev(goff))
        assert torch.equal(a.arrays()["nodes_i"], b.arrays()["nodes_i"])        # bits (links are NaN as floats)
        assert torch.equal(a.arrays()["tris"].view(torch.int32), b.arrays()["tris"].view(torch.int32))
        for x, y in zip(got, ref):
            assert torch.equal(x, y)
    pick = rng.choice(G, min(G, 5000), replace=False)
    idx = dev(pick.astype(np.int64))
    check_gaussians((got[0][idx], got[1][idx], got[2][idx]),
                    oracle.bind_gaussians(V0, F, gface[pick], gbary[pick], goff[pick]))
    # vertices already in the buffer (V = None)
    b.update_vertices(dev(V1))
    got2 = b.refit_bind(None, dev(gstart), dev(gbary), dev(goff))
    a.refit(dev(V1))
    ref2 = a.bind_gaussians(dev(gface), dev(gbary), dev(goff))
    for x, y in zip(got2, ref2):
        assert torch.equal(x, y)
    assert b.status()[0] == 0


def test_refit_bind_skewed_counts_and_no_gaussians():
    """The one-thread-per-Gaussian phase over skewed counts: most faces with none, a few
    with thousands (many passes of a block's threads, long runs of empty leaves in the
    slot search); and a CSR with no Gaussians at all (the refit alone)."""
    V0, F = icosphere(4)
    V1 = (V0 * 0.9 + 0.03 * np.cos(5 * V0[:, [2, 0, 1]])).astype(np.float32)
    rng = np.random.default_rng(77)
    nF = F.shape[0]
    counts = np.where(rng.random(nF) < 0.7, 0, rng.integers(1, 3, nF))
    counts[rng.choice(nF, 3, replace=False)] = [3000, 1700, 513]
    gface = np.repeat(np.arange(nF), counts).astype(np.int32)
    gstart = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    G = int(gstart[-1])
    gbary = osada_barycentrics(rng, G).astype(np.float32)
    goff = rng.normal(scale=0.02, size=G).astype(np.float32)
    a = MeshBVH.from_mesh(dev(V0), dev(F))
    b = MeshBVH.from_mesh(dev(V0), dev(F))
    a.refit(dev(V1))
    ref = a.bind_gaussians(dev(gface), dev(gbary), dev(goff))
    got = b.refit_bind(dev(V1), dev(gstart), dev(gbary), dev(goff))
    assert torch.equal(a.arrays()["nodes_i"], b.arrays()["nodes_i"])
    for x, y in zip(got, ref):
        assert torch.equal(x, y)
    assert b.status()[0] == 0
    # no Gaussians: the refit alone
    empty = np.zeros(nF + 1, np.int32)
    c = MeshBVH.from_mesh(dev(V0), dev(F))
    V2 = (V0 * np.float32(1.1)).astype(np.float32)
    c.refit_bind(dev(V2), dev(empty), torch.empty(0, 3, device="cuda"))
    a.refit(dev(V2))
    assert torch.equal(a.arrays()["nodes_i"], c.arrays()["nodes_i"])
    assert c.status()[0] == 0


def test_refit_bind_bad_ranges_set_status():
    V, F = icosphere(2)
    gstart = np.arange(F.shape[0] + 1, dtype=np.int32)
    gstart[5] = 100000                                      # past nG
    gbary = np.full((F.shape[0], 3), 1 / 3, np.float32)
    b = MeshBVH.from_mesh(dev(V), dev(F))
    b.refit_bind(dev(V), dev(gstart), dev(gbary))
    bits, _ = b.status()
    assert bits & 0x1


def test_chamfer_backward_entry_point_matches_oracle(pair):
    """mesh_chamfer_backward through the C ABI: both directions in one launch, the 1/|S|
    mean scaling and dL/d(out) read on the device, against the oracle's closest-point
    backward composed per direction (same faces and weights), component by component;
    a direction whose outputs are all NULL is skipped."""
    from paper_2606_00444_gb300 import chamfer_backward
    VA, FA, SA, VB, FB, SB = pair
    A = MeshBVH.from_mesh(dev(VA), dev(FA))
    B = MeshBVH.from_mesh(dev(VB), dev(FB))
    out, ps = chamfer(A, dev(SA), B, dev(SB), per_sample=True)
    g = torch.tensor([0.7, -1.3], dtype=torch.float64, device="cuda")
    gSA, gSB = torch.empty(SA.shape[0], 3, device="cuda"), torch.empty(SB.shape[0], 3, device="cuda")
    gVA, gVB = torch.zeros(VA.shape[0], 3, device="cuda"), torch.zeros(VB.shape[0], 3, device="cuda")
    chamfer_backward(A, dev(SA), B, dev(SB), g, ps, gSA, gVA, gSB, gVB)
    nA, nB = SA.shape[0], SB.shape[0]
    rSA, rVB = oracle.closest_point_backward(VB, FB, SA, host(ps["faceA"]),
                                             host(ps["baryA"]).astype(np.float64), np.full(nA, 0.7 / nA))
    rSB, rVA = oracle.closest_point_backward(VA, FA, SB, host(ps["faceB"]),
                                             host(ps["baryB"]).astype(np.float64), np.full(nB, -1.3 / nB))
    # the samples lie on (SA) or near (SB) the other surface, so q - c is small and its
    # float32 rounding is an absolute floor of the comparison
    atA = point_grad_atol(SA, VB, 0.7 / nA)
    atB = point_grad_atol(SB, VA, 1.3 / nB)
    assert_grad_close(host(gSA), rSA, 1e-4, "dL/dSA", atA)
    wB = vertex_weight_sums(VB.shape[0], FB, host(ps["faceA"]), host(ps["baryA"]))
    wA = vertex_weight_sums(VA.shape[0], FA, host(ps["faceB"]), host(ps["baryB"]))
    assert_grad_close(host(gVB), rVB, 1e-4, "dL/dVB", atA * wB)
    assert_grad_close(host(gSB), rSB, 1e-4, "dL/dSB", atB)
    assert_grad_close(host(gVA), rVA, 1e-4, "dL/dVA", atB * wA)
    # only the B -> A direction requested: the A -> B outputs stay untouched
    gVB2 = torch.zeros_like(gVB)
    gVA2 = torch.zeros_like(gVA)
    chamfer_backward(A, dev(SA), B, dev(SB), g, ps, None, gVA2, None, None)
    assert torch.equal(gVA2, gVA) or torch.allclose(gVA2, gVA, rtol=1e-6, atol=1e-9)
    assert not gVB2.any()
    assert A.status()[0] == 0 and B.status()[0] == 0
