"""GPU NearestSurface (Eq. 1 / Eq. 2) against the brute-force oracle: full
comparison on the single-frame workload (642-vertex template projected onto a
5120-face displaced icosphere, plus 4096 points in [-1.5, 1.5]^3), cutoffs,
ties at shared vertices, degenerate faces, ragged sizes, a varying-topology
frame, and the 1M-particle contact workload on the 200k-face skinned torus in
the benchmark's launch configuration (sampled against the oracle; refit and
rebuild answers compared in full)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_00444_gb300 import MeshBVH
from parity import assert_identical, check_closest, dev, host
from workloads.isosurface import BlobSequence
from workloads.meshes import displaced_icosphere, icosphere, torus, TorusSkinning
from workloads.sampling import uniform_box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    rng = np.random.default_rng(1000)
    phi0 = 2 * np.pi * rng.random()
    VT, FT = icosphere(3)
    VG, FG = displaced_icosphere(4, 0.1, phi0)
    Q = np.concatenate([VT, uniform_box(4096, [-1.5] * 3, [1.5] * 3, seed=1001)])
    return VT, FT, VG, FG, Q


def test_single_frame_full_parity(c1):
    VT, FT, VG, FG, Q = c1
    bvh = MeshBVH.from_mesh(dev(VG), dev(FG))
    out = bvh.closest_point(dev(Q))
    st = check_closest(VG, FG, Q, out)
    assert st["hits"] == Q.shape[0]
    assert bvh.status()[0] == 0


@pytest.mark.parametrize("cut", [0.0, 0.05, 0.2])
def test_cutoff(c1, cut):
    _, _, VG, FG, Q = c1
    bvh = MeshBVH.from_mesh(dev(VG), dev(FG))
    out = bvh.closest_point(dev(Q), max_dist=cut)
    check_closest(VG, FG, Q, out, max_dist=cut)


def test_queries_on_vertices_edges_and_faces(c1):
    """Points on the surface: distance ~0 and equal-distance faces around a vertex."""
    _, _, VG, FG, _ = c1
    e = (VG[FG[:, 0]] + VG[FG[:, 1]]) * np.float32(0.5)
    c = (VG[FG[:, 0]] + VG[FG[:, 1]] + VG[FG[:, 2]]) / np.float32(3.0)
    Q = np.concatenate([VG, e[:1500], c[:1500]]).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(VG), dev(FG))
    out = bvh.closest_point(dev(Q))
    check_closest(VG, FG, Q, out, max_tie_frac=0.05)


def test_degenerate_faces_and_ragged_sizes():
    V, F = icosphere(3)
    F = F.copy()
    F[::5, 2] = F[::5, 1]                 # coincident vertices: segment faces
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    for nq in (1, 127, 129, 1000):
        Q = uniform_box(nq, [-1.3] * 3, [1.3] * 3, seed=nq)
        check_closest(V, F, Q, bvh.closest_point(dev(Q)))
    one = MeshBVH.from_mesh(dev(V), dev(F[7:8]))
    Q = uniform_box(300, [-1.3] * 3, [1.3] * 3, seed=5)
    check_closest(V, F[7:8], Q, one.closest_point(dev(Q)))


def test_partial_outputs_match_full():
    V, F = displaced_icosphere(3, 0.1, 0.3)
    Q = uniform_box(777, [-1.4] * 3, [1.4] * 3, seed=9)
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    full = bvh.closest_point(dev(Q))
    part = bvh.closest_point(dev(Q), want=("dist2",))
    assert torch.equal(full["dist2"], part["dist2"])


def test_varying_topology_frame_projection():
    """Template icosphere (10242 vertices) projected onto one extracted frame."""
    V, F = BlobSequence(2000).mesh(33)
    VT, _ = icosphere(5)
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    out = bvh.closest_point(dev(VT))
    pick = np.random.default_rng(2).choice(VT.shape[0], 1500, replace=False)
    sub = {k: v[dev(pick.astype(np.int64))] for k, v in out.items()}
    check_closest(V, F, VT[pick], sub)


def test_contact_workload_full_size():
    """1M particles, cutoff 0.05, against the 200k-face torus after 4-bone skinning:
    sampled parity with the oracle, and refit answers equal rebuild answers bit for bit."""
    V0, F = torus(400, 250)
    sk = TorusSkinning(V0, seed=3000)
    lo, hi = V0.min(0) - 0.2, V0.max(0) + 0.2
    P = uniform_box(1 << 20, lo, hi, seed=3002)
    Pd = dev(P)
    fixed = MeshBVH.from_mesh(dev(V0), dev(F))
    V1 = sk.frame(57)
    fixed.refit(dev(V1))
    out = fixed.closest_point(Pd, max_dist=0.05)
    rebuilt = MeshBVH.from_mesh(dev(V1), dev(F))
    out2 = rebuilt.closest_point(Pd, max_dist=0.05)
    torch.cuda.synchronize()
    # the two trees are traversed in different orders; the tie rule does not depend on it
    assert_identical(out, out2)
    frac = (out["face"] >= 0).float().mean().item()
    assert 0.03 < frac < 0.4
    rng = np.random.default_rng(4)
    hits = np.nonzero(host(out["face"]) >= 0)[0]
    pick = np.concatenate([rng.choice(hits, 300, replace=False),
                           rng.choice(P.shape[0], 300, replace=False)])
    idx = dev(pick.astype(np.int64))
    sub = {k: v[idx] for k, v in out.items()}
    check_closest(V1, F, P[pick], sub, max_dist=0.05)
    assert fixed.status()[0] == 0


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_every_group_width_matches_oracle(c1, lanes):
    """The cooperative traversal (G lanes per query) gives the oracle's answers for every G,
    with and without a cutoff, including a mesh whose shared stacks overflow to the
    private fallback (queries at the centre of a sphere see every face at once)."""
    from paper_2606_00444_gb300 import set_query_group
    _, _, VG, FG, Q = c1
    bvh = MeshBVH.from_mesh(dev(VG), dev(FG))
    try:
        set_query_group(lanes)
        check_closest(VG, FG, Q, bvh.closest_point(dev(Q)))
        check_closest(VG, FG, Q, bvh.closest_point(dev(Q), max_dist=0.05), max_dist=0.05)
        V, F = icosphere(4)
        centre = MeshBVH.from_mesh(dev(V), dev(F))
        Qc = (uniform_box(64, [-0.02] * 3, [0.02] * 3, seed=lanes)).astype(np.float32)
        check_closest(V, F, Qc, centre.closest_point(dev(Qc)))
        assert bvh.status()[0] == 0 and centre.status()[0] == 0
    finally:
        set_query_group(0)


@pytest.mark.parametrize("variant", list(range(14)))
def test_every_thread_traversal_matches_oracle(c1, variant):
    from paper_2606_00444_gb300 import set_query_group, set_traversal
    _, _, VG, FG, Q = c1
    bvh = MeshBVH.from_mesh(dev(VG), dev(FG))
    try:
        set_query_group(1)
        set_traversal(variant)
        check_closest(VG, FG, Q, bvh.closest_point(dev(Q)))
        check_closest(VG, FG, Q, bvh.closest_point(dev(Q), max_dist=0.05), max_dist=0.05)
    finally:
        set_query_group(0)
        set_traversal(0)


@pytest.mark.parametrize("n", [1, 31, 33, 1000])
def test_warp_packet_traversal_ragged_and_sorted(c1, n):
    """Variant 12 shares one traversal per warp: ragged warps (n not a multiple
    of 32), Morton-sorted and shuffled queries all match the oracle."""
    from paper_2606_00444_gb300 import morton_order, set_query_group, set_traversal
    _, _, VG, FG, Q = c1
    Qn = Q[:n]
    bvh = MeshBVH.from_mesh(dev(VG), dev(FG))
    order = host(morton_order(dev(Qn))).astype(np.int64)
    try:
        set_query_group(1)
        set_traversal(12)
        for Qx in (Qn, Qn[order]):
            check_closest(VG, FG, Qx, bvh.closest_point(dev(Qx)))
            check_closest(VG, FG, Qx, bvh.closest_point(dev(Qx), max_dist=0.05), max_dist=0.05)
        assert bvh.status()[0] == 0
    finally:
        set_query_group(0)
        set_traversal(0)


@pytest.mark.parametrize("variant", [0, 2, 3, 9, 13])
def test_warm_start_hint_gives_identical_answers(c1, variant):
    """mesh_closest_point_hinted: exact previous answers, random faces, -1 and
    out-of-range ids as hints, and the hint aliasing the face output, all give
    the unhinted result bit for bit."""
    from paper_2606_00444_gb300 import set_query_group, set_traversal
    _, _, VG, FG, Q = c1
    bvh = MeshBVH.from_mesh(dev(VG), dev(FG))
    rng = np.random.default_rng(77)
    try:
        set_query_group(1)
        set_traversal(variant)
        for cut in (np.inf, 0.05):
            ref = bvh.closest_point(dev(Q), max_dist=cut)
            n = Q.shape[0]
            hints = [ref["face"].clone(),
                     dev(rng.integers(0, FG.shape[0], n).astype(np.int32)),
                     dev(np.full(n, -1, np.int32)),
                     dev(rng.integers(-5, 2 * FG.shape[0], n).astype(np.int32))]
            for hint in hints:
                got = bvh.closest_point(dev(Q), max_dist=cut, hint=hint)
                assert_identical(got, ref)
            out = {k: v.clone() for k, v in ref.items()}          # hint = the face output itself
            out["face"] = dev(rng.integers(0, FG.shape[0], n).astype(np.int32))
            bvh.closest_point(dev(Q), max_dist=cut, out=out, hint=out["face"])
            assert_identical(out, ref)
        assert bvh.status()[0] == 0
    finally:
        set_query_group(0)
        set_traversal(0)


def test_warm_start_over_a_skinned_sequence_full_size():
    """The physics loop: each frame's contact query is hinted with the previous
    frame's faces (refit tree, 1M particles in Morton order, cutoff 0.05); the
    answers equal the unhinted ones bit for bit."""
    from paper_2606_00444_gb300 import morton_order
    V0, F = torus(400, 250)
    sk = TorusSkinning(V0, seed=3000)
    lo, hi = V0.min(0) - 0.2, V0.max(0) + 0.2
    P = dev(uniform_box(1 << 20, lo, hi, seed=3002))
    P = P[morton_order(P).long()].contiguous()
    bvh = MeshBVH.from_mesh(dev(V0), dev(F))
    face = torch.full((P.shape[0],), -1, dtype=torch.int32, device="cuda")
    for t in (0, 1, 2, 12):
        bvh.refit(dev(sk.frame(t)))
        ref = bvh.closest_point(P, 0.05)
        got = bvh.closest_point(P, 0.05, hint=face)
        assert_identical(got, ref)
        face = got["face"]
    assert bvh.status()[0] == 0


@pytest.mark.parametrize("variant,leaf,block", [(0, 1, 128), (2, 1, 128), (5, 1, 128), (12, 1, 128),
                                                (13, 1, 128), (13, 1, 32), (13, 4, 64),
                                                (12, 8, 128), (2, 4, 32), (3, 1, 64)])
def test_contact_step_equals_plain_queries(variant, leaf, block):
    """mesh_contact (previous faces as hints, queries ordered by the previous step's
    work classes, kept in the workspace -- garbage bytes at the first step) gives
    mesh_closest_point's answers over a skinned sequence, bit for bit."""
    from paper_2606_00444_gb300 import morton_order
    V0, F = torus(120, 70)
    sk = TorusSkinning(V0, seed=3001)
    lo, hi = V0.min(0) - 0.2, V0.max(0) + 0.2
    P = dev(uniform_box(50001, lo, hi, seed=3005))
    P = P[morton_order(P).long()].contiguous()
    bvh = MeshBVH.from_mesh(dev(V0), dev(F))
    bvh.set_query_config(1, variant, block)
    bvh.set_leaf_size(leaf, refit=False)                 # applies from the first refit below
    out = dict(face=torch.full((P.shape[0],), -1, dtype=torch.int32, device="cuda"),
               bary=torch.empty(P.shape[0], 3, device="cuda"), point=torch.empty(P.shape[0], 3, device="cuda"),
               dist2=torch.empty(P.shape[0], device="cuda"))
    from paper_2606_00444_gb300 import Workspace, lib
    ws = Workspace(torch.device("cuda"))
    buf = ws.get(lib().mesh_contact_workspace_bytes(P.shape[0]))
    buf.copy_(torch.randint(0, 256, buf.shape, dtype=torch.uint8))   # garbage work classes
    for t in (0, 5, 10, 40):
        bvh.refit(dev(sk.frame(t)))
        ref = bvh.closest_point(P, 0.05)
        bvh.contact(P, 0.05, out, ws=ws)
        assert_identical(out, ref)
    assert bvh.status()[0] == 0


def test_traversal_counters_are_consistent(c1):
    _, _, VG, FG, Q = c1
    bvh = MeshBVH.from_mesh(dev(VG), dev(FG))
    for cut in (np.inf, 0.05):
        st = bvh.closest_point_stats(dev(Q), cut)
        out = bvh.closest_point(dev(Q), max_dist=cut)
        hits = int((out["face"] >= 0).sum().item())
        assert st["hits"] == hits
        assert st["tests"] >= hits and st["visits"] >= Q.shape[0] // 2
        # a bounded search never works harder than an unbounded one
    assert bvh.closest_point_stats(dev(Q), 0.05)["visits"] < bvh.closest_point_stats(dev(Q))["visits"]


def test_contact_writes_pinned_host_outputs():
    """mesh_contact with its face and distance arrays in pinned host memory (reached
    through mesh_mapped_pointer) gives, in those arrays, what it gives in device
    arrays from the same warm-start faces."""
    import ctypes as C
    from paper_2606_00444_gb300 import Workspace, lib, morton_order
    V0, F = torus(120, 70)
    sk = TorusSkinning(V0, seed=3004)
    lo, hi = V0.min(0) - 0.2, V0.max(0) + 0.2
    P = dev(uniform_box(30001, lo, hi, seed=3008))
    P = P[morton_order(P).long()].contiguous()
    bvh = MeshBVH.from_mesh(dev(V0), dev(F))
    n = P.shape[0]
    d_out = dict(face=torch.full((n,), -1, dtype=torch.int32, device="cuda"),
                 dist2=torch.empty(n, device="cuda"))
    h_out = dict(face=torch.full((n,), -1, dtype=torch.int32).pin_memory(),
                 dist2=torch.empty(n).pin_memory())
    wd, wh = Workspace(torch.device("cuda")), Workspace(torch.device("cuda"))
    for t in (3, 9, 30):
        bvh.refit(dev(sk.frame(t)))
        bvh.contact(P, 0.05, d_out, ws=wd)
        bvh.contact(P, 0.05, h_out, ws=wh)
        torch.cuda.synchronize()
        assert torch.equal(h_out["face"], d_out["face"].cpu())
        assert torch.equal(h_out["dist2"], d_out["dist2"].cpu())
    assert (h_out["face"] >= 0).any()
    ptr = C.c_void_p()
    assert lib().mesh_mapped_pointer(None, C.byref(ptr)) == 1


def wide_records_from_nodes(bvh):
    """The 4-wide records restated on the host from the binary node records (layout
    off_nodes / off_wide): per internal node and side, the child's own node record when
    the child is internal, else the node's slot for that leaf link and an empty slot
    (link INT32_MIN, box +inf..-inf, count 0); slots as in the node records."""
    L = bvh.layout()
    nint = L["n_faces"] - 1
    raw = bvh.storage[L["off_nodes"]:L["off_nodes"] + 64 * nint].cpu().numpy()
    nd = raw.view(np.float32).reshape(nint, 4, 4)
    ni = raw.view(np.int32).reshape(nint, 4, 4)
    W = np.zeros((nint, 8, 4), np.float32)
    Wi = W.view(np.int32)
    empty_lo = np.array([np.inf, np.inf, np.inf, 0], np.float32)
    empty_hi = np.array([-np.inf, -np.inf, -np.inf, 0], np.float32)
    empty_lo.view(np.int32)[3] = -2 ** 31
    for n in range(nint):
        for s in (0, 1):
            link = ni[n, 2 * s, 3]
            if link < 0:
                W[n, 4 * s], W[n, 4 * s + 1] = nd[n, 2 * s], nd[n, 2 * s + 1]
                W[n, 4 * s + 2], W[n, 4 * s + 3] = empty_lo, empty_hi
            else:
                W[n, 4 * s:4 * s + 4] = nd[link]
    return W, L


@pytest.mark.parametrize("leaf", [1, 4])
def test_wide_records_follow_the_tree(c1, leaf):
    """Traversal variant 13 reads 4-wide records written from the node records by its
    first query after a build or refit: they equal the host restatement bit for bit
    (also after a refit to new vertices and with leaf collapse), its answers equal the
    binary traversal's (bounded and unbounded) and the oracle's, and its counting form
    visits fewer records than the binary form visits nodes."""
    _, _, VG, FG, Q = c1
    bvh = MeshBVH.from_mesh(dev(VG), dev(FG), method="ploc")
    bvh.set_leaf_size(leaf)
    rng = np.random.default_rng(5)
    V = VG
    for step in range(2):
        if step:
            V = (VG + 0.01 * rng.standard_normal(VG.shape)).astype(np.float32)
            bvh.refit(dev(V))
        ref, bin_stats = {}, None
        bvh.set_query_config(1, 0)
        for cut in (0.05, np.inf):
            ref[cut] = bvh.closest_point(dev(Q), max_dist=cut)
        bin_stats = bvh.closest_point_stats(dev(Q), 0.05)
        bvh.set_query_config(1, 13)
        got = {cut: bvh.closest_point(dev(Q), max_dist=cut) for cut in (0.05, np.inf)}
        torch.cuda.synchronize()
        W, L = wide_records_from_nodes(bvh)
        raw = bvh.storage[L["off_wide"]:L["off_wide"] + W.nbytes].cpu().numpy()
        assert np.array_equal(raw.view(np.uint32).reshape(W.shape), W.view(np.uint32))
        for cut in (0.05, np.inf):
            assert_identical(got[cut], ref[cut])
        wide_stats = bvh.closest_point_stats(dev(Q), 0.05)
        assert wide_stats["hits"] == bin_stats["hits"]
        assert wide_stats["visits"] < 0.7 * bin_stats["visits"]
    check_closest(V, FG, Q, got[0.05], max_dist=0.05)
    bvh.set_query_config(-1, -1)
    assert bvh.status()[0] == 0


def test_wide_traversal_on_tiny_deep_and_degenerate_meshes():
    """Variant 13 on meshes of 1, 2, 3 and 5 faces (a single record, records with empty
    slots), on 40 copies of one triangle (a 39-level chain of ties) and on faces with
    coincident vertices: the oracle's answers, bounded and unbounded."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [2, 0.5, 0.3]], np.float32)
    meshes = [(V, np.array(F, np.int32)) for F in
              ([[0, 1, 2]], [[0, 1, 2], [1, 3, 2]], [[0, 1, 2], [1, 3, 2], [1, 4, 3]],
               [[0, 1, 2], [1, 3, 2], [1, 4, 3], [0, 4, 2], [3, 4, 0]])]
    meshes.append((V, np.tile(np.array([[0, 1, 2]], np.int32), (40, 1))))
    Vd, Fd = icosphere(2)
    Fd = Fd.copy()
    Fd[::7, 1] = Fd[::7, 0]
    meshes.append((Vd.astype(np.float32), Fd))
    for Vm, Fm in meshes:
        lo, hi = Vm.min(0) - 0.5, Vm.max(0) + 0.5
        Q = uniform_box(300, lo, hi, seed=int(Fm.shape[0]))
        for method in ("lbvh", "ploc"):
            bvh = MeshBVH.from_mesh(dev(Vm), dev(Fm), method=method)
            bvh.set_query_config(1, 13)
            check_closest(Vm, Fm, Q, bvh.closest_point(dev(Q)))
            check_closest(Vm, Fm, Q, bvh.closest_point(dev(Q), max_dist=0.3), max_dist=0.3)
            assert bvh.status()[0] == 0
