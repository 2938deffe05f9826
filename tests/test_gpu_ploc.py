"""GPU agglomerative build (mesh_build_ploc) against the oracle's PLOC tree: leaf
order, leaf-order keys, children, parents and node boxes bit-exact on meshes from
one face to 200k faces (ties of equal boxes, zero-area faces, ragged blocks);
refit of that topology equal to the oracle's boxes; NearestSurface on it equal to
the brute-force oracle and to the Karras tree's answers; fewer node visits than
the Karras tree on the contact workload."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_00444_gb300 import MeshBVH
from parity import assert_identical, check_closest, dev, gpu_boxes, host
from workloads.isosurface import BlobSequence
from workloads.meshes import displaced_icosphere, icosphere, torus, TorusSkinning
from workloads.sampling import uniform_box

pytestmark = pytest.mark.gpu


def check_ploc(V, F, bvh=None):
    n = F.shape[0]
    if bvh is None:
        bvh = MeshBVH.from_mesh(dev(V), dev(F), method="ploc")
    T = oracle.build_ploc(V, F)
    A = bvh.arrays()
    torch.cuda.synchronize()
    assert np.array_equal(host(A["perm"]), T["perm"]), "leaf order"
    assert np.array_equal(host(A["keys"]).view(np.uint32), T["leaf_keys"]), "leaf-order keys"
    if n > 1:
        ni = host(A["nodes_i"])
        assert np.array_equal(ni[:, 0, 3], T["left"]), "left children"
        assert np.array_equal(ni[:, 2, 3], T["right"]), "right children"
        par = host(A["parent"])
        assert np.array_equal(par >> 1, T["parent"]), "parents"
    assert np.array_equal(gpu_boxes(A, n), T["boxes"]), "node boxes"
    tris = host(A["tris"])
    assert np.array_equal(tris[:, :, :3], V[F[T["perm"]]]), "packed triangles"
    assert bvh.status()[0] == 0
    return bvh, T


@pytest.mark.parametrize("name,maker", [
    ("ico3", lambda: icosphere(3)),
    ("c1_target", lambda: displaced_icosphere(4, 0.1, 1.3)),
    ("torus_ragged", lambda: torus(37, 29)),
    ("blob_frame", lambda: BlobSequence(2000).mesh(17, N=96)),
])
def test_build_bit_exact(name, maker):
    V, F = maker()
    check_ploc(V, F)


def test_build_full_size_torus_200k():
    V, F = torus(400, 250)
    check_ploc(V, F)


def test_tiny_ties_and_degenerate_inputs():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [2, 0.5, 0.3]], np.float32)
    for F in ([[0, 1, 2]], [[0, 1, 2], [1, 3, 2]], [[0, 1, 2], [1, 3, 2], [1, 4, 3]],
              [[0, 1, 2], [1, 3, 2], [1, 4, 3], [0, 4, 2], [3, 4, 0]]):
        check_ploc(V, np.array(F, np.int32))
    # 40 copies of one triangle: every union has the same area (ties everywhere); the
    # chain it clusters into is 39 levels deep, inside the traversal's 64 (600 copies
    # chain past it: test_deep_agglomerative_tree_falls_back_to_the_karras_tree)
    Fs = np.tile(np.array([[0, 1, 2]], np.int32), (40, 1))
    check_ploc(V, Fs)
    # zero-area faces
    Vd, Fd = icosphere(2)
    Fd = Fd.copy()
    Fd[::7, 1] = Fd[::7, 0]
    check_ploc(Vd, Fd)


def test_refit_of_the_ploc_topology():
    V0, F = torus(120, 70)
    sk = TorusSkinning(V0, seed=3003)
    bvh, T = check_ploc(V0, F)
    for t in (5, 40):
        V = sk.frame(t)
        bvh.refit(dev(V))
        A = bvh.arrays()
        torch.cuda.synchronize()
        want = oracle.node_boxes(V, F, T["perm"], T["first"], T["last"])
        assert np.array_equal(gpu_boxes(A, F.shape[0]), want)


def test_queries_on_the_ploc_tree():
    rng = np.random.default_rng(1000)
    VG, FG = displaced_icosphere(4, 0.1, 2 * np.pi * rng.random())
    Q = np.concatenate([icosphere(3)[0], uniform_box(4096, [-1.5] * 3, [1.5] * 3, seed=1001)])
    ploc = MeshBVH.from_mesh(dev(VG), dev(FG), method="ploc")
    lbvh = MeshBVH.from_mesh(dev(VG), dev(FG))
    for cut in (np.inf, 0.05):
        got = ploc.closest_point(dev(Q), cut)
        check_closest(VG, FG, Q, got, max_dist=cut)
        assert_identical(got, lbvh.closest_point(dev(Q), cut))


def test_contact_workload_fewer_visits_same_answers():
    """1M particles, cutoff 0.05, on a skinned frame of the 200k-face torus refit from
    its rest pose: the agglomerative tree answers as the Karras tree does (bit for bit),
    a sample agrees with the oracle, and it visits fewer nodes."""
    from paper_2606_00444_gb300 import morton_order
    V0, F = torus(400, 250)
    sk = TorusSkinning(V0, seed=3000)
    lo, hi = V0.min(0) - 0.2, V0.max(0) + 0.2
    P = dev(uniform_box(1 << 20, lo, hi, seed=3002))
    P = P[morton_order(P).long()].contiguous()
    ploc = MeshBVH.from_mesh(dev(V0), dev(F), method="ploc")
    lbvh = MeshBVH.from_mesh(dev(V0), dev(F))
    V1 = sk.frame(30)
    ploc.refit(dev(V1))
    lbvh.refit(dev(V1))
    got = ploc.closest_point(P, 0.05)
    assert_identical(got, lbvh.closest_point(P, 0.05))
    pick = np.random.default_rng(5).choice(P.shape[0], 400, replace=False)
    idx = dev(pick.astype(np.int64))
    check_closest(V1, F, host(P)[pick], {k: v[idx] for k, v in got.items()}, max_dist=0.05)
    sp, sl = ploc.closest_point_stats(P, 0.05), lbvh.closest_point_stats(P, 0.05)
    assert sp["hits"] == sl["hits"]
    assert sp["visits"] < 0.95 * sl["visits"]
    assert ploc.status()[0] == 0


def test_every_tree_consumer_runs_on_the_ploc_tree():
    """Warm-started queries, the contact step, signed distance, k-NN projection, the fused
    refit + rebind, Chamfer and the closest-point backward pass give on the agglomerative
    tree what they give on the Karras tree of the same mesh (bit for bit for the
    nearest-face queries)."""
    from paper_2606_00444_gb300 import chamfer, morton_order
    from workloads.sampling import osada_barycentrics, sample_surface
    V0, F = torus(120, 70)
    sk = TorusSkinning(V0, seed=3001)
    V1 = sk.frame(20)
    ploc = MeshBVH.from_mesh(dev(V0), dev(F), method="ploc")
    lbvh = MeshBVH.from_mesh(dev(V0), dev(F))
    for b in (ploc, lbvh):
        b.refit(dev(V1))
    lo, hi = V0.min(0) - 0.2, V0.max(0) + 0.2
    P = dev(uniform_box(40001, lo, hi, seed=3006))
    P = P[morton_order(P).long()].contiguous()
    # hinted queries and the contact step
    ref = lbvh.closest_point(P, 0.05)
    rng = np.random.default_rng(7)
    hint = dev(rng.integers(-1, F.shape[0], P.shape[0]).astype(np.int32))
    assert_identical(ploc.closest_point(P, 0.05, hint=hint), ref)
    out = {k: v.clone() for k, v in ref.items()}
    ploc.contact(P, 0.05, out)
    assert_identical(out, ref)
    # signed distance: the same face, distance and sign, bit for bit
    sp, sl = ploc.signed_distance(P, 0.05), lbvh.signed_distance(P, 0.05)
    assert torch.equal(sp["face"], sl["face"])
    assert torch.equal(sp["sdist"], sl["sdist"])
    # k-NN weighted projection (k faces by distance: equal except near ties)
    pk, fk, _ = ploc.knn_project(P[:5000], k=4, want_faces=True)
    pl, fl, _ = lbvh.knn_project(P[:5000], k=4, want_faces=True)
    rows = (fk == fl).all(1)
    assert (~rows).sum().item() <= 10
    assert torch.equal(pk[rows], pl[rows])
    # fused refit + rebind: the Gaussians do not depend on the tree
    counts = np.full(F.shape[0], 2, np.int32)
    gstart = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    gface = np.repeat(np.arange(F.shape[0], dtype=np.int32), counts)
    gbary = osada_barycentrics(rng, int(gstart[-1])).astype(np.float32)
    got = ploc.refit_bind(dev(V1), dev(gstart), dev(gbary))
    want = lbvh.bind_gaussians(dev(gface), dev(gbary))
    for x, y in zip(got, want):
        torch.testing.assert_close(x, y, rtol=0, atol=1e-6)
    # Chamfer against the rest mesh, per-sample results
    rest_p = MeshBVH.from_mesh(dev(V0), dev(F), method="ploc")
    rest_l = MeshBVH.from_mesh(dev(V0), dev(F))
    sf, sb = (dev(a) for a in sample_surface(V0, F, 4000, seed=3007))
    SA = ploc.interpolate(sf, sb)
    SB = rest_l.interpolate(sf, sb)
    cp, psp = chamfer(ploc, SA, rest_p, SB, per_sample=True)
    cl, psl = chamfer(lbvh, SA, rest_l, SB, per_sample=True)
    assert_identical(psp, psl, "faceA")
    assert_identical(psp, psl, "faceB")
    assert torch.equal(cp, cl)
    # backward of the point-to-mesh distance
    Q = P[:3000].contiguous()
    rp, rl = ploc.closest_point(Q), lbvh.closest_point(Q)
    assert_identical(rp, rl)
    same = rp["face"] == rl["face"]
    g = torch.ones(Q.shape[0], device="cuda")
    gQp, gVp = torch.empty_like(Q), torch.zeros(V1.shape[0], 3, device="cuda")
    gQl, gVl = torch.empty_like(Q), torch.zeros(V1.shape[0], 3, device="cuda")
    ploc.closest_point_backward(Q, rp["face"], rp["bary"], g, gQp, gVp)
    lbvh.closest_point_backward(Q, rl["face"], rl["bary"], g, gQl, gVl)
    assert torch.equal(gQp[same], gQl[same])
    if bool(same.all()):
        torch.testing.assert_close(gVp, gVl, rtol=1e-5, atol=1e-6)
    assert ploc.status()[0] == 0


def test_large_mesh_1_6m_faces():
    """A 1.6M-face torus: the agglomerative tree is a valid layout (the leaf order is a
    permutation; every node but the root fills exactly one child slot, and its parent
    link names that slot) and answers bounded and unbounded queries as the Karras tree
    does."""
    V, F = torus(1000, 800)
    n = F.shape[0]
    ploc = MeshBVH.from_mesh(dev(V), dev(F), method="ploc")
    lbvh = MeshBVH.from_mesh(dev(V), dev(F))
    A = ploc.arrays()
    perm = A["perm"].long()
    assert torch.equal(torch.sort(perm).values, torch.arange(n, device="cuda"))
    par = A["parent"].long()
    assert par[0].item() == -1
    links = A["nodes_i"][:, [0, 2], 3].reshape(-1).long()          # child of each parent slot
    node_ids = torch.where(links >= 0, links, (n - 1) + (-links - 1))
    seen = torch.zeros(2 * n - 1, dtype=torch.int64, device="cuda")
    seen.index_add_(0, node_ids, torch.ones_like(node_ids))
    assert int(seen[0]) == 0 and bool((seen[1:] == 1).all())
    slots = torch.arange(2 * (n - 1), device="cuda")
    assert torch.equal(par[node_ids], slots)                         # parent = 2 * node + side
    Q = dev(uniform_box(200000, V.min(0) - 0.1, V.max(0) + 0.1, seed=77))
    for cut in (0.02, np.inf):
        assert_identical(ploc.closest_point(Q, cut), lbvh.closest_point(Q, cut))
    assert ploc.status()[0] == 0


def test_benchmarked_contact_step_against_the_oracle_full_size():
    """The step the benchmark times, at full size and in its launch configuration:
    mesh_contact on the agglomerative tree built once from the rest pose and refit to a
    skinned frame, traversal chosen by the autotuner on this workload, 1M Morton-ordered
    particles, cutoff 0.05, warm-started from the previous step's faces and ordered by
    its work classes.  Every output equals the plain query's bit for bit, and 4096
    particles with a contact plus 4096 random ones match the brute-force oracle."""
    from paper_2606_00444_gb300 import Workspace, morton_order
    from paper_2606_00444_gb300.tune import tune_closest_point
    V0, F = torus(400, 250)
    sk = TorusSkinning(V0, seed=3000)
    lo, hi = V0.min(0) - 0.2, V0.max(0) + 0.2
    P = dev(uniform_box(1 << 20, lo, hi, seed=3002))
    P = P[morton_order(P).long()].contiguous()
    fixed = MeshBVH.from_mesh(dev(V0), dev(F), method="ploc")
    fixed.refit(dev(sk.frame(0)))
    tuned = tune_closest_point(fixed, P, 0.05, force=True)
    n = P.shape[0]
    out = dict(face=torch.full((n,), -1, dtype=torch.int32, device="cuda"),
               bary=torch.empty(n, 3, device="cuda"), point=torch.empty(n, 3, device="cuda"),
               dist2=torch.empty(n, device="cuda"))
    ws = Workspace(torch.device("cuda"))
    for t in (0, 1, 2):                          # steps 1 and 2 are warm-started and ordered
        V1 = sk.frame(t)
        fixed.refit(dev(V1))
        fixed.contact(P, 0.05, out, ws=ws)
    plain = fixed.closest_point(P, 0.05)
    assert_identical(out, plain)
    hits = np.nonzero(host(out["face"]) >= 0)[0]
    rng = np.random.default_rng(11)
    pick = np.concatenate([rng.choice(hits, 4096, replace=False),
                           rng.choice(n, 4096, replace=False)])
    idx = dev(pick.astype(np.int64))
    sub = {k: v[idx] for k, v in out.items()}
    Pn = host(P)[pick]
    st = check_closest(V1, F, Pn, sub, max_dist=0.05,
                       ref=oracle.closest_point(V1, F, Pn, 0.05, parallel=True))
    print(f"contact step (lanes {tuned['lanes']}, variant {tuned['variant']}): "
          f"{st['hits']} hits of {st['n']} sampled, {st['ties']} float32 tie mismatches, "
          f"{st['cutoff_edge']} at the cutoff")
    assert fixed.status()[0] == 0


@pytest.mark.parametrize("method", ["lbvh", "ploc"])
def test_leaf_collapse_links_equal_the_oracle(method):
    """At leaf sizes 2, 3, 4 and 8 the refit writes, for every internal node, the child links
    of the oracle's collapse (a subtree of at most L faces as one leaf range), on both tree
    kinds and on a mesh larger than one refit block; back at L = 1 the links are the
    tree's own."""
    V, F = torus(120, 70)
    ref = oracle.build_lbvh(V, F) if method == "lbvh" else oracle.build_ploc(V, F)
    b = MeshBVH.from_mesh(dev(V), dev(F), method=method)
    for L in (2, 3, 4, 8, 1):
        b.set_leaf_size(L)
        links = host(b.arrays()["nodes_i"])[:, [0, 1, 2, 3], 3]          # lo_L, hi_L, lo_R, hi_R
        want = oracle.collapse(ref["left"], ref["right"], ref["first"], ref["last"], L)
        np.testing.assert_array_equal(links, want, err_msg=f"leaf size {L}")
    assert b.status()[0] == 0


def test_leaf_collapse_gives_identical_answers_in_every_search():
    """Every search form reads collapsed leaf ranges: at leaf sizes 2, 4 and 8 the
    one-thread variants, the cooperative groups, the contact step, the warm-started query,
    the signed distance, the Chamfer and the k-NN projection give the L = 1 answers bit for
    bit, and the oracle's."""
    from paper_2606_00444_gb300 import Workspace, chamfer, morton_order, set_query_group, set_traversal
    from workloads.sampling import sample_surface
    V0, F = torus(120, 70)
    V1 = TorusSkinning(V0, seed=3001).frame(15)
    b = MeshBVH.from_mesh(dev(V0), dev(F), method="ploc")
    b.refit(dev(V1))
    lo, hi = V0.min(0) - 0.2, V0.max(0) + 0.2
    P = dev(uniform_box(20001, lo, hi, seed=3010))
    P = P[morton_order(P).long()].contiguous()
    sf, sb = (dev(a) for a in sample_surface(V0, F, 3000, seed=3011))
    S = b.interpolate(sf, sb)
    rest = MeshBVH.from_mesh(dev(V0), dev(F))
    SR = rest.interpolate(sf, sb)

    def answers():
        out = {}
        try:
            for v in (0, 1, 2, 5, 10, 12, 13):
                set_query_group(1)
                set_traversal(v)
                for cut in (0.05, np.inf):
                    out[(v, cut)] = b.closest_point(P, cut)
            for g in (4, 32):
                set_query_group(g)
                out[("g", g)] = b.closest_point(P[:3000].contiguous(), 0.05)
        finally:
            set_query_group(0)
            set_traversal(0)
        ct = {k: v.clone() for k, v in out[(0, 0.05)].items()}
        b.contact(P, 0.05, ct, ws=Workspace(torch.device("cuda")))
        out["contact"] = ct
        out["hinted"] = b.closest_point(P, 0.05, hint=out[(0, 0.05)]["face"])
        out["signed"] = b.signed_distance(P, 0.05)
        out["chamfer"] = chamfer(b, S, rest, SR, per_sample=True)
        out["knn"] = b.knn_project(P[:4000].contiguous(), k=4, want_faces=True)
        return out

    base = answers()
    Pn = host(P)
    check_closest(V1, F, Pn, base[(0, 0.05)], max_dist=0.05)
    for L in (2, 4, 8):
        b.set_leaf_size(L)
        got = answers()
        for key in base:
            if key == "chamfer":
                assert torch.equal(got[key][0], base[key][0])
                assert_identical(got[key][1], base[key][1], "faceA")
                assert_identical(got[key][1], base[key][1], "faceB")
            elif key == "knn":
                for x, y in zip(got[key], base[key]):
                    assert torch.equal(x, y), f"knn, leaf size {L}"
            elif key == "signed":
                assert torch.equal(got[key]["face"], base[key]["face"])
                assert torch.equal(got[key]["sdist"].abs(), base[key]["sdist"].abs())
            else:
                assert_identical(got[key], base[key])
    assert b.status()[0] == 0


def test_deep_agglomerative_tree_falls_back_to_the_karras_tree():
    """300 copies of one triangle: clustering would chain them 299 levels deep, past the
    64 levels every traversal keeps.  mesh_build_ploc measures the depth, builds the
    Karras tree instead (equal to the oracle's bit for bit) and sets the informational
    bit MESH_DEV_DEEP_TREE; queries then tie across all 300 faces and return face 0."""
    n = 300
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    F = np.tile(np.array([[0, 1, 2]], np.int32), (n, 1))
    b = MeshBVH.from_mesh(dev(V), dev(F), method="ploc")
    ref = oracle.build_lbvh(V, F)
    A = b.arrays()
    assert np.array_equal(host(A["perm"]), ref["perm"])
    assert np.array_equal(host(A["parent"]) >> 1, ref["parent"])
    Q = uniform_box(500, [-1, -1, -1], [2, 2, 2], seed=9)
    out = b.closest_point(dev(Q))
    check_closest(V, F, Q, out)
    assert (host(out["face"]) == 0).all()
    bits, _ = b.status()
    assert bits == 0x10
    # the limit itself: a chain of 64 internal nodes is kept, one of 65 is not
    for copies, deep in ((65, False), (66, True)):
        Fc = np.tile(np.array([[0, 1, 2]], np.int32), (copies, 1))
        bc = MeshBVH.from_mesh(dev(V), dev(Fc), method="ploc")
        want = oracle.build_lbvh(V, Fc) if deep else oracle.build_ploc(V, Fc)
        assert np.array_equal(host(bc.arrays()["parent"]) >> 1, want["parent"]), copies
        assert bc.status()[0] == (0x10 if deep else 0), copies
    # a mesh of ordinary depth keeps its agglomerative tree and sets nothing
    V2, F2 = torus(40, 25)
    b2 = MeshBVH.from_mesh(dev(V2), dev(F2), method="ploc")
    assert np.array_equal(host(b2.arrays()["perm"]), oracle.build_ploc(V2, F2)["perm"])
    assert b2.status()[0] == 0
