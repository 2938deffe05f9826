"""GPU LBVH build and refit against the oracle: Morton keys, sort permutation,
Karras topology and node boxes bit-exact; refit equal to a build over the same
topology.  Sizes span many sort tiles with ragged tails (1280 ... 200k faces)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_00444_gb300 import MeshBVH
from parity import dev, host, gpu_boxes
from workloads.isosurface import BlobSequence
from workloads.meshes import displaced_icosphere, icosphere, torus, TorusSkinning

pytestmark = pytest.mark.gpu


def check_build(V, F, bvh=None, T=None):
    n = F.shape[0]
    if bvh is None:
        bvh = MeshBVH.from_mesh(dev(V), dev(F))
    T = oracle.build_lbvh(V, F) if T is None else T
    A = bvh.arrays()
    torch.cuda.synchronize()
    keys = host(A["keys"]).view(np.uint32)
    assert np.array_equal(keys, T["sorted_keys"]), "sorted Morton keys"
    assert np.array_equal(host(A["perm"]), T["perm"]), "sort permutation"
    assert np.array_equal(host(A["faces"])[:, :3], F), "face table"
    if n > 1:
        ni = host(A["nodes_i"])
        assert np.array_equal(ni[:, 0, 3], T["left"]), "left children"
        assert np.array_equal(ni[:, 2, 3], T["right"]), "right children"
        par = host(A["parent"])
        assert np.array_equal(par >> 1, T["parent"]), "parents"
    assert np.array_equal(gpu_boxes(A, n), T["boxes"]), "node boxes"
    tris = host(A["tris"])
    assert np.array_equal(tris[:, :, :3], V[F[T["perm"]]]), "packed triangles"
    assert np.array_equal(tris[:, 0, 3].view(np.int32), T["perm"]), "leaf face ids"
    bits, _ = bvh.status()
    assert bits == 0
    return bvh, T


@pytest.mark.parametrize("name,maker", [
    ("ico3", lambda: icosphere(3)),
    ("c1_target", lambda: displaced_icosphere(4, 0.1, 1.3)),
    ("torus_ragged", lambda: torus(37, 29)),
    ("blob_frame", lambda: BlobSequence(2000).mesh(17, N=96)),
])
def test_build_bit_exact(name, maker):
    V, F = maker()
    check_build(V, F)


def test_build_full_size_torus_200k():
    V, F = torus(400, 250)
    V = TorusSkinning(V, seed=3000).frame(41)
    check_build(V, F)


def test_tiny_and_degenerate_inputs():
    # one, two, three faces
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [2, 0.5, 0.3]], np.float32)
    for F in ([[0, 1, 2]], [[0, 1, 2], [1, 3, 2]], [[0, 1, 2], [1, 3, 2], [1, 4, 3]]):
        check_build(V, np.array(F, np.int32))
    # every face with the same centroid: equal keys, tree over sorted positions
    rng = np.random.default_rng(1)
    d = rng.normal(size=(300, 3)).astype(np.float32)
    Vs = np.concatenate([d, -d, np.zeros((300, 3), np.float32)]).astype(np.float32)
    Fs = np.stack([np.arange(300), np.arange(300) + 300, np.arange(300) + 600], 1).astype(np.int32)
    bvh, T = check_build(Vs, Fs)
    assert (T["sorted_keys"] == T["sorted_keys"][0]).all()
    # coincident vertices (zero-area faces)
    Vd, Fd = icosphere(2)
    Fd = Fd.copy()
    Fd[::7, 1] = Fd[::7, 0]
    check_build(Vd, Fd)


def test_empty_mesh_builds():
    V = np.zeros((4, 3), np.float32)
    F = np.zeros((0, 3), np.int32)
    bvh = MeshBVH(4, 0)
    bvh.build(dev(V), dev(F))
    out = bvh.closest_point(dev(np.ones((5, 3), np.float32)))
    assert (host(out["face"]) == -1).all() and np.isinf(host(out["dist2"])).all()


def _deform(V, t):
    """A smooth seeded deformation of any mesh (rigid rotation + bend + scale)."""
    a = 0.3 * t
    R = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    W = V.astype(np.float64) @ R.T
    W[:, 2] += 0.2 * np.sin(2.0 * W[:, 0] + t)
    return (W * (1.0 + 0.05 * t)).astype(np.float32)


@pytest.mark.parametrize("name,maker", [
    ("one_block_80", lambda: icosphere(1)),
    ("two_blocks_ragged_1280", lambda: icosphere(3)),
    ("torus_16800", lambda: torus(120, 70)),
    ("blob_frame", lambda: BlobSequence(2000).mesh(17, N=96)),
])
@pytest.mark.parametrize("form", ["fused", "separate"])
def test_refit_equals_build_over_same_topology(name, maker, form):
    """Refit over the build's topology gives the boxes and packed triangles of
    the oracle over the same topology, bit for bit, from either form of the
    vertex update (in the refit pass, or by mesh_update_vertices first)."""
    V0, F = maker()
    bvh, T = check_build(V0, F)
    for t in (1, 3):
        V1 = _deform(V0, t)
        if form == "fused":
            bvh.refit(dev(V1))
        else:
            bvh.update_vertices(dev(V1))
            bvh.refit()
        boxes = oracle.node_boxes(V1, F, T["perm"], T["first"], T["last"])
        check_build(V1, F, bvh=bvh, T=dict(T, boxes=boxes))
        assert np.array_equal(host(bvh.arrays()["verts"])[:, :3], V1)


def test_refit_skinned_torus_and_topology_change_on_one_handle():
    V0, F = torus(120, 70)
    sk = TorusSkinning(V0, seed=3001)
    bvh, T = check_build(V0, F)
    for t in (7, 23):
        V1 = sk.frame(t)
        bvh.refit(dev(V1))
        boxes = oracle.node_boxes(V1, F, T["perm"], T["first"], T["last"])
        check_build(V1, F, bvh=bvh, T=dict(T, boxes=boxes))
    # a new topology in the same storage: the refit plan is derived again
    V2, F2 = torus(100, 61)
    bvh.build(dev(V2), dev(F2))
    T2 = oracle.build_lbvh(V2, F2)
    V3 = _deform(V2, 2)
    bvh.refit(dev(V3))
    boxes = oracle.node_boxes(V3, F2, T2["perm"], T2["first"], T2["last"])
    check_build(V3, F2, bvh=bvh, T=dict(T2, boxes=boxes))


def test_build_and_refit_with_crossing_nodes_past_shared_memory():
    """1.2M faces: some 13k nodes cross the 1024-leaf blocks, more than the
    finishing block holds in shared memory, so every block climbs its share
    through L2.  Build and refit still equal the oracle bit for bit."""
    V0, F = torus(1000, 600)
    bvh, T = check_build(V0, F)
    V1 = TorusSkinning(V0, seed=3002).frame(40)
    bvh.refit(dev(V1))
    boxes = oracle.node_boxes(V1, F, T["perm"], T["first"], T["last"])
    check_build(V1, F, bvh=bvh, T=dict(T, boxes=boxes))


def test_refit_tiny_meshes():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [2, 0.5, 0.3]], np.float32)
    for F in ([[0, 1, 2]], [[0, 1, 2], [1, 3, 2]], [[0, 1, 2], [1, 3, 2], [1, 4, 3]]):
        F = np.array(F, np.int32)
        bvh, T = check_build(V, F)
        V1 = _deform(V, 1)
        bvh.refit(dev(V1))
        boxes = oracle.node_boxes(V1, F, T["perm"], T["first"], T["last"])
        check_build(V1, F, bvh=bvh, T=dict(T, boxes=boxes))


def test_out_of_range_index_sets_status_not_fault():
    V, F = icosphere(1)
    F = F.copy()
    F[3, 2] = 10 ** 6
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    bits, _ = bvh.status()
    assert bits & 0x1
    assert host(bvh.arrays()["faces"])[3, 2] == 0


@pytest.mark.parametrize("n", [1, 2, 1000, 4099, 250000])
def test_point_morton_order_bit_exact(n):
    """mesh_morton_order keys a point p as the zero-area face (p, p, p): the oracle's
    face recipe and stable sort give the expected permutation exactly."""
    from paper_2606_00444_gb300 import morton_order
    from workloads.sampling import uniform_box
    P = uniform_box(n, [-1, -2, -0.5], [1, 2, 0.5], seed=n)
    if n > 10:
        P[::7] = P[3]                                    # duplicates: ties broken by index
    idx = np.arange(n, dtype=np.int32)
    keys = oracle.morton(P, np.stack([idx, idx, idx], 1))
    _, perm = oracle.sort_pairs(keys)
    got = host(morton_order(dev(P)))
    assert np.array_equal(got, perm)
