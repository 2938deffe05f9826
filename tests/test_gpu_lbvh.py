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


def test_refit_equals_build_over_same_topology():
    V0, F = torus(120, 70)
    sk = TorusSkinning(V0, seed=3001)
    bvh, T = check_build(V0, F)
    for t in (7, 23):
        V1 = sk.frame(t)
        bvh.refit(dev(V1))
        boxes = oracle.node_boxes(V1, F, T["perm"], T["first"], T["last"])
        T1 = dict(T, boxes=boxes)
        check_build(V1, F, bvh=bvh, T=T1)


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
