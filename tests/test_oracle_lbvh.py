"""Pins for the oracle's LBVH build: Morton keys, sort, Karras hierarchy, boxes.

The paper only says the acceleration structure is built once from F0 and
stores indices (Sec. 3.4) and that the varying-topology baseline rebuilds it
every frame (Sec. 4.1); the construction is Karras (2012).  The checks here
are properties that pin each step without re-running its own recipe: key
decoding against the centroid grid cell, extreme corners, permutation
invariance, a library stable sort, hand-built trees, the radix-tree
invariants, and box containment / unions.
"""
import numpy as np
import pytest

import oracle
from workloads.meshes import icosphere, displaced_icosphere, torus
from workloads.isosurface import BlobSequence


def decode(keys):
    keys = np.asarray(keys, np.uint64)
    q = np.zeros((keys.shape[0], 3), np.int64)
    for bit in range(10):
        for ax in range(3):
            q[:, ax] |= ((keys >> np.uint64(3 * bit + (2 - ax))) & np.uint64(1)).astype(np.int64) << bit
    return q


def test_single_face_key_is_zero():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    assert oracle.morton(V, np.array([[0, 1, 2]], np.int32))[0] == 0


def test_extreme_corners():
    V = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.2, 0.7]], np.float32)
    F = np.array([[0, 0, 0], [1, 1, 1], [2, 2, 2]], np.int32)
    k = oracle.morton(V, F)
    assert k[0] == 0 and k[1] == (1 << 30) - 1
    q = decode(k)[2]
    # centroid (0.5, 0.2, 0.7) of a unit box: cells floor(1024 * t)
    assert tuple(q) == (512, 204, 716)


@pytest.mark.parametrize("maker", [lambda: displaced_icosphere(4, 0.1, 1.0),
                                   lambda: torus(40, 25)])
def test_key_decodes_to_the_centroid_cell(maker):
    V, F = maker()
    k = oracle.morton(V, F)
    q = decode(k)
    s = V.astype(np.float64)[F].sum(1)
    lo, hi = s.min(0), s.max(0)
    t = (s - lo) / (hi - lo)
    assert (q >= 0).all() and (q <= 1023).all()
    # the cell contains the normalised centroid, up to float32 rounding of the recipe
    assert (q / 1024.0 <= t + 1e-6).all()
    assert (t < (q + 1) / 1024.0 + 1e-6).all()
    assert (k < (1 << 30)).all()


def test_keys_follow_face_permutation():
    V, F = displaced_icosphere(3, 0.1, 0.2)
    rng = np.random.default_rng(3)
    p = rng.permutation(F.shape[0])
    np.testing.assert_array_equal(oracle.morton(V, F[p]), oracle.morton(V, F)[p])


def test_sort_equals_library_stable_sort():
    rng = np.random.default_rng(4)
    for n in (1, 2, 3, 100, 5000):
        keys = rng.integers(0, 64, size=n).astype(np.uint32)   # many duplicates
        sk, perm = oracle.sort_pairs(keys)
        ref = np.argsort(keys, kind="stable")
        np.testing.assert_array_equal(perm, ref)
        np.testing.assert_array_equal(sk, keys[ref])


def test_karras_hand_examples():
    # keys 1, 2, 4, 5: root [0,3] splits after 1; nodes 1 = [0,1], 2 = [2,3]
    left, right, parent, first, last = oracle.karras(np.array([1, 2, 4, 5], np.uint32))
    np.testing.assert_array_equal(left, [1, -1, -3])
    np.testing.assert_array_equal(right, [2, -2, -4])
    np.testing.assert_array_equal(parent, [-1, 0, 0, 1, 1, 2, 2])
    # five equal keys split by their sorted positions: root [0,4] after 3
    left, right, parent, first, last = oracle.karras(np.full(5, 7, np.uint32))
    np.testing.assert_array_equal(left, [3, -1, -3, 1])
    np.testing.assert_array_equal(right, [-5, -2, -4, 2])
    # n = 2: one internal node over two leaves; n = 1: no internal node
    left, right, parent, _, _ = oracle.karras(np.array([3, 9], np.uint32))
    np.testing.assert_array_equal(left, [-1]) and np.testing.assert_array_equal(right, [-2])
    left, right, parent, _, _ = oracle.karras(np.array([3], np.uint32))
    assert left.shape == (0,) and list(parent) == [-1]


def aug(keys, i):
    return (int(keys[i]) << 32) | int(i)


def check_radix_tree(keys, left, right, parent, first, last):
    """Invariants that determine the binary radix tree over augmented keys uniquely."""
    n = keys.shape[0]
    seen_leaf = np.zeros(n, int)
    seen_int = np.zeros(n - 1, int)
    seen_int[0] += 1
    for i in range(n - 1):
        f, l = first[i], last[i]
        assert f == i or l == i                      # Karras numbering
        assert f < l
        kf, kl = aug(keys, f), aug(keys, l)
        b = (kf ^ kl).bit_length() - 1               # highest differing bit
        ranges = []
        for ch in (left[i], right[i]):
            if ch < 0:
                j = -ch - 1
                seen_leaf[j] += 1
                assert parent[n - 1 + j] == i
                ranges.append((j, j))
            else:
                seen_int[ch] += 1
                assert parent[ch] == i
                ranges.append((first[ch], last[ch]))
        (a0, a1), (b0, b1) = ranges
        assert a0 == f and b1 == l and a1 + 1 == b0  # children partition the range
        for j in range(a0, a1 + 1):
            assert not (aug(keys, j) >> b) & 1
        for j in range(b0, b1 + 1):
            assert (aug(keys, j) >> b) & 1
        assert (kf >> (b + 1)) == (kl >> (b + 1))
    assert (seen_leaf == 1).all() and (seen_int == 1).all()
    assert parent[0] == -1


def test_karras_radix_tree_invariants_random():
    rng = np.random.default_rng(5)
    for n in (2, 3, 7, 64, 513):
        for hi in (4, 1 << 30):
            keys = np.sort(rng.integers(0, hi, size=n).astype(np.uint32))
            check_radix_tree(keys, *oracle.karras(keys))


def test_karras_on_a_mesh_and_depth_bound():
    V, F = displaced_icosphere(4, 0.1, 0.4)
    T = oracle.build_lbvh(V, F)
    n = F.shape[0]
    check_radix_tree(T["sorted_keys"], T["left"], T["right"], T["parent"], T["first"], T["last"])
    def dep(x):
        d = 0
        while T["parent"][x] != -1:
            x = T["parent"][x]
            d += 1
        return d
    dmax = max(dep(n - 1 + j) for j in range(0, n, 7))
    assert dmax <= 30 + int(np.ceil(np.log2(n))) + 1


def test_boxes_are_unions_and_contain_their_faces():
    seq = BlobSequence(7)
    V, F = seq.mesh(10, N=40)
    T = oracle.build_lbvh(V, F)
    n = F.shape[0]
    box = T["boxes"]
    for i in range(n - 1):
        ch = []
        for c in (T["left"][i], T["right"][i]):
            ch.append(box[n - 1 + (-c - 1)] if c < 0 else box[c])
        np.testing.assert_array_equal(box[i, :3], np.minimum(ch[0][:3], ch[1][:3]))
        np.testing.assert_array_equal(box[i, 3:], np.maximum(ch[0][3:], ch[1][3:]))
    tri = V[F[T["perm"]]]                             # leaf order
    np.testing.assert_array_equal(box[n - 1:, :3], tri.min(1))
    np.testing.assert_array_equal(box[n - 1:, 3:], tri.max(1))
    used = V[np.unique(F)]
    np.testing.assert_array_equal(box[0, :3], used.min(0))
    np.testing.assert_array_equal(box[0, 3:], used.max(0))


def test_refit_equals_rebuild_boxes_for_same_topology():
    V, F = torus(30, 20)
    T = oracle.build_lbvh(V, F)
    V2 = (V * 1.3 + np.float32(0.2)).astype(np.float32)
    box2 = oracle.node_boxes(V2, F, T["perm"], T["first"], T["last"])
    # boxes of the moved mesh contain every moved face; union property holds
    n = F.shape[0]
    tri = V2[F[T["perm"]]]
    np.testing.assert_array_equal(box2[n - 1:, :3], tri.min(1))
    np.testing.assert_array_equal(box2[0, 3:], V2.max(0))
