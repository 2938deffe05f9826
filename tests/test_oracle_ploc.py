"""Pins of the oracle's agglomerative build (orc_ploc: parallel locally-ordered
clustering, Meister & Bittner 2018, written as its iterations), which builds the
tree of a fixed-topology mesh once: hand-worked trees, the tie rule, tiny sizes,
the layout invariants shared with the Karras tree, the first iteration's merges
against a brute-force mutual-nearest-neighbour search, and the effect of the
search radius."""
import numpy as np
import pytest

import oracle
from workloads.meshes import torus


def boxes_on_line(starts, width=1.0):
    b = np.zeros((len(starts), 6), np.float32)
    b[:, 0] = starts
    b[:, 3] = np.asarray(starts, np.float32) + np.float32(width)
    b[:, 4:6] = 1.0
    return b


def check_layout(order, left, right, parent, first, last, n):
    """A binary tree over in-order leaves 0..n-1, internal node k numbered by the end of
    its range not shared with its sibling (root 0)."""
    assert sorted(order.tolist()) == list(range(n))
    if n == 1:
        assert parent.tolist() == [-1]
        return
    assert first[0] == 0 and last[0] == n - 1 and parent[0] == -1
    seen_leaf = np.zeros(n, int)
    seen_int = np.zeros(n - 1, int)
    seen_int[0] = 1
    for k in range(n - 1):
        assert k in (first[k], last[k])
        a, b = left[k], right[k]
        la = (first[a], last[a]) if a >= 0 else (-a - 1, -a - 1)
        lb = (first[b], last[b]) if b >= 0 else (-b - 1, -b - 1)
        assert la[0] == first[k] and lb[1] == last[k] and la[1] + 1 == lb[0]
        for c, side in ((a, 0), (b, 1)):
            if c >= 0:
                assert parent[c] == k
                assert c == (last[c] if side == 0 else first[c])
                seen_int[c] += 1
            else:
                assert parent[(n - 1) - c - 1] == k
                seen_leaf[-c - 1] += 1
    assert np.all(seen_leaf == 1) and np.all(seen_int == 1)


def union_area32(a, b):
    lo = np.minimum(a[..., :3], b[..., :3])
    hi = np.maximum(a[..., 3:], b[..., 3:])
    d = (hi - lo).astype(np.float32)
    dx, dy, dz = d[..., 0], d[..., 1], d[..., 2]
    return (dx * dy + dy * dz) + dz * dx


def test_two_pairs_then_root_by_hand():
    # gaps 0.1, 3, 0.1: (0,1) and (2,3) merge first, then the root
    order, left, right, parent, first, last = oracle.ploc(boxes_on_line([0, 1.1, 5, 6.1]))
    assert order.tolist() == [0, 1, 2, 3]
    assert left.tolist() == [1, -1, -3] and right.tolist() == [2, -2, -4]
    assert parent.tolist() == [-1, 0, 0, 1, 1, 2, 2]
    assert first.tolist() == [0, 0, 2] and last.tolist() == [3, 1, 3]


def test_equal_boxes_merge_by_the_lowest_index():
    # every union has the same area: each cluster's neighbour is the lowest other
    # index, only the first two are mutual, so the tree is a left-deep chain
    order, left, right, parent, first, last = oracle.ploc(boxes_on_line([0, 0, 0, 0]))
    assert order.tolist() == [0, 1, 2, 3]
    assert left.tolist() == [2, -1, 1] and right.tolist() == [-4, -2, -3]
    check_layout(order, left, right, parent, first, last, 4)


def test_radius_limits_the_neighbour_search():
    # positions 0 1 2 3 4 at x = 0, 10, 20, 30, 0.5: leaf 4 is nearest to leaf 0 but
    # four positions away.  With radius 4 they merge first; with radius 1 they cannot.
    b = boxes_on_line([0, 10, 20, 30, 0.5])
    o4, l4, r4, p4, f4, e4 = oracle.ploc(b, radius=4)
    o1, l1, r1, p1, f1, e1 = oracle.ploc(b, radius=1)
    def siblings(order, left, right, i, j):
        pos = {int(m): p for p, m in enumerate(order)}
        want = {-(pos[i] + 1), -(pos[j] + 1)}
        return any({int(a), int(c)} == want for a, c in zip(left, right))
    assert siblings(o4, l4, r4, 0, 4)
    assert not siblings(o1, l1, r1, 0, 4)
    check_layout(o4, l4, r4, p4, f4, e4, 5)
    check_layout(o1, l1, r1, p1, f1, e1, 5)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny(n):
    order, left, right, parent, first, last = oracle.ploc(boxes_on_line(np.arange(n) * 2.0))
    check_layout(order, left, right, parent, first, last, n)
    if n == 2:
        assert left.tolist() == [-1] and right.tolist() == [-2]


@pytest.mark.parametrize("radius", [1, 4, 16, 64])
def test_layout_invariants_random_boxes(radius):
    rng = np.random.default_rng(radius)
    c = rng.uniform(-1, 1, (1500, 3)).astype(np.float32)
    e = rng.uniform(0, 0.05, (1500, 3)).astype(np.float32)
    b = np.concatenate([c - e, c + e], 1).astype(np.float32)
    check_layout(*oracle.ploc(b, radius), 1500)


@pytest.mark.parametrize("radius", [4, 16, 10 ** 6])
def test_first_iteration_merges_are_brute_force_mutual_pairs(radius):
    """Leaves that are mutual nearest neighbours (least union area within the radius,
    ties to the lower index; brute force in float32) are siblings in the tree."""
    V, F = torus(30, 20)
    keys = oracle.morton(V, F)
    _, perm0 = oracle.sort_pairs(keys)
    lb = oracle.leaf_boxes(V, F, perm0)
    n = lb.shape[0]
    cost = union_area32(lb[:, None, :], lb[None, :, :])
    idx = np.arange(n)
    far = np.abs(idx[:, None] - idx[None, :]) > radius
    cost[far] = np.inf
    cost[idx, idx] = np.inf
    nn = np.argmin(cost, axis=1)                       # first (lowest) index of the minimum
    order, left, right, parent, first, last = oracle.ploc(lb, radius)
    check_layout(order, left, right, parent, first, last, n)
    pos = np.empty(n, int)
    pos[order] = np.arange(n)
    pairs = {frozenset((-(pos[i] + 1), -(pos[j] + 1))) for i, j in enumerate(nn) if nn[j] == i and i < j}
    assert len(pairs) > n // 8
    kids = {frozenset((int(a), int(b))) for a, b in zip(left, right)}
    assert pairs <= kids


def test_node_boxes_are_unions_and_the_tree_beats_the_lbvh():
    V, F = torus(40, 25)
    b = oracle.build_ploc(V, F)
    n = F.shape[0]
    check_layout(np.argsort(np.argsort(b["perm"])), b["left"], b["right"], b["parent"], b["first"],
                 b["last"], n)
    box = b["boxes"]
    for k in range(n - 1):                             # internal box = union of its children
        a, c = b["left"][k], b["right"][k]
        ba = box[a] if a >= 0 else box[n - 1 - a - 1]
        bc = box[c] if c >= 0 else box[n - 1 - c - 1]
        assert np.array_equal(box[k, :3], np.minimum(ba[:3], bc[:3]))
        assert np.array_equal(box[k, 3:], np.maximum(ba[3:], bc[3:]))

    def sah(boxes):
        d = boxes[: n - 1, 3:].astype(np.float64) - boxes[: n - 1, :3]
        return float(((d[:, 0] * d[:, 1] + d[:, 1] * d[:, 2] + d[:, 2] * d[:, 0])).sum())
    assert sah(box) < 0.95 * sah(oracle.build_lbvh(V, F)["boxes"])


def tree_depth(parent, n):
    """Internal nodes on the longest root-to-leaf path (the oracle's parent links:
    internal nodes first, then leaves; -1 at the root)."""
    best = 0
    for j in range(n):
        p, d = int(parent[(n - 1) + j]), 0
        while p >= 0:
            d += 1
            p = int(parent[p])
        best = max(best, d)
    return best


def test_equal_faces_give_a_chain_deeper_than_the_traversal_stack():
    # n copies of one triangle: every box is the same, so clustering builds a chain of
    # n - 1 internal nodes, far past the 64 levels a traversal keeps; the Karras tree
    # over the same (equal) keys splits on the index bits and stays shallow
    n = 300
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    F = np.tile(np.array([[0, 1, 2]], np.int32), (n, 1))
    t = oracle.build_ploc(V, F)
    assert tree_depth(t["parent"], n) == n - 1
    k = oracle.build_lbvh(V, F)
    assert tree_depth(k["parent"], n) == int(np.ceil(np.log2(n)))
