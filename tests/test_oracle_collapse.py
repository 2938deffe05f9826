"""Pins for the oracle's leaf collapse (orc_collapse): a subtree whose range holds at
most L faces becomes one leaf over that range (the scope's reading of a leaf size L;
the paper fixes no tree at all).  Pinned by: L = 1 leaves every link as built;
hand-worked links on the 4-key Karras tree at L = 2 and L = 4; and, on random trees of
both kinds, that a search from the root meets every face exactly once, each range
leaf holds at most L faces, and no reachable internal node holds L or fewer (the
collapse is maximal)."""
import numpy as np
import pytest

import oracle
from workloads.meshes import displaced_icosphere, torus


def reach(link, n):
    """Faces met from the root following the collapsed links, and the reachable
    internal nodes."""
    faces, internal = [], []
    stack = [0]
    while stack:
        i = stack.pop()
        internal.append(i)
        for side in (0, 2):
            c, cnt = int(link[i, side]), int(link[i, side + 1])
            if c < 0:
                first = -c - 1
                faces.extend(range(first, first + cnt))
            else:
                assert cnt == c
                stack.append(c)
    return sorted(faces), internal


def test_leaf_size_one_keeps_the_links():
    keys = np.sort(np.random.default_rng(1).integers(0, 1 << 30, 300).astype(np.uint32))
    left, right, parent, first, last = oracle.karras(keys)
    link = oracle.collapse(left, right, first, last, 1)
    np.testing.assert_array_equal(link[:, 0], left)
    np.testing.assert_array_equal(link[:, 2], right)
    assert (link[:, 1][left < 0] == 1).all() and (link[:, 3][right < 0] == 1).all()
    assert (link[:, 1][left >= 0] == left[left >= 0]).all()


def test_hand_worked_four_key_tree():
    # keys 1, 2, 4, 5: root 0 = [0,3] with children node 1 = [0,1] and node 2 = [2,3]
    left, right, parent, first, last = oracle.karras(np.array([1, 2, 4, 5], np.uint32))
    l2 = oracle.collapse(left, right, first, last, 2)
    # L = 2: both children of the root hold two faces: ranges [0,1] and [2,3]
    np.testing.assert_array_equal(l2[0], [-1, 2, -3, 2])
    # nodes 1 and 2 keep their own single leaves (unreachable now, written all the same)
    np.testing.assert_array_equal(l2[1], [-1, 1, -2, 1])
    np.testing.assert_array_equal(l2[2], [-3, 1, -4, 1])
    l4 = oracle.collapse(left, right, first, last, 4)
    np.testing.assert_array_equal(l4[0], [-1, 2, -3, 2])   # the root itself is never a leaf
    l1 = oracle.collapse(left, right, first, last, 1)
    np.testing.assert_array_equal(l1[0], [1, 1, 2, 2])


@pytest.mark.parametrize("L", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("kind", ["karras", "ploc"])
def test_every_face_once_and_maximal(L, kind):
    V, F = displaced_icosphere(3, 0.1, 0.4) if kind == "karras" else torus(30, 20)
    if kind == "karras":
        t = oracle.build_lbvh(V, F)
    else:
        t = oracle.build_ploc(V, F)
    n = F.shape[0]
    link = oracle.collapse(t["left"], t["right"], t["first"], t["last"], L)
    faces, internal = reach(link, n)
    assert faces == list(range(n))
    for i in internal:
        assert i == 0 or t["last"][i] - t["first"][i] + 1 > L
        for side in (0, 2):
            if link[i, side] < 0:
                assert 1 <= link[i, side + 1] <= L
