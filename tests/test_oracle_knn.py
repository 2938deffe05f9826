"""Pins of the oracle's k-NN weighted surface projection (the NearestSurface of
temporal tracking, Sec. 3.3 Strategy 1, Eq. 1): closed forms that fix the
selection of the k nearest faces, the inverse-distance weights and the anchor
blend."""
import numpy as np
import pytest

import oracle
from workloads.meshes import icosphere


def two_planes():
    """Two large parallel triangles, z = +1 (face 0) and z = -1 (face 1)."""
    V = np.array([[-10, -10, 1], [10, -10, 1], [0, 10, 1],
                  [-10, -10, -1], [0, 10, -1], [10, -10, -1]], np.float64)
    F = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    return V, F


def test_between_two_parallel_planes_returns_the_query():
    """Inverse-distance weights between planes z = 1 and z = -1 give
    z' = (1/(1-z) - 1/(1+z)) / (1/(1-z) + 1/(1+z)) = z: the projection is the identity."""
    V, F = two_planes()
    rng = np.random.default_rng(0)
    Q = np.column_stack([rng.uniform(-1, 1, 50), rng.uniform(-1, 1, 50), rng.uniform(-0.9, 0.9, 50)])
    r = oracle.knn_project(V, F, Q, k=2)
    np.testing.assert_allclose(r["point"], Q, atol=1e-12)
    assert (np.sort(r["face"], 1) == [0, 1]).all()
    # k = 1 keeps the nearer plane only
    r1 = oracle.knn_project(V, F, Q, k=1)
    expect = Q.copy()
    expect[:, 2] = np.where(Q[:, 2] >= 0, 1.0, -1.0)
    np.testing.assert_allclose(r1["point"], expect, atol=1e-12)
    np.testing.assert_allclose(r1["d2"][:, 0], (1 - np.abs(Q[:, 2])) ** 2, atol=1e-12)


def test_unit_triangle_hand_values():
    """One face: every k gives its closest point; unused slots are face -1."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float64)
    F = np.array([[0, 1, 2]], np.int32)
    Q = np.array([[-1, -1, 0.5], [1, 1, 0], [0.25, 0.25, 2.0]])
    for k in (1, 3):
        r = oracle.knn_project(V, F, Q, k=k)
        np.testing.assert_allclose(r["point"], [[0, 0, 0], [0.5, 0.5, 0], [0.25, 0.25, 0]], atol=1e-12)
        np.testing.assert_allclose(r["d2"][:, 0], [2.25, 0.5, 4.0], atol=1e-12)
        assert (r["face"][:, 1:] == -1).all()


def test_query_on_a_flat_grid_stays_put():
    """A query on a planar triangulated grid is at distance 0 from its face; the weight
    floor (1e-6 of the diagonal) makes the result the query up to that scale."""
    n = 8
    xs = np.linspace(0, 1, n + 1)
    V = np.array([[x, y, 0.0] for y in xs for x in xs])
    F = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = j * (n + 1) + i, j * (n + 1) + i + 1, (j + 1) * (n + 1) + i, (j + 1) * (n + 1) + i + 1
            F += [[a, b, d], [a, d, c]]
    F = np.array(F, np.int32)
    rng = np.random.default_rng(1)
    Q = np.column_stack([rng.uniform(0.1, 0.9, 40), rng.uniform(0.1, 0.9, 40), np.zeros(40)])
    r = oracle.knn_project(V, F, Q, k=4)
    diag = np.sqrt(2.0)
    assert np.abs(r["point"] - Q).max() < 1e-4 * diag
    assert (r["d2"][:, 0] < 1e-24).all()


def test_shared_vertex_picks_lowest_ids_and_returns_the_vertex():
    """Far out along a vertex direction every face around that vertex is at the same
    distance; the k kept are the lowest ids and the blend is the vertex itself."""
    V, F = icosphere(2)
    for vid in (0, 5, 11):
        q = 3.0 * V[vid]
        around = np.flatnonzero((F == vid).any(1))
        r = oracle.knn_project(V, F, q[None], k=4)
        np.testing.assert_allclose(r["point"][0], V[vid], atol=1e-12)
        assert list(r["face"][0]) == sorted(around)[:4]


def test_anchor_blend_and_permutation_invariance():
    V, F = icosphere(2)
    rng = np.random.default_rng(2)
    Q = rng.normal(size=(30, 3)) * 1.3
    anchor = rng.normal(size=(30, 3))
    base = oracle.knn_project(V, F, Q, k=4)
    np.testing.assert_allclose(oracle.knn_project(V, F, Q, k=4, anchor=anchor, anchor_w=1.0)["point"],
                               anchor, atol=1e-12)
    mix = oracle.knn_project(V, F, Q, k=4, anchor=anchor, anchor_w=0.2)["point"]
    np.testing.assert_allclose(mix, 0.8 * base["point"] + 0.2 * anchor, atol=1e-12)
    # reordering the faces changes ids, not the (tie-free) blend
    perm = rng.permutation(F.shape[0])
    r = oracle.knn_project(V, F[perm], Q, k=4)
    gap = np.sqrt(base["d2"][:, 3]) < np.sqrt(np.sort(oracle.closest_point(V, F, Q, all_d2=True)["d2_all"], 1)[:, 4]) * (1 - 1e-9)
    np.testing.assert_allclose(r["point"][gap], base["point"][gap], atol=1e-12)
    np.testing.assert_array_equal(np.sort(perm[r["face"][gap]], 1), np.sort(base["face"][gap], 1))
