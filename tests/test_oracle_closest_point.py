"""Pins for the oracle's NearestSurface (Eq. 1 / Eq. 2, Sec. 3.3).

Each check is independent of the oracle's own Voronoi-region code:
hand-worked values, a different closest-point method (plane projection when it
falls inside, else the best of the three clamped edge projections), closed
forms on spheres, and the tie / cutoff rules on constructed cases.
"""
import os

import numpy as np
import pytest

import oracle
from workloads.meshes import icosphere, displaced_icosphere

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "unit_triangle_regions.txt")
A, B, C = np.zeros(3), np.array([1.0, 0, 0]), np.array([0, 1.0, 0])


def load_regions():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        t = line.split()
        rows.append((np.array(list(map(float, t[:3]))), t[3], float(t[4]),
                     np.array(list(map(float, t[5:8])))))
    return rows


@pytest.mark.parametrize("p,region,d2,bary", load_regions())
def test_unit_triangle_every_region(p, region, d2, bary):
    got_d2, got_b, got_p = oracle.point_triangle(p, A, B, C)
    assert got_d2 == pytest.approx(d2, abs=1e-14)
    np.testing.assert_allclose(got_b, bary, atol=1e-14)
    np.testing.assert_allclose(got_p, bary[0] * A + bary[1] * B + bary[2] * C, atol=1e-14)


def _seg(p, x, y):
    d = y - x
    L = d @ d
    t = 0.0 if L == 0 else np.clip((p - x) @ d / L, 0.0, 1.0)
    q = x + t * d
    return (p - q) @ (p - q), q


def projection_or_edges(p, a, b, c):
    """Independent closest point: in-plane least squares, else nearest edge point."""
    M = np.stack([b - a, c - a], 1)
    st, *_ = np.linalg.lstsq(M, p - a, rcond=None)
    s, t = st
    if s >= 0 and t >= 0 and s + t <= 1:
        q = a + M @ st
        return (p - q) @ (p - q), q
    return min((_seg(p, a, b), _seg(p, b, c), _seg(p, c, a)), key=lambda r: r[0])


def test_random_triangles_against_projection_or_edges():
    rng = np.random.default_rng(11)
    for _ in range(3000):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * rng.choice([0.1, 1.0, 5.0])
        d2, bary, q = oracle.point_triangle(p, a, b, c)
        r2, rq = projection_or_edges(p, a, b, c)
        assert d2 == pytest.approx(r2, rel=1e-9, abs=1e-12)
        np.testing.assert_allclose(q, rq, atol=1e-8)
        assert bary.sum() == pytest.approx(1.0, abs=1e-12)
        assert (bary >= -1e-12).all()
        np.testing.assert_allclose(bary @ np.stack([a, b, c]), q, atol=1e-12)


def test_face_region_residual_is_normal():
    rng = np.random.default_rng(12)
    for _ in range(500):
        a, b, c = rng.normal(size=(3, 3))
        bary = rng.dirichlet([2, 2, 2])
        n = np.cross(b - a, c - a)
        n /= np.linalg.norm(n)
        h = rng.normal()
        p = bary @ np.stack([a, b, c]) + h * n
        d2, got_b, q = oracle.point_triangle(p, a, b, c)
        assert d2 == pytest.approx(h * h, rel=1e-9)
        np.testing.assert_allclose(got_b, bary, atol=1e-9)
        assert abs((p - q) @ (b - a)) < 1e-9 and abs((p - q) @ (c - a)) < 1e-9


def test_degenerate_triangles_reduce_to_segments():
    rng = np.random.default_rng(13)
    for _ in range(300):
        a, u = rng.normal(size=(2, 3))
        p = rng.normal(size=3) * 2
        # coincident vertices: the triangle is the segment a-c
        d2, bary, q = oracle.point_triangle(p, a, a, a + u)
        r2, rq = _seg(p, a, a + u)
        assert d2 == pytest.approx(r2, rel=1e-12, abs=1e-14)
        np.testing.assert_allclose(q, rq, atol=1e-12)
        # all three equal: a point
        d2, bary, q = oracle.point_triangle(p, a, a, a)
        assert d2 == pytest.approx((p - a) @ (p - a), rel=1e-14)
        assert bary.sum() == pytest.approx(1.0)


def test_icosphere_origin_is_nearest_face_plane():
    """Vertices on the unit sphere: the origin's foot on each face plane is the circumcentre,
    inside these acute faces, so d(0, mesh) = min_f |n_f . v0_f| and the point is n (n . v0)."""
    for s in (1, 2, 3):
        V, F = icosphere(s)
        V64 = V.astype(np.float64)
        a, b, c = V64[F[:, 0]], V64[F[:, 1]], V64[F[:, 2]]
        n = np.cross(b - a, c - a)
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        h = np.abs(np.einsum("ij,ij->i", n, a))
        out = oracle.closest_point(V, F, np.zeros((1, 3)))
        f = out["face"][0]
        # symmetric faces tie up to float32 vertex rounding: the lowest id within the
        # 1e-6 relative window is reported, at its own plane distance
        assert h.min() <= np.sqrt(out["d2"][0]) <= h.min() * (1 + 1e-6)
        assert out["d2"][0] == pytest.approx(h[f] ** 2, rel=1e-12)
        assert f == np.nonzero(h <= h.min() * (1 + 1e-6) + 1e-9)[0].min()
        np.testing.assert_allclose(out["point"][0], n[f] * (n[f] @ a[f]), atol=1e-12)
        # circumcentre: equidistant from the three vertices
        q = out["point"][0]
        r = np.linalg.norm(np.stack([a[f], b[f], c[f]]) - q, axis=1)
        np.testing.assert_allclose(r, r[0], rtol=1e-9)


def test_far_queries_on_a_sphere_are_bounded():
    V, F = icosphere(3)
    rng = np.random.default_rng(14)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    P = 5.0 * d
    out = oracle.closest_point(V, F, P)
    dist = np.sqrt(out["d2"])
    nearest_vertex = np.sqrt(((P[:, None, :] - V[None].astype(np.float64)) ** 2).sum(-1)).min(1)
    assert (dist >= 4.0 - 1e-12).all()
    assert (dist <= nearest_vertex + 1e-12).all()


def test_mesh_distance_bounded_by_dense_surface_samples():
    V, F = displaced_icosphere(1, 0.1, 0.3)
    rng = np.random.default_rng(15)
    Q = rng.uniform(-1.5, 1.5, size=(40, 3))
    out = oracle.closest_point(V, F, Q)
    # every surface sample is at least as far as the reported closest point
    bb = rng.dirichlet([1, 1, 1], size=400)
    S = np.einsum("sk,fkc->fsc", bb, V.astype(np.float64)[F]).reshape(-1, 3)
    dmin = np.sqrt(((Q[:, None, :] - S[None]) ** 2).sum(-1)).min(1)
    assert (np.sqrt(out["d2"]) <= dmin + 1e-12).all()
    assert (np.sqrt(out["d2"]) >= dmin - 0.05).all()


def test_tie_picks_lowest_face_id_in_either_order():
    # Two triangles mirrored in the plane x = 0; the query lies on that plane.
    V = np.array([[1, 0, 0], [2, 1, 0], [2, -1, 0], [-1, 0, 0], [-2, -1, 0], [-2, 1, 0]],
                 np.float32)
    F = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    Q = np.array([[0, 0, 0.3], [0, 0.2, -0.1]], np.float32)
    out = oracle.closest_point(V, F, Q)
    assert (out["face"] == 0).all()
    out2 = oracle.closest_point(V, F[::-1].copy(), Q)
    assert (out2["face"] == 0).all()
    # the same point is reported from either mirrored triangle
    np.testing.assert_allclose(out2["point"][:, 0], -out["point"][:, 0], atol=1e-15)


def test_tie_window_is_relative_distance_1e6():
    # Two parallel triangles at distances 1 and 1 + delta; the far one has the lower id.
    def mesh(delta):
        V = np.array([[-1, -1, 1 + delta], [1, -1, 1 + delta], [0, 1, 1 + delta],
                      [-1, -1, -1], [1, -1, -1], [0, 1, -1]], np.float64)
        return V, np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    V, F = mesh(0.5e-6)
    assert oracle.closest_point(V, F, np.zeros((1, 3)))["face"][0] == 0
    V, F = mesh(2e-6)
    assert oracle.closest_point(V, F, np.zeros((1, 3)))["face"][0] == 1


def test_cutoff_returns_no_face():
    V, F = icosphere(2)
    Q = np.array([[0, 0, 0], [0, 0, 1.04], [0, 0, 3.0]], np.float32)
    full = oracle.closest_point(V, F, Q)
    cut = oracle.closest_point(V, F, Q, max_dist=0.05)
    d = np.sqrt(full["d2"])
    for i in range(3):
        if d[i] <= 0.05:
            assert cut["face"][i] == full["face"][i]
        else:
            assert cut["face"][i] == -1 and np.isinf(cut["d2"][i])
    assert cut["face"][1] >= 0 and cut["face"][0] == -1 and cut["face"][2] == -1


def test_empty_mesh_and_empty_queries():
    V = np.zeros((0, 3), np.float32)
    F = np.zeros((0, 3), np.int32)
    out = oracle.closest_point(V, F, np.ones((2, 3), np.float32))
    assert (out["face"] == -1).all() and np.isinf(out["d2"]).all()
    V, F = icosphere(1)
    out = oracle.closest_point(V, F, np.zeros((0, 3), np.float32))
    assert out["face"].shape == (0,)
