"""Pins of the oracle's signed distance (inside negative, angle-weighted
pseudo-normals) for contact: the exact signed distance of a cube, the sign on
spheres and the torus, and the pseudo-normal cases at vertices and edges."""
import numpy as np

import oracle
from workloads.meshes import icosphere, torus


def cube():
    """[-1, 1]^3 as 12 counter-clockwise (outward) triangles."""
    V = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float64)
    idx = lambda x, y, z: ((x > 0) * 4 + (y > 0) * 2 + (z > 0))
    F = []
    for axis in range(3):
        for s in (-1, 1):
            corners = []
            for a in (-1, 1):
                for b in (-1, 1):
                    p = [0, 0, 0]
                    p[axis] = s
                    p[(axis + 1) % 3] = a
                    p[(axis + 2) % 3] = b
                    corners.append(idx(*p))
            c00, c01, c10, c11 = corners
            quad = [c00, c10, c11, c01] if s > 0 else [c00, c01, c11, c10]
            F += [[quad[0], quad[1], quad[2]], [quad[0], quad[2], quad[3]]]
    return V, np.array(F, np.int32)


def box_sdf(P):
    q = np.abs(P) - 1.0
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=1)
    inside = np.minimum(q.max(1), 0.0)
    return outside + inside


def test_cube_signed_distance_is_exact():
    V, F = cube()
    # every face normal points away from the centre
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    assert (np.einsum("ij,ij->i", n, V[F].mean(1)) > 0).all()
    rng = np.random.default_rng(0)
    P = rng.uniform(-2.5, 2.5, (3000, 3))
    # points near the faces, edges and corners of the cube, inside and out
    P = np.concatenate([P, np.sign(rng.normal(size=(500, 3))) * rng.uniform(0.8, 1.2, (500, 3))])
    r = oracle.signed_distance(V, F, P)
    # the tie rule may keep a face up to 1e-6 (relative) farther than the nearest
    np.testing.assert_allclose(r["sd"], box_sdf(P), rtol=1.01e-6, atol=1e-12)


def test_sphere_and_torus_signs():
    V, F = icosphere(3)
    rng = np.random.default_rng(1)
    d = rng.normal(size=(1000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = np.concatenate([rng.uniform(0.0, 0.9, 500), rng.uniform(1.001, 3.0, 500)])
    P = d * rad[:, None]
    sd = oracle.signed_distance(V, F, P)["sd"]
    assert ((sd < 0) == (rad < 1)).all()
    # the vertices of the icosphere lie on the unit sphere: outside points are at least r - 1 away
    assert (np.abs(sd[rad > 1]) >= rad[rad > 1] - 1 - 1e-12).all()
    Vt, Ft = torus(40, 24)
    a = rng.uniform(0, 2 * np.pi, 800)
    b = rng.uniform(0, 2 * np.pi, 800)
    rr = rng.uniform(0.0, 0.6, 800)
    P = np.column_stack([(1.0 + rr * np.cos(b)) * np.cos(a), (1.0 + rr * np.cos(b)) * np.sin(a), rr * np.sin(b)])
    sd = oracle.signed_distance(Vt, Ft, P)["sd"]
    keep = np.abs(rr - 0.35) > 0.03                  # the polygonal tube deviates by < 0.03
    assert ((sd[keep] < 0) == (rr[keep] < 0.35)).all()


def test_vertex_and_edge_regions_use_pseudo_normals():
    """Just outside a cube corner and edge the nearest point is the corner / edge, where
    a single face normal can give the wrong sign; the pseudo-normal gives +."""
    V, F = cube()
    P = np.array([[1.01, 1.01, 1.01], [1.01, 1.01, 0.3], [-1.01, 0.2, -1.01], [0.999, 0.999, 0.999]])
    sd = oracle.signed_distance(V, F, P)["sd"]
    np.testing.assert_allclose(sd, box_sdf(P), atol=1e-12)
    assert (sd[:3] > 0).all() and sd[3] < 0
