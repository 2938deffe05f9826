"""Pins for the oracle's face-bound Gaussian update (Sec. 3.2 dual representation;
binding of Gaussians to faces per Sec. 2 / Sec. 3.1, formula is our reading).

Checked against: orthonormality and handedness of the frame, the frame's axes
computed directly from the face, an independent quaternion-to-matrix formula,
a right triangle worked by hand, rigid-motion and uniform-scale equivariance,
and the degenerate-face rule.
"""
import numpy as np
import pytest

import oracle
from workloads.meshes import displaced_icosphere
from workloads.sampling import osada_barycentrics


def quat_to_matrix(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def random_setup(seed, G=400):
    V, F = displaced_icosphere(2, 0.1, 0.7)
    rng = np.random.default_rng(seed)
    gface = rng.integers(0, F.shape[0], size=G).astype(np.int32)
    gbary = osada_barycentrics(rng, G)
    goff = rng.normal(scale=0.01, size=G)
    return V.astype(np.float64), F, gface, gbary, goff


def test_frame_is_the_face_frame():
    V, F, gface, gbary, goff = random_setup(1)
    out = oracle.bind_gaussians(V, F, gface, gbary, goff)
    a, b, c = V[F[gface, 0]], V[F[gface, 1]], V[F[gface, 2]]
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    e1 = (b - a) / np.linalg.norm(b - a, axis=1, keepdims=True)
    for g in range(gface.shape[0]):
        q = out["quat"][g]
        assert np.linalg.norm(q) == pytest.approx(1.0, abs=1e-12)
        assert q[0] >= 0
        R = quat_to_matrix(q)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
        np.testing.assert_allclose(R[:, 2], n[g], atol=1e-12)
        np.testing.assert_allclose(R[:, 0], e1[g], atol=1e-12)
    mu_ref = (gbary[:, :, None] * np.stack([a, b, c], 1)).sum(1) + goff[:, None] * n
    np.testing.assert_allclose(out["mu"], mu_ref, atol=1e-12)


def test_right_triangle_by_hand():
    V = np.array([[0, 0, 0], [2, 0, 0], [0, 3, 0]], np.float64)
    F = np.array([[0, 1, 2]], np.int32)
    out = oracle.bind_gaussians(V, F, np.zeros(1, np.int32), np.full((1, 3), 1.0 / 3.0))
    np.testing.assert_allclose(out["mu"][0], [2.0 / 3.0, 1.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(out["quat"][0], [1, 0, 0, 0], atol=1e-15)
    # l = 2, h = 2 * area / l = 3
    np.testing.assert_allclose(out["scale"][0], [2.0 / 3.0, 1.0, 0.01 * 5.0 / 6.0], rtol=1e-14)
    # the same face turned a half turn about x: n = -z, e2 = -y -> q = (0, 1, 0, 0)
    V2 = V * np.array([1, -1, -1])
    out = oracle.bind_gaussians(V2, F, np.zeros(1, np.int32), np.full((1, 3), 1.0 / 3.0))
    np.testing.assert_allclose(out["quat"][0], [0, 1, 0, 0], atol=1e-15)


def random_rotation(rng):
    from scipy.spatial.transform import Rotation
    return Rotation.random(random_state=rng).as_matrix()


def test_rigid_motion_equivariance():
    V, F, gface, gbary, goff = random_setup(2)
    rng = np.random.default_rng(3)
    Qm, t = random_rotation(rng), rng.normal(size=3)
    o1 = oracle.bind_gaussians(V, F, gface, gbary, goff)
    o2 = oracle.bind_gaussians(V @ Qm.T + t, F, gface, gbary, goff)
    np.testing.assert_allclose(o2["mu"], o1["mu"] @ Qm.T + t, atol=1e-12)
    np.testing.assert_allclose(o2["scale"], o1["scale"], rtol=1e-12)
    for g in range(gface.shape[0]):
        np.testing.assert_allclose(quat_to_matrix(o2["quat"][g]),
                                   Qm @ quat_to_matrix(o1["quat"][g]), atol=1e-12)


def test_uniform_scale():
    V, F, gface, gbary, goff = random_setup(4)
    o1 = oracle.bind_gaussians(V, F, gface, gbary)
    o2 = oracle.bind_gaussians(2.5 * V, F, gface, gbary)
    np.testing.assert_allclose(o2["scale"], 2.5 * o1["scale"], rtol=1e-12)
    np.testing.assert_allclose(o2["mu"], 2.5 * o1["mu"], rtol=1e-12)
    np.testing.assert_allclose(o2["quat"], o1["quat"], atol=1e-12)


def test_centroid_anchor_and_degenerate_faces():
    V, F = displaced_icosphere(1, 0.1, 0.1)
    G = F.shape[0]
    out = oracle.bind_gaussians(V, F, np.arange(G, dtype=np.int32), np.full((G, 3), 1 / 3.0))
    np.testing.assert_allclose(out["mu"], V.astype(np.float64)[F].mean(1), atol=1e-12)
    assert out["n_degenerate"] == 0
    Vd = np.array([[0, 0, 0], [0, 0, 0], [1, 1, 1], [1, 2, 3]], np.float64)
    Fd = np.array([[0, 1, 2], [2, 3, 3], [2, 2, 2]], np.int32)
    out = oracle.bind_gaussians(Vd, Fd, np.arange(3, dtype=np.int32), np.full((3, 3), 1 / 3.0),
                                np.ones(3))
    assert out["n_degenerate"] == 3 and (out["flags"] == 1).all()
    np.testing.assert_allclose(out["quat"], np.tile([1.0, 0, 0, 0], (3, 1)))
    np.testing.assert_array_equal(out["scale"], 0)
    np.testing.assert_allclose(out["mu"], Vd[Fd].mean(1), atol=1e-15)


def test_every_shepperd_branch_round_trips():
    """Faces whose frames put the largest pivot on w, x, y and z in turn."""
    rng = np.random.default_rng(6)
    seen = set()
    for _ in range(400):
        Rm = random_rotation(rng)
        V = np.stack([np.zeros(3), Rm[:, 0] * 1.7, Rm[:, 0] * 0.4 + Rm[:, 1] * 1.1])
        out = oracle.bind_gaussians(V, np.array([[0, 1, 2]], np.int32), np.zeros(1, np.int32),
                                    np.full((1, 3), 1 / 3.0))
        q = out["quat"][0]
        np.testing.assert_allclose(quat_to_matrix(q), Rm, atol=1e-12)
        tr = np.trace(Rm)
        seen.add(int(np.argmax([tr, Rm[0, 0], Rm[1, 1], Rm[2, 2]])))
    assert seen == {0, 1, 2, 3}
