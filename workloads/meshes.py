"""Seeded synthetic meshes and deformations (input generators only).

Nothing here is part of the dynamic-mesh update itself: these functions
produce the vertex / index buffers that stand in for the paper's
reconstructed mesh sequences (the DG-Mesh scenes of Sec. 4 are not
available), shaped like the workloads the paper describes (N_v of 1e3-1e5,
smooth deformations without topological events, Sec. 5).

All positions are returned as float32 (V, 3) C-contiguous arrays and all
faces as int32 (F, 3), counter-clockwise seen from outside.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import ConvexHull

GOLDEN = (1.0 + 5.0 ** 0.5) / 2.0


def _orient_outward(V: np.ndarray, F: np.ndarray, centre: np.ndarray) -> np.ndarray:
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, (a + b + c) / 3.0 - centre) < 0
    F = F.copy()
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return F


def icosahedron() -> tuple[np.ndarray, np.ndarray]:
    """12 unit vectors (cyclic permutations of (0, +-1, +-phi)); faces from their hull."""
    pts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            pts.append((0.0, s1, s2 * GOLDEN))
            pts.append((s1, s2 * GOLDEN, 0.0))
            pts.append((s2 * GOLDEN, 0.0, s1))
    V = np.array(pts, dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = ConvexHull(V).simplices.astype(np.int64)
    F = _orient_outward(V, F, np.zeros(3))
    return V, F


def icosphere(subdiv: int, radius: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Loop-style 1->4 subdivision of the icosahedron, re-projected to the sphere.

    subdiv s gives V = 10*4^s + 2 and F = 20*4^s (s=3: 642/1280, s=4: 2562/5120,
    s=5: 10242/20480, s=6: 40962/81920).
    """
    V, F = icosahedron()
    for _ in range(subdiv):
        nV = V.shape[0]
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
        e = np.sort(e, axis=1)
        uniq, inv = np.unique(e[:, 0] * nV + e[:, 1], return_inverse=True)
        ua, ub = uniq // nV, uniq % nV
        mid = V[ua] + V[ub]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        m = inv.reshape(3, -1).T + nV          # midpoint ids of edges (01, 12, 20)
        m01, m12, m20 = m[:, 0], m[:, 1], m[:, 2]
        a, b, c = F[:, 0], F[:, 1], F[:, 2]
        F = np.concatenate([
            np.stack([a, m01, m20], 1),
            np.stack([b, m12, m01], 1),
            np.stack([c, m20, m12], 1),
            np.stack([m01, m12, m20], 1),
        ], axis=0)
        V = np.concatenate([V, mid], axis=0)
    V = V * radius
    return np.ascontiguousarray(V, dtype=np.float32), np.ascontiguousarray(F, dtype=np.int32)


def torus(nu: int, nv: int, R: float = 1.0, r: float = 0.35) -> tuple[np.ndarray, np.ndarray]:
    """Grid torus: V = nu*nv, F = 2*nu*nv; u runs around the ring, v around the tube."""
    u = 2.0 * np.pi * np.arange(nu) / nu
    v = 2.0 * np.pi * np.arange(nv) / nv
    uu, vv = np.meshgrid(u, v, indexing="ij")
    x = (R + r * np.cos(vv)) * np.cos(uu)
    y = (R + r * np.cos(vv)) * np.sin(uu)
    z = r * np.sin(vv)
    V = np.stack([x, y, z], -1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    i1, j1 = (i + 1) % nu, (j + 1) % nv
    idx = lambda a, b: (a * nv + b).ravel()
    q00, q10, q11, q01 = idx(i, j), idx(i1, j), idx(i1, j1), idx(i, j1)
    F = np.concatenate([np.stack([q00, q10, q11], 1), np.stack([q00, q11, q01], 1)], 0)
    # Orient against the local tube centre (the ring circle), not the origin.
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    cen = (a + b + c) / 3.0
    ang = np.arctan2(cen[:, 1], cen[:, 0])
    ring = np.stack([R * np.cos(ang), R * np.sin(ang), np.zeros_like(ang)], 1)
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, cen - ring) < 0
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return np.ascontiguousarray(V, dtype=np.float32), np.ascontiguousarray(F, dtype=np.int32)


def spherical_angles(V: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """theta = azimuth in the xy plane, phi = polar angle from +z."""
    V = V.astype(np.float64)
    theta = np.arctan2(V[:, 1], V[:, 0])
    phi = np.arccos(np.clip(V[:, 2] / np.linalg.norm(V, axis=1), -1.0, 1.0))
    return theta, phi


def displaced_icosphere(subdiv: int, amp: float, phi0: float,
                        k_theta: int = 3, k_phi: int = 2) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere with radius 1 + amp*sin(k_theta*theta + phi0)*cos(k_phi*phi)."""
    V, F = icosphere(subdiv)
    theta, phi = spherical_angles(V)
    r = 1.0 + amp * np.sin(k_theta * theta + phi0) * np.cos(k_phi * phi)
    V = V.astype(np.float64) * r[:, None]
    return np.ascontiguousarray(V, dtype=np.float32), F


def displaced_torus(nu: int, nv: int, amp: float, ku: int, kv: int, ph: float,
                    R: float = 1.0, r: float = 0.35) -> tuple[np.ndarray, np.ndarray]:
    """Torus whose tube radius is r*(1 + amp*sin(ku*u + ph)*cos(kv*v))."""
    V, F = torus(nu, nv, R, r)
    u = np.repeat(2.0 * np.pi * np.arange(nu) / nu, nv)
    v = np.tile(2.0 * np.pi * np.arange(nv) / nv, nu)
    rr = r * (1.0 + amp * np.sin(ku * u + ph) * np.cos(kv * v))
    x = (R + rr * np.cos(v)) * np.cos(u)
    y = (R + rr * np.cos(v)) * np.sin(u)
    z = rr * np.sin(v)
    V = np.stack([x, y, z], -1)
    return np.ascontiguousarray(V, dtype=np.float32), F


def _axis_angle_matrix(axis: np.ndarray, angle: float) -> np.ndarray:
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)


class TorusSkinning:
    """4-bone linear-blend skinning of a ring-shaped mesh (the deforming physics mesh).

    Bones sit on the ring at angles 0, 90, 180, 270 degrees. Vertex weights are
    w_b ~ exp(-kappa * dangle_b^2) normalised, with dangle the wrapped ring-angle
    difference and kappa seeded in [2, 6]. Bone b rotates about a seeded unit axis
    through its pivot by 30deg * sin(2*pi*t/period + phase_b), so |angle| <= 30deg.
    """

    def __init__(self, V_rest: np.ndarray, seed: int, R: float = 1.0, period: int = 125):
        rng = np.random.default_rng(seed)
        self.V = V_rest.astype(np.float64)
        self.period = period
        self.kappa = rng.uniform(2.0, 6.0)
        self.bone_angle = np.deg2rad([0.0, 90.0, 180.0, 270.0])
        self.pivot = np.stack([R * np.cos(self.bone_angle), R * np.sin(self.bone_angle),
                               np.zeros(4)], 1)
        ax = rng.normal(size=(4, 3))
        self.axis = ax / np.linalg.norm(ax, axis=1, keepdims=True)
        self.phase = rng.uniform(0.0, 2.0 * np.pi, size=4)
        ang = np.arctan2(self.V[:, 1], self.V[:, 0])
        d = ang[:, None] - self.bone_angle[None, :]
        d = (d + np.pi) % (2.0 * np.pi) - np.pi
        w = np.exp(-self.kappa * d * d)
        self.w = w / w.sum(1, keepdims=True)

    def frame(self, t: int) -> np.ndarray:
        out = np.zeros_like(self.V)
        for b in range(4):
            ang = np.deg2rad(30.0) * np.sin(2.0 * np.pi * t / self.period + self.phase[b])
            M = _axis_angle_matrix(self.axis[b], ang)
            out += self.w[:, b:b + 1] * ((self.V - self.pivot[b]) @ M.T + self.pivot[b])
        return np.ascontiguousarray(out, dtype=np.float32)


def bbox(V: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    return V.min(0).astype(np.float64), V.max(0).astype(np.float64)


def batch_scenes(n_scenes: int = 64, seed: int = 4000, fmin: int = 1000, fmax: int = 200000):
    """Independent scenes with log-uniform face counts in [fmin, fmax]: even scenes are
    grid tori with 2*nu*nv ~ F (nu/nv ~ 1.6), odd scenes icospheres at the subdivision
    level nearest F; every scene gets a seeded sinusoidal radial displacement of
    amplitude 0.05-0.15.  Returns a list of (V, F)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scenes):
        F_target = int(round(np.exp(rng.uniform(np.log(fmin), np.log(fmax)))))
        amp = rng.uniform(0.05, 0.15)
        k1, k2 = int(rng.integers(2, 6)), int(rng.integers(1, 4))
        ph = rng.uniform(0, 2 * np.pi)
        if i % 2 == 0:
            nv = max(3, int(round(np.sqrt(F_target / (2 * 1.6)))))
            nu = max(3, int(round(1.6 * nv)))
            out.append(displaced_torus(nu, nv, amp, k1, k2, ph))
        else:
            s = int(np.clip(np.round(np.log(F_target / 20.0) / np.log(4.0)), 0, 7))
            out.append(displaced_icosphere(s, amp, ph, k_theta=k1, k_phi=k2))
    return out
