"""Seeded random draws on a triangle mesh (input generators only).

Uniform surface sampling in the usual two-step form: pick a face with
probability proportional to its area, then a point inside it with the
square-root warp of Osada et al. (2002), b = (1 - sqrt(r1), sqrt(r1)(1 - r2),
sqrt(r1) r2). Only the face ids and barycentric weights are random; they are
returned so that either side of a comparison can place the samples on its own
vertex buffer. `points_from` places them in float64 on the host for static
inputs (e.g. samples of a target mesh that never moves).
"""
from __future__ import annotations

import numpy as np


def face_areas(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    V = V.astype(np.float64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def osada_barycentrics(rng: np.random.Generator, n: int) -> np.ndarray:
    r1 = rng.random(n)
    r2 = rng.random(n)
    s = np.sqrt(r1)
    return np.stack([1.0 - s, s * (1.0 - r2), s * r2], 1)


def sample_surface(V: np.ndarray, F: np.ndarray, n: int, seed: int):
    """Return (face_ids int32 [n], bary float32 [n,3]) for n area-uniform samples."""
    rng = np.random.default_rng(seed)
    area = face_areas(V, F)
    cdf = np.cumsum(area)
    cdf /= cdf[-1]
    face = np.searchsorted(cdf, rng.random(n), side="right")
    face = np.minimum(face, F.shape[0] - 1).astype(np.int32)
    bary = osada_barycentrics(rng, n).astype(np.float32)
    return face, bary


def points_from(V: np.ndarray, F: np.ndarray, face: np.ndarray, bary: np.ndarray) -> np.ndarray:
    V = V.astype(np.float64)
    b = bary.astype(np.float64)
    tri = V[F[face]]                                   # [n, 3, 3]
    p = (b[:, :, None] * tri).sum(1)
    return np.ascontiguousarray(p, dtype=np.float32)


def uniform_box(n: int, lo, hi, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    p = lo + (hi - lo) * rng.random((n, 3))
    return np.ascontiguousarray(p, dtype=np.float32)
