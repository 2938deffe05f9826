"""Seeded varying-topology mesh sequence (input generator only).

Stands in for the DG-Mesh sequences of Sec. 4 (not available here): each
frame is a triangle mesh extracted by marching cubes from a seeded signed
distance field, so vertex count and connectivity change from frame to frame
(the "varying topology" of Sec. 3.1), and merging / splitting blobs change
its genus as in the paper's dynamic scenes.

SDF: polynomial smooth minimum (k = 0.1) of four spheres of radius
U[0.2, 0.4] whose centres follow seeded Lissajous curves
c_i(tau) = A_i * sin(w_i * tau + phi_i), A_i in [0.3, 0.55]^3,
w_i in {1, 2, 3}^3, tau = 2 pi frame / 120.

The marching-cubes case table is *derived* here from the cube's own
edge/face structure (no published table is used): for each of the 256 corner
sign patterns the crossing edges on every cube face are paired into segments
(on a face with four crossings each inside corner is cut off on its own, so
neighbouring cubes agree), the segments are chained into closed loops, each
loop is oriented so that its normal points from the inside (negative) corners
to the outside ones, and fanned into triangles.
"""
from __future__ import annotations

import functools

import numpy as np

CORNER = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], dtype=np.int64)


def _edges():
    ed = []
    for axis in range(3):
        for c0 in range(8):
            if not (c0 >> axis) & 1:
                ed.append((axis, c0, c0 | (1 << axis)))
    return ed


EDGES = _edges()                                       # 12 x (axis, lo corner, hi corner)
_EDGE_OF = {frozenset((e[1], e[2])): i for i, e in enumerate(EDGES)}


def _faces():
    """Each cube face as its 4 corners in cyclic order."""
    out = []
    for a in range(3):
        b, c = [x for x in range(3) if x != a]
        for s in range(2):
            cyc = []
            for (pb, pc) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                cyc.append((s << a) | (pb << b) | (pc << c))
            out.append(cyc)
    return out


FACES = _faces()


@functools.lru_cache(maxsize=1)
def case_table():
    """(tri[256, 8, 3] edge ids padded with -1, ntri[256])."""
    tri = -np.ones((256, 8, 3), dtype=np.int64)
    ntri = np.zeros(256, dtype=np.int64)
    mid = np.array([(CORNER[e[1]] + CORNER[e[2]]) / 2.0 for e in EDGES])
    for case in range(256):
        inside = [(case >> c) & 1 for c in range(8)]
        adj = {}
        for cyc in FACES:
            fe = [_EDGE_OF[frozenset((cyc[i], cyc[(i + 1) % 4]))] for i in range(4)]
            cross = [inside[cyc[i]] != inside[cyc[(i + 1) % 4]] for i in range(4)]
            segs = []
            if sum(cross) == 2:
                segs.append(tuple(fe[i] for i in range(4) if cross[i]))
            elif sum(cross) == 4:
                for i in range(4):                     # cut off each inside corner
                    if inside[cyc[i]]:
                        segs.append((fe[(i - 1) % 4], fe[i]))
            for s0, s1 in segs:
                adj.setdefault(s0, []).append(s1)
                adj.setdefault(s1, []).append(s0)
        seen = set()
        tris = []
        for start in sorted(adj):
            if start in seen:
                continue
            loop = [start]
            seen.add(start)
            prev, cur = None, start
            while True:
                nxt = [x for x in adj[cur] if x != prev]
                nxt = nxt[0] if nxt else adj[cur][0]
                if nxt == start:
                    break
                loop.append(nxt)
                seen.add(nxt)
                prev, cur = cur, nxt
            P = mid[loop]
            nrm = np.zeros(3)
            for i in range(len(loop)):
                p, q = P[i], P[(i + 1) % len(loop)]
                nrm += np.cross(p, q)
            outward = np.zeros(3)
            for e in loop:
                _, c0, c1 = EDGES[e]
                cin, cout = (c0, c1) if inside[c0] else (c1, c0)
                outward += CORNER[cout] - CORNER[cin]
            if np.dot(nrm, outward) < 0:
                loop = loop[::-1]
            for i in range(1, len(loop) - 1):
                tris.append((loop[0], loop[i], loop[i + 1]))
        ntri[case] = len(tris)
        for t, tr in enumerate(tris):
            tri[case, t] = tr
    return tri, ntri


def marching_cubes(f: np.ndarray, lo: float = -1.0, hi: float = 1.0):
    """Extract the f = 0 surface of samples f[i, j, k] on a regular grid over [lo, hi]^3.

    Vertices lie on grid edges (linear interpolation) and are shared between
    the cubes that meet at an edge, so the mesh is welded. Inside is f < 0.
    """
    N = f.shape[0]
    assert f.shape == (N, N, N)
    h = (hi - lo) / (N - 1)
    tri, ntri = case_table()
    inside = (f < 0).astype(np.int64)
    M = N - 1
    case = np.zeros((M, M, M), dtype=np.int64)
    for c in range(8):
        ox, oy, oz = CORNER[c]
        case |= inside[ox:ox + M, oy:oy + M, oz:oz + M] << c
    case = case.ravel()
    nt = ntri[case]
    cubes = np.nonzero(nt)[0]
    ci, cj, ck = np.unravel_index(cubes, (M, M, M))
    gid = []
    for t in range(tri.shape[1]):
        sel = nt[cubes] > t
        if not sel.any():
            break
        le = tri[case[cubes[sel]], t]                  # [m, 3] local edges
        ax = np.array([e[0] for e in EDGES])[le]
        c0 = np.array([e[1] for e in EDGES])[le]
        gi = ci[sel][:, None] + CORNER[c0, 0]
        gj = cj[sel][:, None] + CORNER[c0, 1]
        gk = ck[sel][:, None] + CORNER[c0, 2]
        gid.append(ax * N ** 3 + (gi * N + gj) * N + gk)
    gid = np.concatenate(gid, 0)
    uniq, inv = np.unique(gid.ravel(), return_inverse=True)
    F = inv.reshape(-1, 3).astype(np.int32)
    ax = uniq // N ** 3
    lin = uniq % N ** 3
    i0, j0, k0 = np.unravel_index(lin, (N, N, N))
    i1 = i0 + (ax == 0)
    j1 = j0 + (ax == 1)
    k1 = k0 + (ax == 2)
    f0 = f[i0, j0, k0].astype(np.float64)
    f1 = f[i1, j1, k1].astype(np.float64)
    t = f0 / (f0 - f1)
    p0 = lo + h * np.stack([i0, j0, k0], 1).astype(np.float64)
    p1 = lo + h * np.stack([i1, j1, k1], 1).astype(np.float64)
    V = p0 + t[:, None] * (p1 - p0)
    return np.ascontiguousarray(V, dtype=np.float32), np.ascontiguousarray(F, dtype=np.int32)


def smin(a: np.ndarray, b: np.ndarray, k: float) -> np.ndarray:
    h = np.maximum(k - np.abs(a - b), 0.0) / k
    return np.minimum(a, b) - h * h * k / 4.0


class BlobSequence:
    """The seeded four-sphere smooth-union SDF, evaluated per frame."""

    def __init__(self, seed: int, n_frames: int = 120, n_spheres: int = 4, k: float = 0.1):
        rng = np.random.default_rng(seed)
        self.n_frames = n_frames
        self.k = k
        self.radius = rng.uniform(0.2, 0.4, size=n_spheres)
        self.amp = rng.uniform(0.3, 0.55, size=(n_spheres, 3))
        self.omega = rng.integers(1, 4, size=(n_spheres, 3)).astype(np.float64)
        self.phase = rng.uniform(0.0, 2.0 * np.pi, size=(n_spheres, 3))

    def centres(self, tau: float) -> np.ndarray:
        return self.amp * np.sin(self.omega * tau + self.phase)

    def sdf(self, tau: float, N: int = 128) -> np.ndarray:
        x = np.linspace(-1.0, 1.0, N)
        X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
        d = None
        for c, r in zip(self.centres(tau), self.radius):
            di = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - r
            d = di if d is None else smin(d, di, self.k)
        return d

    def tau(self, frame: float) -> float:
        return 2.0 * np.pi * frame / self.n_frames

    def mesh(self, frame: float, N: int = 128):
        return marching_cubes(self.sdf(self.tau(frame), N))
