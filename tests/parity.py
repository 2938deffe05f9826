"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (float32 GPU against the float64 oracle):
  * Morton keys, sort permutation, tree topology, node boxes: bit-exact.
  * distance: |d_gpu - d_ref| <= 1e-5 * max(d_ref, 1e-3 * diag)  (relative, with a
    floor because projected points sit at distance ~0).
  * nearest face: equal, except where float32 rounding moves a face across the
    tie window: the GPU's and the oracle's faces then have float64 distances
    within the window's width plus twice the float32 bound
    8 * 2^-24 * (|q| + max|v|) of each other.  Those are counted separately and
    must stay a handful.
  * two GPU answers for the same queries and mesh (another tree, traversal
    variant, lane width, warm start or query order): identical, bit for bit.
  * gradients: per component, |g - g_ref| <= 1e-4 * max(|g_ref|, |row|,
    1e-3 * max |row|), |row| the norm of that vertex's / query's gradient.
  * barycentric weights: 1e-5 absolute on faces whose smallest altitude is at
    least 1e-2 of their longest edge (slivers compare the point instead).
  * Gaussian centre / rotation / scale: 1e-5 absolute.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

TIE_REL = 1e-6
TIE_ABS = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def well_conditioned(V, F, faces):
    tri = V.astype(np.float64)[F[faces]]
    e = np.stack([tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 1], tri[:, 0] - tri[:, 2]], 1)
    L = np.linalg.norm(e, axis=2)
    area2 = np.linalg.norm(np.cross(e[:, 0], -e[:, 2]), axis=1)
    lmax = L.max(1)
    return (area2 / np.maximum(lmax, 1e-30)) >= 1e-2 * lmax


def check_closest(V, F, Q, got, max_dist=np.inf, ref=None, max_tie_frac=2e-3):
    """Compare GPU NearestSurface outputs with the oracle; returns stats."""
    V = np.asarray(V, np.float32)
    Q = np.asarray(Q, np.float32)
    ref = oracle.closest_point(V, F, Q, max_dist) if ref is None else ref
    diag = oracle.mesh_diag(V, F)
    tau = TIE_ABS * diag
    fg = host(got["face"])
    fr = ref["face"]
    d2g = host(got["dist2"]).astype(np.float64)
    dr = np.sqrt(ref["d2"])
    vmax = np.abs(V).max() if V.size else 0.0
    eps32 = 8 * 2.0 ** -24 * (np.linalg.norm(Q, axis=1) + vmax) * 3    # hit/miss at the cutoff only
    # hit / miss agreement (a miss on one side only is allowed right at the cutoff)
    miss_g, miss_r = fg < 0, fr < 0
    odd = np.nonzero(miss_g != miss_r)[0]
    for i in odd:
        d_true = dr[i] if fr[i] >= 0 else np.sqrt(oracle.closest_point(V, F, Q[i:i + 1])["d2"][0])
        assert abs(d_true - max_dist) <= 1e-5 * max(max_dist, 1e-3 * diag) + eps32[i], \
            f"query {i}: hit/miss differs away from the cutoff (d={d_true}, cut={max_dist})"
    both = (~miss_g) & (~miss_r)
    assert np.all(np.isinf(d2g[miss_g])) and np.all(fg[miss_g] == -1)
    dg = np.sqrt(d2g[both])
    err = np.abs(dg - dr[both])
    lim = 1e-5 * np.maximum(dr[both], 1e-3 * diag)
    bad = np.nonzero(err > lim)[0]
    assert bad.size == 0, (f"{bad.size} distances off; worst rel "
                           f"{(err / np.maximum(dr[both], 1e-3 * diag)).max():.3g}")
    # nearest face: the oracle's, unless float32 rounding moved a face across the
    # window; then the two faces' float64 distances are within the window's width
    # plus the float32 bound of each of them
    idx = np.nonzero(both & (fg != fr))[0]
    eps = 8 * 2.0 ** -24 * (np.linalg.norm(Q.astype(np.float64), axis=1) + vmax)
    ties = 0
    for i in idx:
        a, b, c = (V[F[fg[i]]][k].astype(np.float64) for k in range(3))
        d2_alt, _, _ = oracle.point_triangle(Q[i].astype(np.float64), a, b, c)
        width = dr[i] * TIE_REL + tau
        gap = abs(np.sqrt(d2_alt) - dr[i])
        assert gap <= width + 2 * eps[i], \
            (f"query {i}: GPU face {fg[i]} at {np.sqrt(d2_alt)!r} vs oracle face {fr[i]} at "
             f"{dr[i]!r}: gap {gap:.3g} > window {width:.3g} + 2 x float32 bound {eps[i]:.3g}")
        ties += 1
    assert ties <= max(3, max_tie_frac * Q.shape[0]), f"{ties} float32 tie mismatches"
    # barycentrics and points on agreeing faces
    same = np.nonzero(both & (fg == fr))[0]
    if "bary" in got and same.size:
        bg = host(got["bary"])[same]
        br = ref["bary"][same]
        wc = well_conditioned(V, F, fr[same])
        assert np.abs(bg[wc] - br[wc]).max(initial=0) <= 1e-5, "barycentric weights"
        assert np.all(np.abs(bg.sum(1) - 1) <= 1e-5)
    if "point" in got and same.size:
        pg = host(got["point"])[same]
        assert np.abs(pg - ref["point"][same]).max(initial=0) <= 1e-5 * max(diag, 1.0), "points"
    return dict(n=Q.shape[0], hits=int(both.sum()), ties=ties, cutoff_edge=len(odd))


def check_gaussians(got, ref, tol=1e-5):
    mu, quat, scale = (host(x) for x in got)
    assert np.abs(mu - ref["mu"]).max(initial=0) <= tol, "mu"
    assert np.abs(scale - ref["scale"]).max(initial=0) <= tol, "scale"
    q, qr = quat.astype(np.float64), ref["quat"]
    # q and -q are the same rotation; the sign rule can flip when |w| is at rounding level
    flip = (np.abs(qr[:, 0]) < 1e-5) & ((q * qr).sum(1) < 0)
    q[flip] *= -1
    assert np.abs(q - qr).max(initial=0) <= tol, "quaternion"


def gpu_boxes(A, n):
    """Per-node boxes [2n-1, 6] (internal then leaves) read from the child slots of the
    node records; also checks that each slot carries the child's own index."""
    nodes = host(A["nodes"])
    nodes_i = host(A["nodes_i"])
    parent = host(A["parent"]).astype(np.int64)
    root = host(A["root"])
    boxes = np.empty((2 * n - 1, 6), np.float32)
    is_root = parent < 0
    boxes[is_root] = np.r_[root[0], root[1]]
    nid = np.nonzero(~is_root)[0]
    p, side = parent[nid] >> 1, parent[nid] & 1
    boxes[nid, :3] = nodes[p, 2 * side, :3]
    boxes[nid, 3:] = nodes[p, 2 * side + 1, :3]
    enc = nodes_i[p, 2 * side, 3]
    expect = np.where(nid < n - 1, nid, -(nid - (n - 1) + 1))
    assert np.array_equal(enc, expect), "record slots must carry their child's index"
    return boxes


def assert_identical(got: dict, ref: dict, face: str = "face") -> None:
    """Two NearestSurface results for the same queries and mesh that differ only in how
    they were searched (another tree, traversal variant, lane width, warm start or
    query order): the tie rule makes the answer a function of the query and the mesh,
    so every output must be equal bit for bit.  Only the keys of `got` that share the
    face's suffix are compared ("face", "bary", ... or "faceA", "baryA", ...)."""
    suffix = face[len("face"):]
    keys = [k for k in got if k.endswith(suffix) and k in ref]
    assert face in keys
    for k in keys:
        a, b = got[k], ref[k]
        if not torch.equal(a, b):
            diff = (a != b) if a.dim() == 1 else (a != b).any(dim=1)
            n = int(diff.sum().item())
            i = int(torch.nonzero(diff)[0].item())
            raise AssertionError(f"{k}: {n} of {a.shape[0]} differ; first at {i}: "
                                 f"{a[i].tolist()} vs {b[i].tolist()}")


def point_grad_atol(Q, V, gmax: float) -> float:
    """Float32 error bound of a point-to-mesh gradient 2 g (q - c): q - c is formed from
    coordinates of magnitude up to |q| + max|v| (c = sum_j b_j v_j in float32), so its
    rounding is about 8 x 2^-24 x (|q| + max|v|) per component whatever its size; a
    sample on or near the surface has q - c at that level itself."""
    s = float(np.abs(np.asarray(Q)).max(initial=0.0)) + float(np.abs(np.asarray(V)).max(initial=0.0))
    return 2.0 * abs(gmax) * 8 * 2.0 ** -24 * s


def vertex_weight_sums(nV, F, face, bary):
    """Per vertex, the sum over queries of the barycentric weight it receives (face -1
    skipped): a vertex gradient accumulates that many per-query errors."""
    face = np.asarray(face)
    keep = face >= 0
    idx = np.asarray(F)[face[keep]].reshape(-1)
    return np.bincount(idx, weights=np.asarray(bary, np.float64)[keep].reshape(-1), minlength=nV)


def assert_grad_close(got, ref, rtol: float = 1e-4, what: str = "gradient", atol=0.0) -> None:
    """Element-wise gradient check: |g - g_ref| <= rtol * max(|g_ref|, |row|,
    1e-3 max|row|) + atol for every component, |row| the norm of the component's row (a
    vertex's or query's gradient vector).  The row term covers components that cancel
    to near zero inside a row; the global floor covers rows whose float32 atomic sums
    cancel; atol (a scalar or one value per row) is the float32 error of forming q - c
    itself (see point_grad_atol)."""
    g = np.asarray(got, np.float64).reshape(np.shape(ref)[0], -1)
    r = np.asarray(ref, np.float64).reshape(g.shape)
    row = np.linalg.norm(r, axis=1, keepdims=True)
    scale = np.maximum(np.maximum(np.abs(r), row), 1e-3 * row.max(initial=0.0))
    at = np.asarray(atol, np.float64)
    at = at.reshape(-1, 1) if at.ndim == 1 else at
    err = np.maximum(np.abs(g - r) - at, 0.0)
    bad = err > rtol * scale
    if bad.any():
        i, j = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {int(bad.sum())} components off; first [{i},{j}]: "
                             f"{g[i, j]!r} vs {r[i, j]!r} (scale {scale[i, j]:.3g}); "
                             f"worst |g - g_ref| / scale {(err / np.maximum(scale, 1e-300)).max():.3g} "
                             f"(limit {rtol:g})")
