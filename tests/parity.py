"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (float32 GPU against the float64 oracle):
  * Morton keys, sort permutation, tree topology, node boxes: bit-exact.
  * distance: |d_gpu - d_ref| <= 1e-5 * max(d_ref, 1e-3 * diag)  (relative, with a
    floor because projected points sit at distance ~0).
  * nearest face: equal, except when the GPU's face is within the float32 error
    bound 8 * 2^-24 * (|q| + max|v|) of the oracle's tie window; those are
    counted separately and must stay a handful.
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
    eps32 = 8 * 2.0 ** -24 * (np.linalg.norm(Q, axis=1) + vmax) * 3
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
    # nearest face: exact unless a float32-scale tie
    idx = np.nonzero(both & (fg != fr))[0]
    ties = 0
    for i in idx:
        a, b, c = (V[F[fg[i]]][k].astype(np.float64) for k in range(3))
        d2_alt, _, _ = oracle.point_triangle(Q[i].astype(np.float64), a, b, c)
        window = dr[i] * (1 + TIE_REL) + tau
        assert np.sqrt(d2_alt) <= window + eps32[i], \
            f"query {i}: GPU face {fg[i]} at {np.sqrt(d2_alt)} vs oracle {fr[i]} at {dr[i]}"
        ties += 1
    assert ties <= max(3, max_tie_frac * Q.shape[0]), f"{ties} tie-rule mismatches"
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


def assert_same_up_to_near_ties(got: dict, ref: dict, face: str = "face", dist2: str = "dist2",
                                max_frac: float = 1e-3):
    """Two NearestSurface results for the same queries that differ only in the order in
    which faces were met (a warm start, a traversal variant, a query order): equal bit
    for bit, except queries whose kept face differs inside the tie rule's window (the
    online rule can keep a different face when three or more faces lie within about
    2e-6 of one another).  Those must be rare, both must be hits, and their distances
    must agree within that window.  Only the keys of `got` that share the face's
    suffix are compared ("face", "bary", ... or "faceA", "baryA", ...)."""
    suffix = face[len("face"):]
    keys = [k for k in got if k.endswith(suffix) and k in ref]
    fg, fr = got[face], ref[face]
    diff = fg != fr
    n = int(diff.sum().item())
    assert n <= max(2, max_frac * fg.numel()), f"{n} faces differ"
    keep = ~diff
    for k in keys:
        assert torch.equal(got[k][keep], ref[k][keep]), k
    if n:
        assert bool(((fg[diff] >= 0) & (fr[diff] >= 0)).all().item())
        if dist2 in got and dist2 in ref:
            dg = got[dist2][diff].double().sqrt()
            dr = ref[dist2][diff].double().sqrt()
            assert bool(((dg - dr).abs() <= 3 * TIE_REL * torch.maximum(dg, dr) + 1e-9).all().item())
    return n
