"""CPU float64 oracle for the per-frame dynamic-mesh update -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package; the CUDA library never does, and the two
share no code.  The arithmetic lives in ``oracle.c`` (plain serial C, float64,
with the Morton-key step in float32 as its recipe defines; OpenMP forms of the
brute-force closest point, the rebind and the Chamfer run the same per-query
arithmetic over the host's cores); this module only compiles it and marshals
numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

F32P = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
U32P = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
I64 = C.c_int64


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FMA contraction), with OpenMP for
    the *_omp forms when the compiler supports it (otherwise they run on one thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
        r = subprocess.run(base + ["-fopenmp", _SRC, "-lm", "-o", tmp], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base + [_SRC, "-lm", "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_point_triangle.restype = C.c_double
        L.orc_point_triangle.argtypes = [F64P, F64P, F64P, F64P, F64P, F64P]
        L.orc_mesh_diag.restype = C.c_double
        L.orc_mesh_diag.argtypes = [F64P, I32P, I64]
        L.orc_closest_point_mesh.restype = None
        L.orc_closest_point_mesh.argtypes = [F64P, I32P, I64, F64P, I64, C.c_double,
                                             I32P, F64P, F64P, F64P, C.c_void_p]
        L.orc_morton.restype = None
        L.orc_morton.argtypes = [F32P, I32P, I64, U32P]
        L.orc_sort_pairs.restype = None
        L.orc_sort_pairs.argtypes = [U32P, I64, U32P, I32P]
        L.orc_karras.restype = None
        L.orc_karras.argtypes = [U32P, I64, I32P, I32P, I32P, I32P, I32P]
        L.orc_ploc.restype = None
        L.orc_ploc.argtypes = [F32P, I64, C.c_int, I32P, I32P, I32P, I32P, I32P, I32P]
        L.orc_collapse.restype = None
        L.orc_collapse.argtypes = [I32P, I32P, I32P, I32P, I64, C.c_int, I32P]
        L.orc_node_boxes.restype = None
        L.orc_node_boxes.argtypes = [F32P, I32P, I32P, I64, I32P, I32P, F32P]
        L.orc_bind_gaussians.restype = C.c_int64
        L.orc_bind_gaussians.argtypes = [F64P, I32P, I32P, F64P, C.c_void_p, I64,
                                         F64P, F64P, F64P, I32P]
        L.orc_num_threads.restype = C.c_int
        L.orc_num_threads.argtypes = []
        L.orc_closest_point_mesh_omp.restype = None
        L.orc_closest_point_mesh_omp.argtypes = [F64P, I32P, I64, F64P, I64, C.c_double,
                                                 I32P, F64P, F64P, F64P]
        L.orc_bind_gaussians_omp.restype = C.c_int64
        L.orc_bind_gaussians_omp.argtypes = [F64P, I32P, I32P, F64P, C.c_void_p, I64,
                                             F64P, F64P, F64P, I32P]
        L.orc_chamfer_omp.restype = None
        L.orc_chamfer_omp.argtypes = [F64P, I32P, I64, F64P, I64, F64P, I32P, I64, F64P, I64,
                                      F64P, F64P, F64P]
        L.orc_chamfer.restype = None
        L.orc_chamfer.argtypes = [F64P, I32P, I64, F64P, I64, F64P, I32P, I64, F64P, I64,
                                  F64P, F64P, F64P]
        L.orc_closest_point_backward.restype = None
        L.orc_closest_point_backward.argtypes = [F64P, I32P, F64P, I64, I32P, F64P, F64P,
                                                 F64P, F64P]
        L.orc_interpolate.restype = None
        L.orc_interpolate.argtypes = [F64P, I32P, I32P, F64P, I64, F64P]
        L.orc_interpolate_backward.restype = None
        L.orc_interpolate_backward.argtypes = [I32P, I32P, F64P, I64, F64P, F64P]
        L.orc_bind_gaussians_backward.restype = None
        L.orc_bind_gaussians_backward.argtypes = [F64P, I32P, I32P, F64P, C.c_void_p, I64,
                                                  F64P, F64P, F64P, F64P]
        L.orc_knn_project.restype = None
        L.orc_knn_project.argtypes = [F64P, I32P, I64, F64P, I64, C.c_int, C.c_void_p, C.c_double,
                                      F64P, I32P, F64P]
        L.orc_signed_distance.restype = None
        L.orc_signed_distance.argtypes = [F64P, I32P, I64, F64P, I64, F64P, I32P]
        L.orc_gs_render.restype = None
        L.orc_gs_render.argtypes = [F64P, F64P, F64P, F64P, F64P, I64, F64P, F64P, C.c_double,
                                    C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double,
                                    F64P, F64P, F64P]
        L.orc_gs_render_flags.restype = None
        L.orc_gs_render_flags.argtypes = [F64P, F64P, F64P, F64P, F64P, I64, F64P, F64P, C.c_double,
                                          C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double,
                                          F64P, C.c_double, F64P, F64P,
                                          np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")]
        _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def point_triangle(p, a, b, c):
    """(d2, bary[3], point[3]) of the closest point of triangle abc to p (float64)."""
    bary = np.zeros(3)
    point = np.zeros(3)
    d2 = lib().orc_point_triangle(_f64(p), _f64(a), _f64(b), _f64(c), bary, point)
    return d2, bary, point


def mesh_diag(V, F):
    return lib().orc_mesh_diag(_f64(V), _i32(F), F.shape[0])


def num_threads() -> int:
    """Threads the *_omp forms use (1 when built without OpenMP)."""
    return int(lib().orc_num_threads())


def closest_point(V, F, Q, max_dist=np.inf, all_d2=False, parallel=False):
    """Brute-force NearestSurface of every query: dict(face, bary, point, d2[, d2_all]).
    parallel=True runs the queries over every host core (orc_closest_point_mesh_omp,
    identical results; all_d2 is then unavailable)."""
    V, F, Q = _f64(V), _i32(F), _f64(Q).reshape(-1, 3)
    nQ, nF = Q.shape[0], F.shape[0]
    face = np.empty(nQ, np.int32)
    bary = np.empty((nQ, 3))
    point = np.empty((nQ, 3))
    d2 = np.empty(nQ)
    if parallel:
        if all_d2:
            raise ValueError("all_d2 needs the serial form")
        lib().orc_closest_point_mesh_omp(V, F, nF, Q, nQ, float(max_dist), face, bary, point, d2)
        return dict(face=face, bary=bary, point=point, d2=d2)
    d2a = np.empty((nQ, nF)) if all_d2 else None
    lib().orc_closest_point_mesh(V, F, nF, Q, nQ, float(max_dist), face, bary, point, d2,
                                 d2a.ctypes.data if all_d2 else None)
    out = dict(face=face, bary=bary, point=point, d2=d2)
    if all_d2:
        out["d2_all"] = d2a
    return out


def morton(V, F):
    F = _i32(F)
    keys = np.empty(F.shape[0], np.uint32)
    lib().orc_morton(_f32(V), F, F.shape[0], keys)
    return keys


def sort_pairs(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    sk = np.empty_like(keys)
    perm = np.empty(keys.shape[0], np.int32)
    lib().orc_sort_pairs(keys, keys.shape[0], sk, perm)
    return sk, perm


def karras(sorted_keys):
    """(left, right, parent, first, last); children: internal c >= 0, leaf j as -(j+1)."""
    k = np.ascontiguousarray(sorted_keys, dtype=np.uint32)
    n = k.shape[0]
    m = max(n - 1, 1)
    left = np.zeros(m, np.int32)
    right = np.zeros(m, np.int32)
    first = np.zeros(m, np.int32)
    last = np.zeros(m, np.int32)
    parent = np.zeros(max(2 * n - 1, 1), np.int32)
    lib().orc_karras(k, n, left, right, parent, first, last)
    if n <= 1:
        return (left[:0], right[:0], parent[:max(2 * n - 1, 0)], first[:0], last[:0])
    return left, right, parent, first, last


def leaf_boxes(V, F, perm):
    """[n, 6] float32 boxes (lo, hi) of the faces perm[0..n-1] (exact min / max)."""
    V = np.asarray(V, np.float32)
    tri = V[np.asarray(F)[np.asarray(perm)]]
    return np.ascontiguousarray(np.concatenate([tri.min(1), tri.max(1)], 1), dtype=np.float32)


def ploc(leaf_box, radius=16):
    """Agglomerative tree (orc_ploc) over leaf boxes in Morton order:
    (order, left, right, parent, first, last) in the layout of karras()."""
    lb = np.ascontiguousarray(leaf_box, dtype=np.float32)
    n = lb.shape[0]
    m = max(n - 1, 1)
    order = np.zeros(max(n, 1), np.int32)
    left = np.zeros(m, np.int32)
    right = np.zeros(m, np.int32)
    first = np.zeros(m, np.int32)
    last = np.zeros(m, np.int32)
    parent = np.zeros(max(2 * n - 1, 1), np.int32)
    lib().orc_ploc(lb, n, int(radius), order, left, right, parent, first, last)
    if n <= 1:
        return (order[:n], left[:0], right[:0], parent[:max(2 * n - 1, 0)], first[:0], last[:0])
    return order, left, right, parent, first, last


def build_ploc(V, F, radius=16):
    """Whole serial agglomerative build: the Morton order of build_lbvh, orc_ploc over
    its leaf boxes, and the node boxes of the resulting layout."""
    keys = morton(V, F)
    sk, perm0 = sort_pairs(keys)
    order, left, right, parent, first, last = ploc(leaf_boxes(V, F, perm0), radius)
    perm = perm0[order]
    boxes = node_boxes(V, F, perm, first, last)
    return dict(keys=keys, leaf_keys=sk[order], perm=perm, left=left, right=right, parent=parent,
                first=first, last=last, boxes=boxes)


def collapse(left, right, first, last, leaf_size):
    """Child links of every internal node with leaf collapse at leaf_size (orc_collapse):
    [n-1, 4] int32 = (left link, left count, right link, right count); a leaf range is
    (-(first + 1), faces), an internal child (c, c)."""
    left = np.ascontiguousarray(left, dtype=np.int32)
    m = left.shape[0]
    link = np.zeros((max(m, 1), 4), np.int32)
    lib().orc_collapse(left, np.ascontiguousarray(right, dtype=np.int32),
                       np.ascontiguousarray(first, dtype=np.int32),
                       np.ascontiguousarray(last, dtype=np.int32), m + 1, int(leaf_size), link)
    return link[:m]


def node_boxes(V, F, perm, first, last):
    """[2n-1, 6] (lo, hi) boxes: internal nodes 0..n-2 then leaves 0..n-1."""
    n = perm.shape[0]
    boxes = np.empty((2 * n - 1, 6), np.float32)
    f_ = _i32(first) if n > 1 else np.zeros(1, np.int32)
    l_ = _i32(last) if n > 1 else np.zeros(1, np.int32)
    lib().orc_node_boxes(_f32(V), _i32(F), _i32(perm), n, f_, l_, boxes)
    return boxes


def build_lbvh(V, F):
    """Whole serial LBVH build: dict(keys, sorted_keys, perm, left, right, parent, boxes)."""
    keys = morton(V, F)
    sk, perm = sort_pairs(keys)
    left, right, parent, first, last = karras(sk)
    boxes = node_boxes(V, F, perm, first, last)
    return dict(keys=keys, sorted_keys=sk, perm=perm, left=left, right=right, parent=parent,
                first=first, last=last, boxes=boxes)


def bind_gaussians(V, F, gface, gbary, goff=None, parallel=False):
    """dict(mu [G,3], quat [G,4] (w,x,y,z), scale [G,3], flags [G], n_degenerate);
    parallel=True: orc_bind_gaussians_omp over every host core (identical results)."""
    gface = _i32(gface)
    G = gface.shape[0]
    mu = np.empty((G, 3))
    quat = np.empty((G, 4))
    scale = np.empty((G, 3))
    flags = np.empty(G, np.int32)
    go = None if goff is None else _f64(goff)
    fn = lib().orc_bind_gaussians_omp if parallel else lib().orc_bind_gaussians
    nd = fn(_f64(V), _i32(F), gface, _f64(gbary),
                                  None if go is None else go.ctypes.data, G, mu, quat, scale,
                                  flags)
    return dict(mu=mu, quat=quat, scale=scale, flags=flags, n_degenerate=int(nd))


def chamfer(VA, FA, SA, VB, FB, SB, parallel=False):
    """(out[2] = [mean d(SA, B)^2, mean d(SB, A)^2], dA, dB) in float64; parallel=True:
    orc_chamfer_omp over every host core (identical results)."""
    SA, SB = _f64(SA).reshape(-1, 3), _f64(SB).reshape(-1, 3)
    out = np.zeros(2)
    dA = np.empty(SA.shape[0])
    dB = np.empty(SB.shape[0])
    (lib().orc_chamfer_omp if parallel else lib().orc_chamfer)(_f64(VA), _i32(FA), FA.shape[0], SA, SA.shape[0],
                      _f64(VB), _i32(FB), FB.shape[0], SB, SB.shape[0], out, dA, dB)
    return out, dA, dB


def closest_point_backward(V, F, Q, face, bary, g):
    """(dL/dQ [nQ,3], dL/dV [nV,3]) for upstream dL/d(d2) = g [nQ]."""
    Q = _f64(Q).reshape(-1, 3)
    gQ = np.zeros((Q.shape[0], 3))
    gV = np.zeros((V.shape[0], 3))
    lib().orc_closest_point_backward(_f64(V), _i32(F), Q, Q.shape[0], _i32(face), _f64(bary),
                                     _f64(g), gQ, gV)
    return gQ, gV


def interpolate(V, F, face, bary):
    face = _i32(face)
    out = np.empty((face.shape[0], 3))
    lib().orc_interpolate(_f64(V), _i32(F), face, _f64(bary), face.shape[0], out)
    return out


def interpolate_backward(nV, F, face, bary, gP):
    face = _i32(face)
    gV = np.zeros((nV, 3))
    lib().orc_interpolate_backward(_i32(F), face, _f64(bary), face.shape[0], _f64(gP), gV)
    return gV


def bind_gaussians_backward(V, F, gface, gbary, gmu, gq, gs, goff=None):
    gface = _i32(gface)
    gV = np.zeros((V.shape[0], 3))
    go = None if goff is None else _f64(goff)
    lib().orc_bind_gaussians_backward(_f64(V), _i32(F), gface, _f64(gbary),
                                      None if go is None else go.ctypes.data, gface.shape[0],
                                      _f64(gmu), _f64(gq), _f64(gs), gV)
    return gV


def knn_project(V, F, Q, k=4, anchor=None, anchor_w=0.0):
    """k-NN weighted surface projection (the NearestSurface of Eq. 1, temporal tracking):
    blend of the k nearest faces' closest points with weights 1/max(d, 1e-6 diag), then
    optionally (1 - anchor_w) * that + anchor_w * anchor.  dict(point, face[Q,k], d2[Q,k])."""
    V, F, Q = _f64(V), _i32(F), _f64(Q).reshape(-1, 3)
    nQ = Q.shape[0]
    point = np.empty((nQ, 3))
    face = np.empty((nQ, k), np.int32)
    d2 = np.empty((nQ, k))
    A = None if anchor is None else _f64(anchor).reshape(-1, 3)
    lib().orc_knn_project(V, F, F.shape[0], Q, nQ, int(k), None if A is None else A.ctypes.data,
                          float(anchor_w), point, face, d2)
    return dict(point=point, face=face, d2=d2)


def signed_distance(V, F, Q):
    """Signed NearestSurface distance (inside negative) by angle-weighted pseudo-normals;
    dict(sd, face).  Assumes a closed, outward-oriented manifold mesh."""
    V, F, Q = _f64(V), _i32(F), _f64(Q).reshape(-1, 3)
    nQ = Q.shape[0]
    sd = np.empty(nQ)
    face = np.empty(nQ, np.int32)
    lib().orc_signed_distance(V, F, F.shape[0], Q, nQ, sd, face)
    return dict(sd=sd, face=face)


def emd(A, B):
    """Earth Mover's Distance between two equal-size point sets (Sec. 4.2's EMD on
    sampled points): the minimum over bijections sigma of the mean Euclidean distance
    |a_i - b_sigma(i)|, by exact linear assignment (scipy's solver as the library step).
    Returns (emd, sigma)."""
    from scipy.optimize import linear_sum_assignment
    from scipy.spatial.distance import cdist
    A = _f64(A).reshape(-1, 3)
    B = _f64(B).reshape(-1, 3)
    if A.shape[0] != B.shape[0]:
        raise ValueError("EMD needs equal-size point sets")
    if A.shape[0] == 0:
        return 0.0, np.zeros(0, np.int64)
    C = cdist(A, B)
    r, c = linear_sum_assignment(C)
    sigma = np.empty(A.shape[0], np.int64)
    sigma[r] = c
    return float(C[r, c].mean()), sigma


def gs_render(mu, quat, scale, opacity, color, Rc, tc, fx, fy, cx, cy, W, H, near=0.01,
              background=(0.0, 0.0, 0.0), flags=False, margin=2e-3):
    """Gaussian splatting render (forward equations of 3DGS, 16 x 16 tiles): image [H, W, 3]
    and final transmittance [H, W], float64.  flags=True adds the parity flags of
    orc_gs_render_flags (bool [H, W]: pixels a float32 implementation may legitimately
    render differently, a decision within float32 reach of its threshold; relative
    margin `margin` for the per-pixel thresholds); the image is the same either way."""
    mu, quat, scale = _f64(mu).reshape(-1, 3), _f64(quat).reshape(-1, 4), _f64(scale).reshape(-1, 3)
    opacity, color = _f64(opacity).reshape(-1), _f64(color).reshape(-1, 3)
    n = mu.shape[0]
    image = np.empty((H, W, 3))
    trans = np.empty((H, W))
    args = (mu, quat, scale, opacity, color, n, _f64(Rc).reshape(3, 3), _f64(tc).reshape(3),
            float(fx), float(fy), float(cx), float(cy), int(W), int(H), float(near), _f64(background).reshape(3))
    if not flags:
        lib().orc_gs_render(*args, image, trans)
        return image, trans
    fragile = np.zeros((H, W), np.uint8)
    lib().orc_gs_render_flags(*args, float(margin), image, trans, fragile)
    return image, trans, fragile.astype(bool)
