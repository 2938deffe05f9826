"""Pins for the oracle's Chamfer distance (Sec. 4.2 reading: squared, mean per
direction, point-to-mesh) and for its analytic gradients, checked against
closed forms and float64 central differences of the oracle's own forward
functions (step 1e-6, points in general position).
"""
import numpy as np
import pytest

import oracle
from workloads.meshes import icosphere, displaced_icosphere
from workloads.sampling import sample_surface, points_from, osada_barycentrics


def square(z, half=1.0):
    V = np.array([[-half, -half, z], [half, -half, z], [half, half, z], [-half, half, z]])
    return V, np.array([[0, 1, 2], [0, 2, 3]], np.int32)


def test_parallel_squares_closed_form():
    h = 0.37
    VA, FA = square(0.0)
    VB, FB = square(h)
    rng = np.random.default_rng(1)
    SA = np.c_[rng.uniform(-0.9, 0.9, (500, 2)), np.zeros(500)]
    SB = np.c_[rng.uniform(-0.9, 0.9, (300, 2)), np.full(300, h)]
    out, dA, dB = oracle.chamfer(VA, FA, SA, VB, FB, SB)
    np.testing.assert_allclose(out, [h * h, h * h], rtol=1e-13)
    np.testing.assert_allclose(dA, h * h, rtol=1e-13)


def test_identical_meshes_have_zero_chamfer_and_symmetry():
    V, F = displaced_icosphere(2, 0.1, 0.5)
    fa, ba = sample_surface(V, F, 400, seed=2)
    fb, bb = sample_surface(V, F, 300, seed=3)
    # float32 weights need not sum to 1; renormalise so the samples lie on the surface
    ba = ba.astype(np.float64) / ba.sum(1, keepdims=True, dtype=np.float64)
    bb = bb.astype(np.float64) / bb.sum(1, keepdims=True, dtype=np.float64)
    SA = oracle.interpolate(V, F, fa, ba)
    SB = oracle.interpolate(V, F, fb, bb)
    out, _, _ = oracle.chamfer(V, F, SA, V, F, SB)
    assert out.max() < 1e-28
    V2, F2 = icosphere(3)
    o1, _, _ = oracle.chamfer(V, F, SA, V2, F2, SB)
    o2, _, _ = oracle.chamfer(V2, F2, SB, V, F, SA)
    np.testing.assert_allclose(o1, o2[::-1], rtol=1e-14)


def test_sphere_samples_against_inscribed_icosphere():
    """Exact-sphere samples of radius 1 against the unit icosphere (vertices on the sphere,
    faces inside it): every distance lies in [0, 1 - min face-plane distance]."""
    V, F = icosphere(3)
    a, b, c = [V.astype(np.float64)[F[:, k]] for k in range(3)]
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    hmin = np.abs(np.einsum("ij,ij->i", n, a)).min()
    rng = np.random.default_rng(4)
    S = rng.normal(size=(300, 3))
    S /= np.linalg.norm(S, axis=1, keepdims=True)
    out = oracle.closest_point(V, F, S)
    d = np.sqrt(out["d2"])
    assert (d <= 1 - hmin + 1e-12).all() and (d >= 0).all()


def general_position_queries(V, F, n, seed, r=1e-5):
    """Queries in general position: moving one by +-r along any axis keeps its nearest face
    and the set of its barycentric weights that are exactly 0 (its Voronoi region), so the
    central differences below (step 1e-6) never straddle a region boundary or a tie."""
    rng = np.random.default_rng(seed)
    Q = []
    while len(Q) < n:
        q = rng.uniform(-1.4, 1.4, size=(1, 3))
        o = oracle.closest_point(V, F, q)
        pattern = o["bary"][0] == 0.0
        ok = True
        for ax in range(3):
            for sgn in (-1.0, 1.0):
                qq = q.copy()
                qq[0, ax] += sgn * r
                o2 = oracle.closest_point(V, F, qq)
                if o2["face"][0] != o["face"][0] or ((o2["bary"][0] == 0.0) != pattern).any():
                    ok = False
        if ok:
            Q.append(q[0])
    return np.array(Q)


def test_closest_point_gradient_central_differences():
    V, F = displaced_icosphere(1, 0.1, 0.9)
    V = V.astype(np.float64)
    Q = general_position_queries(V, F, 25, seed=5)
    rng = np.random.default_rng(6)
    g = rng.normal(size=Q.shape[0])
    o = oracle.closest_point(V, F, Q)
    gQ, gV = oracle.closest_point_backward(V, F, Q, o["face"], o["bary"], g)
    L = lambda V_, Q_: g @ oracle.closest_point(V_, F, Q_)["d2"]
    h = 1e-6
    num_Q = np.zeros_like(Q)
    for i in range(Q.shape[0]):
        for c in range(3):
            Qp, Qm = Q.copy(), Q.copy()
            Qp[i, c] += h
            Qm[i, c] -= h
            num_Q[i, c] = (L(V, Qp) - L(V, Qm)) / (2 * h)
    np.testing.assert_allclose(gQ, num_Q, rtol=1e-6, atol=1e-8)
    used = np.unique(F[o["face"]])
    for v in used[:30]:
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[v, c] += h
            Vm[v, c] -= h
            num = (L(Vp, Q) - L(Vm, Q)) / (2 * h)
            assert gV[v, c] == pytest.approx(num, rel=1e-6, abs=1e-8)


def test_rebind_gradient_central_differences():
    V, F = displaced_icosphere(1, 0.1, 0.3)
    V = V.astype(np.float64)
    rng = np.random.default_rng(7)
    G = 60
    gface = rng.integers(0, F.shape[0], size=G).astype(np.int32)
    gbary = osada_barycentrics(rng, G)
    goff = rng.normal(scale=0.05, size=G)
    wm, wq, ws = rng.normal(size=(G, 3)), rng.normal(size=(G, 4)), rng.normal(size=(G, 3))

    def L(V_):
        o = oracle.bind_gaussians(V_, F, gface, gbary, goff)
        return (wm * o["mu"]).sum() + (wq * o["quat"]).sum() + (ws * o["scale"]).sum()

    gV = oracle.bind_gaussians_backward(V, F, gface, gbary, wm, wq, ws, goff)
    h = 1e-6
    for v in np.unique(F[gface])[:40]:
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[v, c] += h
            Vm[v, c] -= h
            num = (L(Vp) - L(Vm)) / (2 * h)
            assert gV[v, c] == pytest.approx(num, rel=1e-6, abs=1e-7)


def test_template_chamfer_gradient_central_differences():
    """Template (162-vertex icosphere) samples follow V; target is a displaced icosphere.
    L = w0 * mean d(S_T(V), target)^2 + w1 * mean d(S_target, template(V))^2."""
    VT, FT = icosphere(2, radius=0.95)
    VT = VT.astype(np.float64)
    VG, FG = displaced_icosphere(1, 0.1, 0.4)
    ft, bt = sample_surface(VT, FT, 80, seed=8)
    fg, bg = sample_surface(VG, FG, 60, seed=9)
    SG = points_from(VG, FG, fg, bg).astype(np.float64)
    w0, w1 = 0.7, 1.3

    def L(V_):
        S = oracle.interpolate(V_, FT, ft, bt)
        out, _, _ = oracle.chamfer(V_, FT, S, VG, FG, SG)
        return w0 * out[0] + w1 * out[1]

    S = oracle.interpolate(VT, FT, ft, bt)
    oA = oracle.closest_point(VG, FG, S)                 # template samples -> target
    oB = oracle.closest_point(VT, FT, SG)                # target samples -> template
    gS, _ = oracle.closest_point_backward(VG, FG, S, oA["face"], oA["bary"],
                                          np.full(S.shape[0], w0 / S.shape[0]))
    gV = oracle.interpolate_backward(VT.shape[0], FT, ft, bt, gS)
    _, gV2 = oracle.closest_point_backward(VT, FT, SG, oB["face"], oB["bary"],
                                           np.full(SG.shape[0], w1 / SG.shape[0]))
    gV = gV + gV2
    h = 1e-6
    rng = np.random.default_rng(10)
    for v in rng.choice(VT.shape[0], 30, replace=False):
        for c in range(3):
            Vp, Vm = VT.copy(), VT.copy()
            Vp[v, c] += h
            Vm[v, c] -= h
            num = (L(Vp) - L(Vm)) / (2 * h)
            assert gV[v, c] == pytest.approx(num, rel=1e-5, abs=1e-9)
