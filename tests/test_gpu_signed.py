"""GPU signed distance (inside negative, angle-weighted pseudo-normals) against
the oracle: signs equal wherever the distance exceeds 1e-4 of the diagonal,
magnitudes within float32 rounding; the exact cube; refit between calls."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_00444_gb300 import MeshBVH
from parity import dev, host
from test_oracle_signed import box_sdf, cube
from workloads.meshes import icosphere, torus, TorusSkinning
from workloads.sampling import uniform_box

pytestmark = pytest.mark.gpu


def check_signed(V, F, Q, got, max_dist=np.inf):
    ref = oracle.signed_distance(V, F, Q)["sd"]
    diag = oracle.mesh_diag(V, F)
    sd = host(got["sdist"]).astype(np.float64)
    far = np.abs(ref) > max_dist
    assert np.isinf(sd[far]).all()
    ok = ~far
    assert np.abs(np.abs(sd[ok]) - np.abs(ref[ok])).max() <= 1e-5 * diag + 3e-6 * np.abs(ref[ok]).max()
    clear = ok & (np.abs(ref) > 1e-4 * diag)
    assert (np.sign(sd[clear]) == np.sign(ref[clear])).all()


def test_cube_signed_distance():
    V, F = cube()
    rng = np.random.default_rng(3)
    P = np.concatenate([rng.uniform(-2.5, 2.5, (3000, 3)),
                        np.sign(rng.normal(size=(800, 3))) * rng.uniform(0.8, 1.2, (800, 3))]).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V.astype(np.float32)), dev(F))
    got = bvh.signed_distance(dev(P))
    sd = host(got["sdist"]).astype(np.float64)
    np.testing.assert_allclose(sd, box_sdf(P.astype(np.float64)), atol=2e-6)
    check_signed(V, F, P, got)
    assert bvh.status()[0] == 0


def test_icosphere_and_cutoff():
    V, F = icosphere(4)
    Q = uniform_box(4001, [-1.5] * 3, [1.5] * 3, seed=4).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    check_signed(V, F, Q, bvh.signed_distance(dev(Q)))
    check_signed(V, F, Q, bvh.signed_distance(dev(Q), max_dist=0.1), max_dist=0.1)


def test_skinned_torus_full_size_refit_between_calls():
    """200k faces: the normals follow the refit vertices; sampled against the oracle."""
    V0, F = torus(400, 250)
    sk = TorusSkinning(V0, seed=3000)
    lo, hi = V0.min(0) - 0.2, V0.max(0) + 0.2
    Q = uniform_box(1 << 18, lo, hi, seed=5).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V0), dev(F))
    pick = np.random.default_rng(6).choice(Q.shape[0], 1500, replace=False)
    for t in (0, 30):
        V = sk.frame(t)
        bvh.refit(dev(V))
        got = bvh.signed_distance(dev(Q), max_dist=0.05)
        sub = {k: v[dev(pick.astype(np.int64))] for k, v in got.items()}
        check_signed(V, F, Q[pick], sub, max_dist=0.05)
        inside = host(got["sdist"]) < 0
        assert 0.0 < inside.mean() < 0.2
    assert bvh.status()[0] & ~0x4 == 0


def test_reproducible_run_to_run_and_vertex_normals():
    """Queries placed just off the vertices of a skinned torus (their nearest point is a
    vertex, where the pseudo-normal is the angle-weighted sum over the vertex's faces):
    two calls give the same signed distances bit for bit, and the signs match the
    oracle's."""
    V0, F = torus(60, 40)
    V = TorusSkinning(V0, seed=3003).frame(20)
    rng = np.random.default_rng(8)
    idx = rng.choice(V.shape[0], 2000, replace=False)
    # offsets along the vertex normals (mean of the incident face normals): outward at
    # the convex vertices of the outer half lands in their vertex regions
    V64 = V.astype(np.float64)
    fn = np.cross(V64[F[:, 1]] - V64[F[:, 0]], V64[F[:, 2]] - V64[F[:, 0]])
    vn = np.zeros_like(V64)
    for k in range(3):
        np.add.at(vn, F[:, k], fn)
    d = vn[idx] / np.linalg.norm(vn[idx], axis=1, keepdims=True)
    Q = np.concatenate([V64[idx] + 0.004 * d, V64[idx] - 0.004 * d]).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V0), dev(F))
    bvh.refit(dev(V))
    a = bvh.signed_distance(dev(Q))
    b = bvh.signed_distance(dev(Q))
    for k in a:
        assert torch.equal(a[k], b[k]), k
    bary = host(a["bary"])
    on_vertex = ((bary == 0).sum(1) == 2).mean()
    assert on_vertex > 0.1
    check_signed(V, F, Q, a)
    assert bvh.status()[0] == 0
