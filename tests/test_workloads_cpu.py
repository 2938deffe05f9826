"""The seeded input generators (no GPU): the marching-cubes surface of the varying-topology
sequence is a closed, consistently oriented triangle mesh whose vertices lie on the SDF's
zero set, with the face counts the design states; its derived case table has the
textbook properties; surface sampling is uniform by area and Osada's barycentres are
uniform on the triangle; the torus grid and the icospheres have their closed-form sizes."""
import numpy as np
import pytest

from workloads.isosurface import BlobSequence, case_table, marching_cubes, smin
from workloads.meshes import icosphere, torus
from workloads.sampling import face_areas, osada_barycentrics, sample_surface


def edge_counts(F):
    """Directed and undirected edge multiplicities of a triangle list."""
    d = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    und = np.sort(d, axis=1)
    _, cu = np.unique(und, axis=0, return_counts=True)
    _, cd = np.unique(d, axis=0, return_counts=True)
    return cu, cd


def point_sdf(seq, tau, P):
    d = None
    for c, r in zip(seq.centres(tau), seq.radius):
        di = np.linalg.norm(P - c, axis=1) - r
        d = di if d is None else smin(d, di, seq.k)
    return d


@pytest.mark.parametrize("frame", [0, 33, 60])
def test_blob_surface_is_closed_oriented_and_on_the_zero_set(frame):
    seq = BlobSequence(2000)
    V, F = seq.mesh(frame, N=64)
    cu, cd = edge_counts(F)
    assert np.all(cu == 2), "every edge is shared by exactly two faces"
    assert np.all(cd == 1), "each directed edge once: neighbours are consistently oriented"
    h = 2.0 / 63
    sd = point_sdf(seq, seq.tau(frame), V.astype(np.float64))
    assert np.abs(sd).max() < 0.25 * h, "vertices interpolate the zero crossing of each edge"
    # outward orientation: the signed volume is positive
    a, b, c = (V[F[:, k]].astype(np.float64) for k in range(3))
    assert np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0 > 0


def test_blob_face_counts_at_the_benchmark_resolution():
    seq = BlobSequence(2000)
    counts = [seq.mesh(k)[1].shape[0] for k in (0, 30, 60, 90)]
    assert all(30000 <= c <= 55000 for c in counts), counts


def test_case_table_textbook_properties():
    tris, count = case_table()                 # [256, max, 3] edge triples, [256] counts
    assert tris.shape[0] == 256 and count.shape[0] == 256
    assert count[0] == 0 and count[255] == 0
    for c in range(8):                        # one corner inside: one triangle
        assert count[1 << c] == 1 and count[255 ^ (1 << c)] == 1
    # a plane through the cube (a face's four corners on one side) needs two triangles
    assert count[0b01010101] == 2 and count[0b00001111] == 2
    # complementary sign patterns cut the same edges
    for c in range(256):
        a = {frozenset(t) for t in tris[c, :count[c]].tolist()}
        b = {frozenset(t) for t in tris[255 ^ c, :count[255 ^ c]].tolist()}
        ea = set().union(*a) if a else set()
        eb = set().union(*b) if b else set()
        assert ea == eb


def test_marching_cubes_of_a_sphere_has_the_sphere_area():
    N = 48
    x = np.linspace(-1, 1, N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    f = np.sqrt(X * X + Y * Y + Z * Z) - 0.6
    V, F = marching_cubes(f)
    area = face_areas(V, F).sum()
    assert abs(area - 4 * np.pi * 0.36) / (4 * np.pi * 0.36) < 0.02
    assert np.all(edge_counts(F)[0] == 2)


def test_osada_barycentres_are_uniform_on_the_triangle():
    b = osada_barycentrics(np.random.default_rng(0), 200000)
    assert np.allclose(b.sum(1), 1.0) and (b >= 0).all()
    assert np.allclose(b.mean(0), 1.0 / 3.0, atol=3e-3)
    # a uniform point's weight b0 has density 2 (1 - b0): P(b0 < 1/2) = 3/4
    assert abs((b[:, 0] < 0.5).mean() - 0.75) < 5e-3


def test_surface_samples_follow_face_area():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [3, 0, 0], [3, 3, 0], [0, 3, 0]], np.float32)
    F = np.array([[0, 1, 2], [3, 4, 5]], np.int32)     # areas 0.5 and 4.5
    face, bary = sample_surface(V, F, 100000, seed=3)
    assert abs((face == 1).mean() - 0.9) < 5e-3
    assert bary.dtype == np.float32 and np.allclose(bary.sum(1), 1.0, atol=1e-6)


def test_closed_form_mesh_sizes():
    V, F = torus(400, 250)
    assert V.shape == (100000, 3) and F.shape == (200000, 3)
    assert np.all(edge_counts(F)[0] == 2)
    for level, nv in ((3, 642), (5, 10242), (6, 40962)):
        V, F = icosphere(level)
        assert V.shape[0] == nv and F.shape[0] == 2 * (nv - 2)   # Euler: V - E + F = 2
        assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-6)


def test_torus_skinning():
    """4-bone linear-blend skinning: weights form a partition of unity, the motion has the
    stated period, and no vertex moves farther than its largest bone rotation (30 degrees)
    can carry it."""
    from workloads.meshes import TorusSkinning
    V0, F = torus(40, 25)
    sk = TorusSkinning(V0, seed=3000)
    assert np.allclose(sk.w.sum(1), 1.0) and (sk.w > 0).all()
    assert np.allclose(sk.frame(7), sk.frame(7 + sk.period), atol=1e-6)
    reach = np.linalg.norm(V0[:, None, :] - sk.pivot[None, :, :], axis=2).max(1)
    bound = 2.0 * np.sin(np.deg2rad(30.0) / 2.0) * reach
    for t in (0, 31, 62, 90):
        move = np.linalg.norm(sk.frame(t).astype(np.float64) - V0, axis=1)
        assert (move <= bound + 1e-5).all()
