"""The oracle's all-core forms (OpenMP over queries / Gaussians) give exactly the
serial oracle's results: brute-force closest point with and without a cutoff,
ragged and empty inputs, degenerate faces; rebind with degenerate faces and
offsets; Chamfer.  They exist to time the CPU baseline on every host core and to
check large samples; the serial functions stay the reference."""
import numpy as np

import oracle
from workloads.meshes import displaced_icosphere, icosphere
from workloads.sampling import osada_barycentrics, points_from, sample_surface, uniform_box


def _same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_closest_point_parallel_equals_serial():
    V, F = displaced_icosphere(3, 0.1, 1.3)
    F = F.copy()
    F[::9, 2] = F[::9, 0]                                   # degenerate (segment) faces
    for n in (0, 1, 7, 1001):
        Q = uniform_box(n, [-1.4] * 3, [1.4] * 3, seed=n + 11)
        for cut in (np.inf, 0.05, 0.0):
            _same(oracle.closest_point(V, F, Q, cut), oracle.closest_point(V, F, Q, cut, parallel=True))
    Q = np.concatenate([V[:200], uniform_box(50, [-1.2] * 3, [1.2] * 3, seed=3)])   # on vertices: ties
    _same(oracle.closest_point(V, F, Q), oracle.closest_point(V, F, Q, parallel=True))
    Q = uniform_box(20, [-1] * 3, [1] * 3, seed=4)
    _same(oracle.closest_point(V, F[:0], Q), oracle.closest_point(V, F[:0], Q, parallel=True))


def test_bind_and_chamfer_parallel_equal_serial():
    V, F = displaced_icosphere(2, 0.1, 0.2)
    F = F.copy()
    F[::7, 1] = F[::7, 0]
    rng = np.random.default_rng(8)
    G = 3000
    gface = rng.integers(0, F.shape[0], G).astype(np.int32)
    gbary = osada_barycentrics(rng, G)
    goff = rng.normal(scale=0.02, size=G)
    a = oracle.bind_gaussians(V, F, gface, gbary, goff)
    b = oracle.bind_gaussians(V, F, gface, gbary, goff, parallel=True)
    _same(a, b)
    assert a["n_degenerate"] > 0
    VA, FA = icosphere(2)
    fa, ba = sample_surface(VA, FA, 700, seed=9)
    fb, bb = sample_surface(V, F, 600, seed=10)
    SA, SB = points_from(VA, FA, fa, ba), points_from(V, F, fb, bb)
    r1 = oracle.chamfer(VA, FA, SA, V, F, SB)
    r2 = oracle.chamfer(VA, FA, SA, V, F, SB, parallel=True)
    for x, y in zip(r1, r2):
        assert np.array_equal(x, y)


def test_thread_count_is_reported():
    assert oracle.num_threads() >= 1
