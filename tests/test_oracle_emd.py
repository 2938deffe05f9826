"""Pins of the oracle's Earth Mover's Distance (exact assignment, mean Euclidean
cost): brute force over all permutations on tiny sets, the sorted matching of
points on a line, and a pure translation (EMD = |t| exactly: by the triangle
inequality no permutation beats the identity)."""
import itertools

import numpy as np

import oracle


def test_brute_force_permutations():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5, 7):
        A, B = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
        C = np.linalg.norm(A[:, None] - B[None], axis=2)
        best = min(C[np.arange(n), list(p)].mean() for p in itertools.permutations(range(n)))
        e, sigma = oracle.emd(A, B)
        assert abs(e - best) < 1e-12
        assert sorted(sigma) == list(range(n))


def test_points_on_a_line_match_in_sorted_order():
    rng = np.random.default_rng(1)
    a, b = rng.uniform(0, 10, 300), rng.uniform(-3, 7, 300)
    d = np.array([0.3, -0.4, 0.866])
    d /= np.linalg.norm(d)
    e, _ = oracle.emd(a[:, None] * d, b[:, None] * d)
    assert abs(e - np.abs(np.sort(a) - np.sort(b)).mean()) < 1e-9


def test_translation_is_its_length():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(400, 3))
    t = np.array([0.05, -0.02, 0.1])
    e, sigma = oracle.emd(A, A + t)
    assert abs(e - np.linalg.norm(t)) < 1e-12
    assert (sigma == np.arange(400)).all()
