"""GPU Earth Mover's Distance (auction with epsilon scaling) against the
oracle's exact assignment: the value lies in [exact, exact + eps x diagonal]
(the epsilon-optimality bound), the assignment is a bijection whose float64
cost is the value returned, repeated calls agree bit for bit, and a pure
translation at the paper's 10K points gives its length."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_00444_gb300 import emd
from parity import dev, host
from workloads.meshes import displaced_icosphere, icosphere
from workloads.sampling import points_from, sample_surface

pytestmark = pytest.mark.gpu


def diag(A, B):
    P = np.concatenate([A, B])
    return float(np.linalg.norm(P.max(0) - P.min(0)))


def check_emd(A, B, eps_rel=1e-5):
    val, sigma, iters = emd(dev(A), dev(B), eps_rel=eps_rel, want_assignment=True)
    v = float(val.item())
    s = host(sigma).astype(np.int64)
    assert sorted(s) == list(range(A.shape[0]))
    cost = np.linalg.norm(A.astype(np.float64) - B[s].astype(np.float64), axis=1).mean()
    assert abs(cost - v) <= 1e-12 * max(1.0, abs(v))
    exact, _ = oracle.emd(A, B)
    C = diag(A, B)
    assert exact - 1e-7 * C <= v <= exact + eps_rel * C + 1e-7 * C, (v, exact, iters)
    return v, iters


@pytest.mark.parametrize("n", [1, 2, 7, 500, 1500])
def test_emd_random_sets(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, 3)).astype(np.float32)
    B = (rng.normal(size=(n, 3)) * 0.8 + 0.3).astype(np.float32)
    check_emd(A, B)


def test_emd_mesh_samples_and_repeatability():
    VA, FA = icosphere(3)
    VB, FB = displaced_icosphere(3, 0.1, 0.5)
    A = points_from(VA, FA, *sample_surface(VA, FA, 2000, seed=60)).astype(np.float32)
    B = points_from(VB, FB, *sample_surface(VB, FB, 2000, seed=61)).astype(np.float32)
    check_emd(A, B)
    x, y = emd(dev(A), dev(B)), emd(dev(A), dev(B))
    assert torch.equal(x, y)


def test_emd_translation_at_10k_points():
    V, F = icosphere(5)
    A = points_from(V, F, *sample_surface(V, F, 10000, seed=62)).astype(np.float32)
    t = np.array([0.01, -0.02, 0.015], np.float32)
    B = A + t
    v = float(emd(dev(A), dev(B), eps_rel=1e-5).item())
    C = diag(A, B)
    assert abs(v - np.linalg.norm(t)) <= 1e-5 * C + 1e-6
