"""Batched forms (one launch per phase over many scenes): every scene's tree,
query answers and Gaussians equal those of building that scene alone, bit for
bit; a sample is also checked against the oracle.  Scenes of very uneven size,
an empty scene and a one-face scene are included."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_00444_gb300 import MeshBatch, MeshBVH
from parity import check_closest, check_gaussians, dev, host
from workloads.meshes import displaced_icosphere, displaced_torus, icosphere, torus
from workloads.sampling import osada_barycentrics, uniform_box

pytestmark = pytest.mark.gpu


def scenes():
    out = [displaced_icosphere(3, 0.1, 0.3), displaced_torus(40, 25, 0.1, 3, 2, 0.5),
           (np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32)),
           (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), np.array([[0, 1, 2]], np.int32)),
           displaced_icosphere(5, 0.05, 1.1), torus(120, 75), icosphere(1)]
    return out


@pytest.fixture(scope="module")
def batch_and_singles():
    S = scenes()
    batch = MeshBatch.from_meshes(S)
    singles = [MeshBVH.from_mesh(dev(V), dev(F)) if len(F) else None for V, F in S]
    return S, batch, singles


def test_batched_trees_equal_single_builds(batch_and_singles):
    S, batch, singles = batch_and_singles
    A = batch.arrays()
    fo = host(batch.face_off)
    for s, (V, F) in enumerate(S):
        if len(F) == 0:
            continue
        a, b = fo[s], fo[s + 1]
        single = singles[s].arrays()
        assert np.array_equal(host(A["keys"])[a:b], host(single["keys"]))
        assert np.array_equal(host(A["perm"])[a:b] - a, host(single["perm"]))
        n = b - a
        if n > 1:
            assert np.array_equal(host(A["nodes_i"])[a:a + n - 1], host(single["nodes_i"]))
            assert np.array_equal(host(A["nodes"])[a:a + n - 1, :, :3], host(single["nodes"])[:, :, :3])
        tris = host(A["tris"])[a:b]
        st = host(single["tris"])
        assert np.array_equal(tris[:, :, :3], st[:, :, :3])
        assert np.array_equal(host(A["scene_box"])[s], host(single["root"]))
    assert batch.status()[0] == 0


def test_batched_queries_and_gaussians_equal_single(batch_and_singles):
    S, batch, singles = batch_and_singles
    rng = np.random.default_rng(3)
    Qs, G_face, G_bary, counts, gcounts = [], [], [], [], []
    for V, F in S:
        nq = int(rng.integers(0, 700))
        lo, hi = V.min(0) - 0.3, V.max(0) + 0.3
        Qs.append(uniform_box(nq, lo, hi, seed=nq))
        counts.append(nq)
        ng = len(F) and int(rng.integers(1, 900))
        G_face.append(rng.integers(0, max(len(F), 1), ng).astype(np.int32))
        G_bary.append(osada_barycentrics(rng, ng).astype(np.float32))
        gcounts.append(ng)
    Q = np.concatenate(Qs)
    qoff = dev(np.concatenate([[0], np.cumsum(counts)]).astype(np.int32))
    from paper_2606_00444_gb300 import set_query_group
    set_query_group(1)                        # the batched kernel is one thread per query
    try:
        _compare_queries(S, singles, batch, Q, Qs, qoff)
    finally:
        set_query_group(0)
    _compare_gaussians(S, singles, batch, G_face, G_bary, gcounts)
    # one scene against the oracle directly
    s = 1
    a, b = host(qoff)[s], host(qoff)[s + 1]
    sub = batch.closest_point(dev(Q), qoff)
    check_closest(S[s][0], S[s][1], Qs[s], {k: v[a:b] for k, v in sub.items()})


def _compare_queries(S, singles, batch, Q, Qs, qoff):
    for cut in (np.inf, 0.05):
        out = batch.closest_point(dev(Q), qoff, max_dist=cut)
        qo = host(qoff)
        for s, (V, F) in enumerate(S):
            a, b = qo[s], qo[s + 1]
            if b == a:
                continue
            if len(F) == 0:
                assert (host(out["face"])[a:b] == -1).all()
                continue
            ref = singles[s].closest_point(dev(Qs[s]), max_dist=cut)
            for k in ("face", "dist2", "bary", "point"):
                assert torch.equal(out[k][a:b], ref[k]), (s, k)


def _compare_gaussians(S, singles, batch, G_face, G_bary, gcounts):
    gf, gb = np.concatenate(G_face), np.concatenate(G_bary)
    goff = dev(np.concatenate([[0], np.cumsum(gcounts)]).astype(np.int32))
    mu, quat, scale = batch.bind_gaussians(dev(gf), goff, dev(gb))
    go = host(goff)
    for s, (V, F) in enumerate(S):
        a, b = go[s], go[s + 1]
        if b == a:
            continue
        rmu, rq, rs = singles[s].bind_gaussians(dev(G_face[s]), dev(G_bary[s]))
        assert torch.equal(mu[a:b], rmu) and torch.equal(quat[a:b], rq) and torch.equal(scale[a:b], rs)
        if s == 4:
            check_gaussians((mu[a:b], quat[a:b], scale[a:b]),
                            oracle.bind_gaussians(V, F, G_face[s], G_bary[s]))


def test_batched_refit_equals_single_refit():
    S = [displaced_icosphere(3, 0.1, 0.3), torus(60, 40), icosphere(4)]
    batch = MeshBatch.from_meshes(S)
    singles = [MeshBVH.from_mesh(dev(V), dev(F)) for V, F in S]
    moved = [(V * np.float32(1.1) + np.float32(0.05), F) for V, F in S]
    Vall, _, _, _ = MeshBatch.concat(moved)
    batch.refit(Vall)
    for sg, (V, _) in zip(singles, moved):
        sg.refit(dev(V))
    A = batch.arrays()
    fo = host(batch.face_off)
    for s in range(len(S)):
        a, b = fo[s], fo[s + 1]
        assert np.array_equal(host(A["nodes"])[a:b - 1, :, :3],
                              host(singles[s].arrays()["nodes"])[:, :, :3])
