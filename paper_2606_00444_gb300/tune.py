"""Autotuner for the closest-point and Chamfer traversals.

The best traversal depends on the workload: how many queries there are
(whether one thread per query fills the GPU), whether a cutoff bounds the
search, and the mesh.  `tune_closest_point` times every candidate -- the leaf
size of the tree (1, 2, 4, 8 faces per collapsed leaf), lanes per query (1, 2,
4, ..., 32) and, for one lane, the fourteen traversal variants of
mesh_set_traversal, the main ones also in blocks of 32 and 64 threads -- on
the caller's own BVH and queries with CUDA events, keeps the fastest, and
applies it (a new leaf size takes a refit of the tree from its current
vertices; the answers do not depend on any of these choices).  `tune_chamfer` does the same for the
lanes of the Chamfer kernel.  Results are cached in memory, and in a JSON file
when MESHGS_TUNE_CACHE names one, keyed by device, mesh size class, query
count class and cutoff kind, so a workload is tuned once.
"""
from __future__ import annotations

import json
import math
import os

import torch

from .api import MeshBVH, chamfer, set_query_group, set_traversal

_CACHE: dict = {}


def _cache_path():
    return os.environ.get("MESHGS_TUNE_CACHE")


def _load():
    p = _cache_path()
    if p and os.path.exists(p) and not _CACHE:
        try:
            _CACHE.update(json.load(open(p)))
        except (OSError, ValueError):
            pass


def _save():
    p = _cache_path()
    if p:
        os.makedirs(os.path.dirname(os.path.abspath(p)), exist_ok=True)
        tmp = p + ".tmp"
        json.dump(_CACHE, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, p)


def _bucket(n: int) -> int:
    return 0 if n <= 0 else int(round(math.log2(n)))


def _key(kind: str, n_faces: int, n_queries: int, bounded: bool) -> str:
    name = torch.cuda.get_device_name()
    return f"{kind}|{name}|F2^{_bucket(n_faces)}|Q2^{_bucket(n_queries)}|{'cut' if bounded else 'inf'}"


def _time(fn, repeats: int) -> float:
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def _pick(results: list) -> dict:
    """The fastest candidate, with hysteresis: in candidate order, a candidate replaces the
    best so far only if it is more than 2 % faster, so that near-equal candidates resolve
    the same way from run to run."""
    best = results[0]
    for r in results[1:]:
        if r["ms"] < 0.98 * best["ms"]:
            best = r
    return best


LEAF_SIZES = (1, 2, 4, 8)


def _apply(bvh: MeshBVH, cfg: dict) -> None:
    if cfg.get("leaf", 1) != getattr(bvh, "leaf_size", 1):
        bvh.set_leaf_size(cfg.get("leaf", 1))          # refits from the current vertices
    bvh.set_query_config(cfg["lanes"], cfg["variant"], cfg.get("block", 128))


def closest_point_candidates(leaf_sizes=LEAF_SIZES):
    out = []
    for L in leaf_sizes:
        out += [dict(leaf=L, lanes=1, variant=v, block=128) for v in range(14)]
        out += [dict(leaf=L, lanes=1, variant=v, block=b) for v in (0, 2, 3, 13) for b in (32, 64)]
        out += [dict(leaf=L, lanes=g, variant=0, block=128) for g in (2, 4, 8, 16, 32)]
    return out


def _label(r: dict) -> str:
    return f"L{r.get('leaf', 1)}/{r['lanes']}/{r['variant']}/b{r.get('block', 128)}"


def tune_closest_point(bvh: MeshBVH, Q: torch.Tensor, max_dist: float = math.inf,
                       repeats: int = 5, force: bool = False, leaf_sizes=LEAF_SIZES) -> dict:
    """Time every candidate on (bvh, Q, max_dist); set the fastest on this handle (its leaf
    size too: the tree is refit from its current vertex buffer)."""
    _load()
    key = _key("closest_point", bvh.n_faces, Q.shape[0], math.isfinite(max_dist))
    if key in _CACHE and not force:
        _apply(bvh, _CACHE[key])
        return _CACHE[key]
    out = bvh.closest_point(Q, max_dist)
    results = []
    for cfg in closest_point_candidates(leaf_sizes):
        _apply(bvh, cfg)
        ms = _time(lambda: bvh.closest_point(Q, max_dist, out=out), repeats)
        results.append(dict(cfg, ms=ms))
    best = _pick(results)
    best = dict(leaf=best["leaf"], lanes=best["lanes"], variant=best["variant"], block=best["block"],
                ms=best["ms"], tried={_label(r): round(r["ms"], 4) for r in results})
    _CACHE[key] = best
    _save()
    _apply(bvh, best)
    return best


def tune_contact(bvh: MeshBVH, Q: torch.Tensor, max_dist: float, frames=None, repeats: int = 4,
                 force: bool = False, leaf_sizes=LEAF_SIZES) -> dict:
    """Tune the physics step's contact query itself (mesh_contact: warm-started from the
    previous step's faces, run in the order of its work classes) rather than the plain
    query.  `frames`: vertex buffers the timed steps cycle through (refit before each
    step, the same for every candidate), so the warm start meets moving geometry as in a
    simulation; None = the current pose.  Sets the fastest on this handle."""
    from .api import Workspace
    _load()
    key = _key("contact", bvh.n_faces, Q.shape[0], True)
    if key in _CACHE and not force:
        _apply(bvh, _CACHE[key])
        return _CACHE[key]
    n = Q.shape[0]
    dev = Q.device
    out = dict(face=torch.full((n,), -1, dtype=torch.int32, device=dev),
               bary=torch.empty(n, 3, device=dev), point=torch.empty(n, 3, device=dev),
               dist2=torch.empty(n, device=dev))
    frames = list(frames) if frames else [None]
    results = []
    for cfg in closest_point_candidates(leaf_sizes):
        if cfg["lanes"] > 1 and n >= (1 << 18):
            continue                                   # many queries: one thread per query
        _apply(bvh, cfg)
        ws = Workspace(dev)
        out["face"].fill_(-1)
        k = [0]

        def step():
            V = frames[k[0] % len(frames)]
            k[0] += 1
            if V is not None:
                bvh.refit(V)
            bvh.contact(Q, max_dist, out, ws=ws)

        for _ in range(2):                             # classes and hints from a real step
            step()
        ms = _time(step, repeats)
        results.append(dict(cfg, ms=ms))
    best = _pick(results)
    best = dict(leaf=best["leaf"], lanes=best["lanes"], variant=best["variant"], block=best["block"],
                ms=best["ms"], tried={_label(r): round(r["ms"], 4) for r in results})
    _CACHE[key] = best
    _save()
    _apply(bvh, best)
    if frames[0] is not None:
        bvh.refit(frames[0])
    return best


def tune_chamfer(A: MeshBVH, SA: torch.Tensor, B: MeshBVH, SB: torch.Tensor, repeats: int = 5,
                 force: bool = False, step: bool = False) -> dict:
    """Pick the lanes per query of the Chamfer kernel (process-wide setting), timing
    chamfer() or, with step=True, chamfer_step() (the ordered, warm-started form of a
    sequence: each candidate times its own warmed-up state)."""
    from .api import Workspace, chamfer_step
    _load()
    key = _key("chamfer_step" if step else "chamfer", A.n_faces + B.n_faces, SA.shape[0] + SB.shape[0], False)
    if key in _CACHE and not force:
        set_query_group(_CACHE[key]["lanes"])
        return _CACHE[key]
    res = torch.empty(2, dtype=torch.float64, device=SA.device)
    results = []
    for g in (1, 2, 4, 8, 16, 32):
        set_query_group(g)
        if step:
            dev = SA.device
            ps = dict(faceA=torch.full((SA.shape[0],), -1, dtype=torch.int32, device=dev),
                      faceB=torch.full((SB.shape[0],), -1, dtype=torch.int32, device=dev))
            ws = Workspace(dev)
            chamfer_step(A, SA, B, SB, ps, ws, out=res)           # faces and costs of this state
            fn = lambda: chamfer_step(A, SA, B, SB, ps, ws, out=res)   # noqa: E731
        else:
            fn = lambda: chamfer(A, SA, B, SB, out=res)              # noqa: E731
        results.append(dict(lanes=g, ms=_time(fn, repeats)))
    best = _pick(results)
    best = dict(lanes=best["lanes"], variant=0, ms=best["ms"],
                tried={str(r["lanes"]): round(r["ms"], 4) for r in results})
    _CACHE[key] = best
    _save()
    set_query_group(best["lanes"])
    return best


def reset(*bvhs: MeshBVH) -> None:
    """Back to the defaults (lanes from the query count, depth-first traversal, blocks of
    128 threads, leaf size 1)."""
    set_query_group(0)
    set_traversal(0)
    for b in bvhs:
        b.set_query_config(-1, -1, 128)
        if getattr(b, "leaf_size", 1) != 1:
            b.set_leaf_size(1)
