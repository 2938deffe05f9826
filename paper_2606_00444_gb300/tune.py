"""Autotuner for the closest-point and Chamfer traversals.

The best traversal depends on the workload: how many queries there are
(whether one thread per query fills the GPU), whether a cutoff bounds the
search, and the mesh.  `tune_closest_point` times every candidate -- lanes per
query (1, 2, 4, ..., 32) and, for one lane, the thirteen traversal variants of
mesh_set_traversal -- on the caller's own BVH and queries with CUDA events,
keeps the fastest, and applies it.  `tune_chamfer` does the same for the
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


def _apply(bvh: MeshBVH, cfg: dict) -> None:
    bvh.set_query_config(cfg["lanes"], cfg["variant"])


def closest_point_candidates():
    return [dict(lanes=1, variant=v) for v in range(13)] + \
           [dict(lanes=g, variant=0) for g in (2, 4, 8, 16, 32)]


def tune_closest_point(bvh: MeshBVH, Q: torch.Tensor, max_dist: float = math.inf,
                       repeats: int = 5, force: bool = False) -> dict:
    """Time every candidate on (bvh, Q, max_dist); set the fastest on this handle."""
    _load()
    key = _key("closest_point", bvh.n_faces, Q.shape[0], math.isfinite(max_dist))
    if key in _CACHE and not force:
        _apply(bvh, _CACHE[key])
        return _CACHE[key]
    out = bvh.closest_point(Q, max_dist)
    results = []
    for cfg in closest_point_candidates():
        _apply(bvh, cfg)
        ms = _time(lambda: bvh.closest_point(Q, max_dist, out=out), repeats)
        results.append(dict(cfg, ms=ms))
    best = _pick(results)
    best = dict(lanes=best["lanes"], variant=best["variant"], ms=best["ms"],
                tried={f"{r['lanes']}/{r['variant']}": round(r["ms"], 4) for r in results})
    _CACHE[key] = best
    _save()
    _apply(bvh, best)
    return best


def tune_chamfer(A: MeshBVH, SA: torch.Tensor, B: MeshBVH, SB: torch.Tensor, repeats: int = 5,
                 force: bool = False) -> dict:
    """Pick the lanes per query of the Chamfer kernel (process-wide setting)."""
    _load()
    key = _key("chamfer", A.n_faces + B.n_faces, SA.shape[0] + SB.shape[0], False)
    if key in _CACHE and not force:
        set_query_group(_CACHE[key]["lanes"])
        return _CACHE[key]
    res = torch.empty(2, dtype=torch.float64, device=SA.device)
    results = []
    for g in (1, 2, 4, 8, 16, 32):
        set_query_group(g)
        results.append(dict(lanes=g, ms=_time(lambda: chamfer(A, SA, B, SB, out=res), repeats)))
    best = _pick(results)
    best = dict(lanes=best["lanes"], variant=0, ms=best["ms"],
                tried={str(r["lanes"]): round(r["ms"], 4) for r in results})
    _CACHE[key] = best
    _save()
    set_query_group(best["lanes"])
    return best


def reset(*bvhs: MeshBVH) -> None:
    """Back to the defaults (lanes from the query count, depth-first traversal)."""
    set_query_group(0)
    set_traversal(0)
    for b in bvhs:
        b.set_query_config(-1, -1)
