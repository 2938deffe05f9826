"""Topology conversion of a varying-topology sequence (Sec. 3.3).

Strategy 1, temporal correspondence tracking (Eq. 1): the template's vertices
are carried from frame to frame by the k-NN weighted surface projection onto
the next frame (mesh_knn_project), and every `reanchor_every` frames the
result is mixed `keep` : 1 - `keep` with the direct projection of the template
onto that frame (mesh_closest_point, Eq. 2) -- the paper's 80 % / 20 % every
50 frames.  Strategy 2, template projection (Eq. 2), is one closest-point call
per frame and needs no state.  Each frame's target is rebuilt (its topology
changes); all arithmetic runs in the library's kernels, this module only
sequences the calls.
"""
from __future__ import annotations

import torch

from .api import MeshBVH


class TemporalTracker:
    def __init__(self, V0: torch.Tensor, max_verts: int, max_faces: int, k: int = 4,
                 reanchor_every: int = 50, keep: float = 0.8):
        if V0.dtype != torch.float32 or V0.dim() != 2 or V0.shape[1] != 3 or not V0.is_cuda:
            raise ValueError("V0 must be a CUDA float32 tensor [n, 3]")
        self.V0 = V0.contiguous()
        self.tracked = self.V0.clone()
        self.anchor = torch.empty_like(self.V0)
        self.target = MeshBVH(max_verts, max_faces, V0.device)
        self.k, self.reanchor_every, self.keep = int(k), int(reanchor_every), float(keep)
        self.t = 0

    def step(self, V: torch.Tensor, F: torch.Tensor) -> torch.Tensor:
        """Advance to the next frame (V, F); returns the tracked template vertices."""
        self.t += 1
        self.target.build(V, F)
        if self.reanchor_every > 0 and self.t % self.reanchor_every == 0:
            self.target.closest_point(self.V0, want=("point",), out={"point": self.anchor})
            self.target.knn_project(self.tracked, self.k, anchor=self.anchor,
                                    anchor_weight=1.0 - self.keep, out=self.tracked)
        else:
            self.target.knn_project(self.tracked, self.k, out=self.tracked)
        return self.tracked


def project_template(target: MeshBVH, V0: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """Strategy 2 (Eq. 2): the template's vertices projected onto the target's surface."""
    out = torch.empty_like(V0) if out is None else out
    target.closest_point(V0, want=("point",), out={"point": out})
    return out
