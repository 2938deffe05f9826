"""torch.autograd.Function wrappers over the meshgs forward and backward kernels.

Each forward makes the BVH's vertex buffer equal to the vertex tensor it is
given (and refits the boxes where a traversal follows), so a gradient always
refers to the geometry the forward saw.  Backward passes run the library's
hand-written gradient kernels; nothing is differentiated by PyTorch itself.
"""
from __future__ import annotations

import math

import torch

from .api import MeshBVH, Workspace, chamfer, chamfer_backward, chamfer_step


def chamfer_state(nA: int, nB: int, device="cuda") -> dict:
    """State for Chamfer.apply over a sequence of steps on the same samples (an
    optimisation, a simulation): the per-sample faces (-1 = none yet) and the
    workspace of mesh_chamfer_step that carries the samples' costs to the next step."""
    dev = torch.device(device)
    ps = dict(faceA=torch.full((nA,), -1, dtype=torch.int32, device=dev), baryA=torch.empty(nA, 3, device=dev),
              faceB=torch.full((nB,), -1, dtype=torch.int32, device=dev), baryB=torch.empty(nB, 3, device=dev))
    return dict(ps=ps, ws=Workspace(dev))


class PointMeshDistance(torch.autograd.Function):
    """dist2[i] = squared distance from Q[i] to the mesh (V, topology of bvh).

    Returns (dist2, face); face is not differentiable (-1 beyond max_dist,
    where dist2 is +inf and the gradient is 0).
    """

    @staticmethod
    def forward(ctx, Q, V, bvh: MeshBVH, max_dist=math.inf):
        bvh.refit(V.detach())
        out = bvh.closest_point(Q.detach(), max_dist, want=("face", "bary", "dist2"))
        ctx.save_for_backward(Q.detach(), V.detach(), out["face"], out["bary"])
        ctx.bvh = bvh
        ctx.mark_non_differentiable(out["face"])
        return out["dist2"], out["face"]

    @staticmethod
    def backward(ctx, g, _gface):
        Q, V, face, bary = ctx.saved_tensors
        bvh = ctx.bvh
        bvh.update_vertices(V)
        gQ = torch.empty_like(Q) if ctx.needs_input_grad[0] else None
        gV = torch.zeros_like(V) if ctx.needs_input_grad[1] else None
        if gQ is not None or gV is not None:
            bvh.closest_point_backward(Q, face, bary, g.float().contiguous(), gQ, gV)
        return gQ, gV, None, None


class Interpolate(torch.autograd.Function):
    """Points sum_j bary[i, j] V[F[face[i], j]] on the mesh held by bvh."""

    @staticmethod
    def forward(ctx, V, bvh: MeshBVH, face, bary):
        bvh.update_vertices(V.detach())
        P = bvh.interpolate(face, bary)
        ctx.save_for_backward(face, bary)
        ctx.bvh, ctx.nV = bvh, V.shape[0]
        return P

    @staticmethod
    def backward(ctx, gP):
        face, bary = ctx.saved_tensors
        gV = torch.zeros(ctx.nV, 3, device=gP.device, dtype=torch.float32)
        ctx.bvh.interpolate_backward(face, bary, gP.float().contiguous(), gV)
        return gV, None, None, None


class Chamfer(torch.autograd.Function):
    """[mean_a d(a, B)^2, mean_b d(b, A)^2] for samples SA / SB and meshes (VA, bvhA),
    (VB, bvhB); differentiable in SA, VA, SB and VB.  With `state` (chamfer_state) the
    forward is the step of a sequence (mesh_chamfer_step: warm-started from the previous
    step's faces, samples heaviest first): the same per-sample faces and weights, hence
    the same gradients (up to the order of the backward's float atomic sums)."""

    @staticmethod
    def forward(ctx, SA, VA, bvhA: MeshBVH, SB, VB, bvhB: MeshBVH, state=None):
        bvhA.refit(VA.detach())
        bvhB.refit(VB.detach())
        if state is None:
            out, ps = chamfer(bvhA, SA.detach(), bvhB, SB.detach(), per_sample=True)
        else:
            out = chamfer_step(bvhA, SA.detach(), bvhB, SB.detach(), state["ps"], state["ws"])
            ps = {k: v.clone() for k, v in state["ps"].items()}   # the next step rewrites the state
        ctx.save_for_backward(SA.detach(), VA.detach(), SB.detach(), VB.detach(), ps["faceA"],
                              ps["baryA"], ps["faceB"], ps["baryB"])
        ctx.bvhA, ctx.bvhB = bvhA, bvhB
        return out

    @staticmethod
    def backward(ctx, g):
        SA, VA, SB, VB, faceA, baryA, faceB, baryB = ctx.saved_tensors
        bvhA, bvhB = ctx.bvhA, ctx.bvhB
        need = ctx.needs_input_grad
        gSA = torch.empty_like(SA) if need[0] else None
        gVA = torch.zeros_like(VA) if need[1] else None
        gSB = torch.empty_like(SB) if need[3] else None
        gVB = torch.zeros_like(VB) if need[4] else None
        bvhA.update_vertices(VA)
        bvhB.update_vertices(VB)
        chamfer_backward(bvhA, SA, bvhB, SB, g.detach().to(torch.float64).contiguous(),
                         dict(faceA=faceA, baryA=baryA, faceB=faceB, baryB=baryB),
                         gSA, gVA, gSB, gVB)
        return gSA, gVA, None, gSB, gVB, None, None


class BindGaussians(torch.autograd.Function):
    """(mu, quat, scale) of face-bound Gaussians on the mesh (V, topology of bvh)."""

    @staticmethod
    def forward(ctx, V, bvh: MeshBVH, gface, gbary, goff=None):
        bvh.update_vertices(V.detach())
        mu, quat, scale = bvh.bind_gaussians(gface, gbary, goff)
        ctx.save_for_backward(V.detach(), gface, gbary, goff if goff is not None else gbary[:0])
        ctx.bvh, ctx.has_off = bvh, goff is not None
        return mu, quat, scale

    @staticmethod
    def backward(ctx, gmu, gquat, gscale):
        V, gface, gbary, goff = ctx.saved_tensors
        bvh = ctx.bvh
        bvh.update_vertices(V)
        gV = torch.zeros_like(V)
        bvh.bind_gaussians_backward(gface, gbary, goff if ctx.has_off else None, gmu, gquat,
                                    gscale, gV)
        return gV, None, None, None, None
