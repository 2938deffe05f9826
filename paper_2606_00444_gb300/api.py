"""PyTorch-facing binding of the meshgs C ABI: argument marshalling only.

PyTorch provides device memory (storage, workspace, outputs) and the current
CUDA stream; every step of the update runs in the library's CUDA kernels.
Inputs must be CUDA tensors of the documented dtype and shape (float32 xyz
rows, int32 indices); they are made contiguous, never converted on the host.
"""
from __future__ import annotations

import ctypes as C
import math

import torch

from . import _abi
from ._abi import check, lib


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _io_ptr(t: torch.Tensor, name: str) -> int:
    """Device-accessible address of a CUDA tensor, or of a pinned host tensor (which a
    kernel then reads / writes in place over the host link)."""
    if t.is_cuda:
        return t.data_ptr()
    if t.is_pinned():
        d = C.c_void_p()
        check(lib().mesh_mapped_pointer(t.data_ptr(), C.byref(d)), "mesh_mapped_pointer")
        return d.value
    raise ValueError(f"{name} must be a CUDA tensor or a pinned host tensor")


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _f32(t: torch.Tensor, cols: int | None = None, name: str = "tensor") -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32, got {t.dtype}")
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"{name} must have shape [n, {cols}], got {tuple(t.shape)}")
    return t.contiguous()


def _i32(t: torch.Tensor, cols: int | None = None, name: str = "tensor") -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.int32:
        raise TypeError(f"{name} must be int32, got {t.dtype}")
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"{name} must have shape [n, {cols}], got {tuple(t.shape)}")
    return t.contiguous()


class Workspace:
    """A grow-only device scratch buffer (256-byte aligned torch allocation)."""

    def __init__(self, device):
        self.device = device
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.buf


class MeshBVH:
    """A triangle mesh with its LBVH, vertex buffer and face table in device storage.

    The same vertex buffer serves collision queries and the face-bound
    Gaussians (the paper's shared physics / rendering mesh).
    """

    def __init__(self, max_verts: int, max_faces: int, device="cuda"):
        self.device = torch.device(device)
        nbytes = lib().mesh_bvh_storage_bytes(max_verts, max_faces)
        if nbytes == 0:
            raise ValueError("mesh too large")
        self.storage = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        check(lib().mesh_bvh_create(self.storage.data_ptr(), nbytes, max_verts, max_faces,
                                    C.byref(h)), "mesh_bvh_create")
        self.handle = h
        self.max_verts, self.max_faces = max_verts, max_faces
        self._ws = Workspace(self.device)
        self._chamfer_ws = Workspace(self.device)
        self.n_verts = 0
        self.n_faces = 0
        self.leaf_size = 1

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().mesh_bvh_destroy(h)
            except Exception:
                pass
            self.handle = None

    @classmethod
    def from_mesh(cls, V: torch.Tensor, F: torch.Tensor, method: str = "lbvh") -> "MeshBVH":
        b = cls(V.shape[0], F.shape[0], V.device)
        b.build(V, F, method)
        return b

    # -- the update steps -------------------------------------------------
    def build(self, V: torch.Tensor, F: torch.Tensor, method: str = "lbvh") -> "MeshBVH":
        """Build the tree over (V, F).  "lbvh": Karras's radix tree (mesh_build_lbvh,
        asynchronous, the per-frame rebuild).  "ploc": agglomerative clustering
        (mesh_build_ploc, synchronous) -- a tree with fewer node visits per query, for
        a mesh built once and then refit."""
        V = _f32(V, 3, "V")
        F = _i32(F, 3, "F")
        if method == "lbvh":
            ws = self._ws.get(lib().mesh_build_workspace_bytes(F.shape[0]))
            check(lib().mesh_build_lbvh(self.handle, V.data_ptr(), V.shape[0], F.data_ptr(),
                                        F.shape[0], ws.data_ptr(), ws.numel(), _stream()),
                  "mesh_build_lbvh")
        elif method == "ploc":
            ws = self._ws.get(lib().mesh_build_ploc_workspace_bytes(F.shape[0]))
            check(lib().mesh_build_ploc(self.handle, V.data_ptr(), V.shape[0], F.data_ptr(),
                                        F.shape[0], ws.data_ptr(), ws.numel(), _stream()),
                  "mesh_build_ploc")
        else:
            raise ValueError(f"unknown build method {method!r}")
        self.n_verts, self.n_faces = V.shape[0], F.shape[0]
        return self

    def update_vertices(self, V: torch.Tensor) -> None:
        V = _f32(V, 3, "V")
        check(lib().mesh_update_vertices(self.handle, V.data_ptr(), V.shape[0], _stream()),
              "mesh_update_vertices")

    def refit(self, V: torch.Tensor | None = None) -> None:
        if V is not None:
            V = _f32(V, 3, "V")
        check(lib().mesh_refit(self.handle, _ptr(V), 0 if V is None else V.shape[0], _stream()),
              "mesh_refit")

    def refit_bind(self, V, gstart, gbary, goff=None, out=None):
        """refit(V) and bind_gaussians in one pass; the Gaussians of face f are
        gstart[f] .. gstart[f + 1] - 1 (int32 CSR over faces)."""
        if V is not None:
            V = _f32(V, 3, "V")
        gstart = _i32(gstart, None, "gstart")
        gbary = _f32(gbary, 3, "gbary")
        goff = None if goff is None else _f32(goff, None, "goff")
        nG = gbary.shape[0]
        if gstart.shape[0] != self.n_faces + 1:
            raise ValueError("gstart must have n_faces + 1 entries")
        if out is None:
            d = gbary.device
            out = (torch.empty(nG, 3, device=d), torch.empty(nG, 4, device=d), torch.empty(nG, 3, device=d))
        mu, quat, scale = out
        check(lib().mesh_refit_bind(self.handle, _ptr(V), 0 if V is None else V.shape[0], gstart.data_ptr(),
                                    gbary.data_ptr(), _ptr(goff), nG, mu.data_ptr(), quat.data_ptr(),
                                    scale.data_ptr(), _stream()), "mesh_refit_bind")
        return out

    def closest_point(self, Q: torch.Tensor, max_dist: float = math.inf, want=("face", "bary",
                      "point", "dist2"), out: dict | None = None,
                      hint: torch.Tensor | None = None) -> dict:
        """NearestSurface of every query.  `hint` (int32 face ids, -1 = none; may be
        out["face"] itself) warm-starts the search, e.g. with the previous frame's
        answers; the result is the one without it, bit for bit (the tie rule does not
        depend on the order in which faces are met; see mesh_closest_point)."""
        Q = _f32(Q, 3, "Q")
        n = Q.shape[0]
        if hint is not None:
            hint = _i32(hint, None, "hint")
            if hint.shape[0] != n:
                raise ValueError("hint must have one entry per query")
        out = {} if out is None else out
        if "face" in want and "face" not in out:
            out["face"] = torch.empty(n, dtype=torch.int32, device=Q.device)
        for k, c in (("bary", 3), ("point", 3)):
            if k in want and k not in out:
                out[k] = torch.empty(n, c, dtype=torch.float32, device=Q.device)
        if "dist2" in want and "dist2" not in out:
            out["dist2"] = torch.empty(n, dtype=torch.float32, device=Q.device)
        check(lib().mesh_closest_point_hinted(self.handle, Q.data_ptr(), n, float(max_dist), _ptr(hint),
                                              _ptr(out.get("face")), _ptr(out.get("bary")),
                                              _ptr(out.get("point")), _ptr(out.get("dist2")), _stream()),
              "mesh_closest_point")
        return out

    def knn_project(self, Q: torch.Tensor, k: int = 4, anchor: torch.Tensor | None = None,
                    anchor_weight: float = 0.2, out: torch.Tensor | None = None,
                    want_faces: bool = False):
        """k-NN weighted surface projection (mesh_knn_project); `out` may be Q itself."""
        Q = _f32(Q, 3, "Q")
        n = Q.shape[0]
        if anchor is not None:
            anchor = _f32(anchor, 3, "anchor")
            if anchor.shape[0] != n:
                raise ValueError("anchor must have one row per query")
        out = torch.empty_like(Q) if out is None else out
        face = torch.empty(n, k, dtype=torch.int32, device=Q.device) if want_faces else None
        d2 = torch.empty(n, k, device=Q.device) if want_faces else None
        check(lib().mesh_knn_project(self.handle, Q.data_ptr(), n, int(k), _ptr(anchor),
                                     float(anchor_weight if anchor is not None else 0.0), out.data_ptr(),
                                     _ptr(face), _ptr(d2), _stream()), "mesh_knn_project")
        return (out, face, d2) if want_faces else out

    def signed_distance(self, Q: torch.Tensor, max_dist: float = math.inf, out: dict | None = None) -> dict:
        """Signed NearestSurface distance (inside negative; mesh_signed_distance):
        dict(face, bary, point, sdist)."""
        Q = _f32(Q, 3, "Q")
        n = Q.shape[0]
        out = {} if out is None else out
        out.setdefault("face", torch.empty(n, dtype=torch.int32, device=Q.device))
        out.setdefault("bary", torch.empty(n, 3, device=Q.device))
        out.setdefault("point", torch.empty(n, 3, device=Q.device))
        out.setdefault("sdist", torch.empty(n, device=Q.device))
        ws = self._ws.get(lib().mesh_signed_workspace_bytes(max(self.n_faces, 1)))
        check(lib().mesh_signed_distance(self.handle, Q.data_ptr(), n, float(max_dist), ws.data_ptr(),
                                         ws.numel(), _ptr(out["face"]), _ptr(out["bary"]), _ptr(out["point"]),
                                         out["sdist"].data_ptr(), _stream()), "mesh_signed_distance")
        return out

    def contact(self, Q: torch.Tensor, max_dist: float, out: dict, ws: "Workspace | None" = None) -> dict:
        """Physics-step contact query (mesh_contact): out["face"] holds the previous
        step's faces on entry (-1 = none) and this step's on return.  The arrays of
        `out` (face, and optionally bary, point, dist2) may be CUDA tensors or pinned
        host tensors; the kernel writes pinned ones directly (mesh_mapped_pointer).
        `ws` carries the work classes that order the next step: pass the same one
        every step."""
        Q = _f32(Q, 3, "Q")
        n = Q.shape[0]
        shapes = dict(face=(torch.int32, (n,)), bary=(torch.float32, (n, 3)),
                      point=(torch.float32, (n, 3)), dist2=(torch.float32, (n,)))
        ptrs = {}
        for k, (dt, shape) in shapes.items():
            t = out.get(k)
            if t is None:
                if k == "face":
                    raise ValueError("out['face'] is required")
                ptrs[k] = None
                continue
            if t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"out[{k!r}] must be a contiguous {dt} tensor of shape {shape}")
            ptrs[k] = _io_ptr(t, k)
        ws = self._ws if ws is None else ws
        buf = ws.get(lib().mesh_contact_workspace_bytes(n))
        check(lib().mesh_contact(self.handle, Q.data_ptr(), n, float(max_dist), ptrs["face"], ptrs["bary"],
                                 ptrs["point"], ptrs["dist2"], buf.data_ptr(), buf.numel(), _stream()),
              "mesh_contact")
        return out

    def closest_point_stats(self, Q: torch.Tensor, max_dist: float = math.inf) -> dict:
        """Traversal work for these queries: node visits, triangle tests, hits (totals)."""
        Q = _f32(Q, 3, "Q")
        c = torch.zeros(3, dtype=torch.int64, device=Q.device)
        check(lib().mesh_closest_point_stats(self.handle, Q.data_ptr(), Q.shape[0], float(max_dist),
                                             c.data_ptr(), _stream()), "mesh_closest_point_stats")
        v = c.tolist()
        return dict(visits=v[0], tests=v[1], hits=v[2])

    def bind_gaussians(self, gface, gbary, goff=None, out=None):
        gface = _i32(gface, None, "gface")
        gbary = _f32(gbary, 3, "gbary")
        goff = None if goff is None else _f32(goff, None, "goff")
        n = gface.shape[0]
        if out is None:
            out = (torch.empty(n, 3, device=gface.device), torch.empty(n, 4, device=gface.device),
                   torch.empty(n, 3, device=gface.device))
        mu, quat, scale = out
        check(lib().mesh_bind_gaussians(self.handle, gface.data_ptr(), gbary.data_ptr(), _ptr(goff),
                                        n, mu.data_ptr(), quat.data_ptr(), scale.data_ptr(),
                                        _stream()), "mesh_bind_gaussians")
        return mu, quat, scale

    def interpolate(self, face, bary, out=None):
        face = _i32(face, None, "face")
        bary = _f32(bary, 3, "bary")
        out = torch.empty(face.shape[0], 3, device=face.device) if out is None else out
        check(lib().mesh_interpolate(self.handle, face.data_ptr(), bary.data_ptr(), face.shape[0],
                                     out.data_ptr(), _stream()), "mesh_interpolate")
        return out

    # -- gradients -------------------------------------------------------
    def closest_point_backward(self, Q, face, bary, g, gQ=None, gV=None):
        Q = _f32(Q, 3, "Q")
        check(lib().mesh_closest_point_backward(self.handle, Q.data_ptr(), Q.shape[0],
                                                _i32(face).data_ptr(), _f32(bary, 3).data_ptr(),
                                                _f32(g).data_ptr(), _ptr(gQ), _ptr(gV), _stream()),
              "mesh_closest_point_backward")

    def interpolate_backward(self, face, bary, gP, gV):
        check(lib().mesh_interpolate_backward(self.handle, _i32(face).data_ptr(),
                                              _f32(bary, 3).data_ptr(), face.shape[0],
                                              _f32(gP, 3).data_ptr(), gV.data_ptr(), _stream()),
              "mesh_interpolate_backward")

    def bind_gaussians_backward(self, gface, gbary, goff, gmu, gquat, gscale, gV):
        gface = _i32(gface)
        check(lib().mesh_bind_gaussians_backward(
            self.handle, gface.data_ptr(), _f32(gbary, 3).data_ptr(),
            _ptr(None if goff is None else _f32(goff)), gface.shape[0],
            _ptr(None if gmu is None else _f32(gmu, 3)),
            _ptr(None if gquat is None else _f32(gquat, 4)),
            _ptr(None if gscale is None else _f32(gscale, 3)), gV.data_ptr(), _stream()),
            "mesh_bind_gaussians_backward")

    def set_query_config(self, lanes: int = -1, variant: int = -1, block: int | None = None) -> None:
        """Traversal choice for this handle's closest-point calls (-1 = process-wide);
        `block`: threads per block of the one-thread variants 0, 2, 3 (32, 64, 128)."""
        check(lib().mesh_bvh_set_query_config(self.handle, int(lanes), int(variant)),
              "mesh_bvh_set_query_config")
        if block is not None:
            check(lib().mesh_bvh_set_query_block(self.handle, int(block)), "mesh_bvh_set_query_block")

    def set_leaf_size(self, leaf_size: int, refit: bool = True) -> None:
        """Leaf collapse at `leaf_size` faces (mesh_bvh_set_leaf_size); with refit=True the
        tree is refit from its current vertex buffer at once so the new links apply."""
        check(lib().mesh_bvh_set_leaf_size(self.handle, int(leaf_size)), "mesh_bvh_set_leaf_size")
        self.leaf_size = int(leaf_size)
        if refit and self.n_faces > 0:
            self.refit()

    # -- inspection -----------------------------------------------------
    def status(self) -> tuple[int, int]:
        bits = C.c_uint32()
        ndeg = C.c_uint32()
        st = lib().mesh_bvh_status(self.handle, C.byref(bits), C.byref(ndeg), _stream())
        if st not in (_abi.MESH_OK, _abi.MESH_ERR_DEVICE):
            check(st, "mesh_bvh_status")
        return bits.value, ndeg.value

    def layout(self) -> dict:
        L = _abi.Layout()
        check(lib().mesh_bvh_get_layout(self.handle, C.byref(L)), "mesh_bvh_get_layout")
        return {k: getattr(L, k) for k, _ in _abi.Layout._fields_}

    def arrays(self) -> dict:
        """Views of the device arrays (see mesh_bvh_layout in include/meshgs.h)."""
        L = self.layout()
        n, nv = L["n_faces"], L["n_verts"]
        s = self.storage

        def view(off, count, dtype, shape):
            nbytes = count * torch.tensor([], dtype=dtype).element_size()
            return s[off:off + nbytes].view(dtype).reshape(shape)

        out = dict(
            root=view(L["off_header"], 8, torch.float32, (2, 4))[:, :3],
            verts=view(L["off_verts"], 4 * nv, torch.float32, (nv, 4)),
            faces=view(L["off_faces"], 4 * n, torch.int32, (n, 4)),
            keys=view(L["off_keys"], n, torch.int32, (n,)),
            perm=view(L["off_perm"], n, torch.int32, (n,)),
            parent=view(L["off_parent"], max(2 * n - 1, 0), torch.int32, (max(2 * n - 1, 0),)),
            tris=view(L["off_tris"], 12 * n, torch.float32, (n, 3, 4)),
            header=view(L["off_header"], 10, torch.int32, (10,)),     # root box, status, degenerate count
        )
        m = max(n - 1, 0)
        out["nodes"] = view(L["off_nodes"], 16 * m, torch.float32, (m, 4, 4))
        out["nodes_i"] = view(L["off_nodes"], 16 * m, torch.int32, (m, 4, 4))
        return out


def _offsets(counts, device) -> torch.Tensor:
    off = [0]
    for c in counts:
        off.append(off[-1] + int(c))
    return torch.tensor(off, dtype=torch.int32, device=device)


class MeshBatch:
    """Many independent meshes (scenes) in one storage block, each with its own LBVH.

    Vertices / faces are concatenated with int32 CSR offsets; faces hold
    scene-local vertex indices.  Every phase of the build, the queries and the
    Gaussian update run as single launches over all scenes.
    """

    def __init__(self, max_scenes: int, max_verts: int, max_faces: int, device="cuda"):
        self.device = torch.device(device)
        nbytes = lib().mesh_batch_storage_bytes(max_scenes, max_verts, max_faces)
        if nbytes == 0:
            raise ValueError("batch too large")
        self.storage = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        check(lib().mesh_batch_create(self.storage.data_ptr(), nbytes, max_scenes, max_verts,
                                      max_faces, C.byref(h)), "mesh_batch_create")
        self.handle = h
        self._ws = Workspace(self.device)
        self.vert_off = self.face_off = None

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().mesh_batch_destroy(h)
            except Exception:
                pass
            self.handle = None

    @staticmethod
    def concat(meshes, device="cuda"):
        """(V [sum V, 3], vert_off, F [sum F, 3] scene-local, face_off) from [(V_s, F_s)]."""
        V = torch.cat([torch.as_tensor(v, dtype=torch.float32) for v, _ in meshes]).to(device)
        F = torch.cat([torch.as_tensor(f, dtype=torch.int32) for _, f in meshes]).to(device)
        return (V.contiguous(), _offsets([len(v) for v, _ in meshes], device), F.contiguous(),
                _offsets([len(f) for _, f in meshes], device))

    @classmethod
    def from_meshes(cls, meshes, device="cuda") -> "MeshBatch":
        V, vo, F, fo = cls.concat(meshes, device)
        b = cls(len(meshes), V.shape[0], F.shape[0], device)
        b.build(V, vo, F, fo)
        return b

    def build(self, V, vert_off, F, face_off):
        V = _f32(V, 3, "V")
        F = _i32(F, 3, "F")
        vert_off, face_off = _i32(vert_off, None, "vert_off"), _i32(face_off, None, "face_off")
        B = face_off.shape[0] - 1
        ws = self._ws.get(lib().mesh_batch_workspace_bytes(B, F.shape[0]))
        check(lib().mesh_batch_build(self.handle, B, V.data_ptr(), vert_off.data_ptr(), V.shape[0],
                                     F.data_ptr(), face_off.data_ptr(), F.shape[0], ws.data_ptr(),
                                     ws.numel(), _stream()), "mesh_batch_build")
        self.vert_off, self.face_off = vert_off, face_off
        return self

    def refit(self, V=None):
        if V is not None:
            V = _f32(V, 3, "V")
        check(lib().mesh_batch_refit(self.handle, _ptr(V), 0 if V is None else V.shape[0],
                                     _stream()), "mesh_batch_refit")

    def closest_point(self, Q, query_off, max_dist=math.inf, want=("face", "bary", "point", "dist2"),
                      out=None):
        Q = _f32(Q, 3, "Q")
        query_off = _i32(query_off, None, "query_off")
        n = Q.shape[0]
        out = {} if out is None else out
        if "face" in want and "face" not in out:
            out["face"] = torch.empty(n, dtype=torch.int32, device=Q.device)
        for k in ("bary", "point"):
            if k in want and k not in out:
                out[k] = torch.empty(n, 3, device=Q.device)
        if "dist2" in want and "dist2" not in out:
            out["dist2"] = torch.empty(n, device=Q.device)
        check(lib().mesh_batch_closest_point(self.handle, Q.data_ptr(), query_off.data_ptr(), n,
                                             float(max_dist), _ptr(out.get("face")),
                                             _ptr(out.get("bary")), _ptr(out.get("point")),
                                             _ptr(out.get("dist2")), _stream()),
              "mesh_batch_closest_point")
        return out

    def bind_gaussians(self, gface, gauss_off, gbary, goff=None, out=None):
        gface = _i32(gface, None, "gface")
        gauss_off = _i32(gauss_off, None, "gauss_off")
        gbary = _f32(gbary, 3, "gbary")
        n = gface.shape[0]
        if out is None:
            out = (torch.empty(n, 3, device=gface.device), torch.empty(n, 4, device=gface.device),
                   torch.empty(n, 3, device=gface.device))
        mu, quat, scale = out
        check(lib().mesh_batch_bind_gaussians(self.handle, gface.data_ptr(), gauss_off.data_ptr(),
                                              gbary.data_ptr(),
                                              _ptr(None if goff is None else _f32(goff)), n,
                                              mu.data_ptr(), quat.data_ptr(), scale.data_ptr(),
                                              _stream()), "mesh_batch_bind_gaussians")
        return mu, quat, scale

    def status(self):
        bits, ndeg = C.c_uint32(), C.c_uint32()
        st = lib().mesh_batch_status(self.handle, C.byref(bits), C.byref(ndeg), _stream())
        if st not in (_abi.MESH_OK, _abi.MESH_ERR_DEVICE):
            check(st, "mesh_batch_status")
        return bits.value, ndeg.value

    def layout(self) -> dict:
        L = _abi.BatchLayout()
        check(lib().mesh_batch_get_layout(self.handle, C.byref(L)), "mesh_batch_get_layout")
        return {k: getattr(L, k) for k, _ in _abi.BatchLayout._fields_}

    def arrays(self) -> dict:
        L = self.layout()
        n, B = L["n_faces"], L["n_scenes"]
        s = self.storage

        def view(off, count, dtype, shape):
            nbytes = count * torch.tensor([], dtype=dtype).element_size()
            return s[off:off + nbytes].view(dtype).reshape(shape)

        return dict(
            scene_box=view(L["off_scene"], 8 * B, torch.float32, (B, 2, 4))[:, :, :3],
            keys=view(L["off_keys"], n, torch.int32, (n,)),
            perm=view(L["off_perm"], n, torch.int32, (n,)),
            nodes=view(L["off_nodes"], 16 * n, torch.float32, (n, 4, 4)),
            nodes_i=view(L["off_nodes"], 16 * n, torch.int32, (n, 4, 4)),
            parent_int=view(L["off_parent_int"], n, torch.int32, (n,)),
            parent_leaf=view(L["off_parent_leaf"], n, torch.int32, (n,)),
            tris=view(L["off_tris"], 12 * n, torch.float32, (n, 3, 4)),
        )


def chamfer(A: MeshBVH, SA: torch.Tensor, B: MeshBVH, SB: torch.Tensor, per_sample=False,
            ws: Workspace | None = None, out: torch.Tensor | None = None, ps: dict | None = None,
            hints=None):
    """[mean d(SA, B)^2, mean d(SB, A)^2] (float64) and optional per-sample results.

    `ps` reuses per-sample output arrays (faceA, baryA, dist2A, faceB, baryB, dist2B);
    `hints` = (faces of B for SA, faces of A for SB), int32 (-1 = none, either may be
    None, and each may be the matching face output itself), warm-starts the searches,
    e.g. with the previous frame's answers; the results are those without them, bit
    for bit."""
    SA = _f32(SA, 3, "SA")
    SB = _f32(SB, 3, "SB")
    nA, nB = SA.shape[0], SB.shape[0]
    ws = A._chamfer_ws if ws is None else ws
    buf = ws.get(lib().mesh_chamfer_workspace_bytes(nA, nB))
    out = torch.empty(2, dtype=torch.float64, device=SA.device) if out is None else out
    if per_sample and ps is None:
        dev = SA.device
        ps = dict(faceA=torch.empty(nA, dtype=torch.int32, device=dev),
                  baryA=torch.empty(nA, 3, device=dev), dist2A=torch.empty(nA, device=dev),
                  faceB=torch.empty(nB, dtype=torch.int32, device=dev),
                  baryB=torch.empty(nB, 3, device=dev), dist2B=torch.empty(nB, device=dev))
    ps = {} if ps is None else ps
    hA, hB = (None, None) if hints is None else hints
    if hA is not None:
        hA = _i32(hA, None, "hints[0]")
        if hA.shape[0] != nA:
            raise ValueError("hints[0] must have one entry per sample of SA")
    if hB is not None:
        hB = _i32(hB, None, "hints[1]")
        if hB.shape[0] != nB:
            raise ValueError("hints[1] must have one entry per sample of SB")
    check(lib().mesh_chamfer_hinted(A.handle, SA.data_ptr(), nA, B.handle, SB.data_ptr(), nB,
                                    buf.data_ptr(), buf.numel(), out.data_ptr(), _ptr(hA), _ptr(hB),
                                    _ptr(ps.get("faceA")), _ptr(ps.get("baryA")), _ptr(ps.get("dist2A")),
                                    _ptr(ps.get("faceB")), _ptr(ps.get("baryB")), _ptr(ps.get("dist2B")),
                                    _stream()), "mesh_chamfer")
    return (out, ps) if per_sample else out


def chamfer_step(A: MeshBVH, SA: torch.Tensor, B: MeshBVH, SB: torch.Tensor, ps: dict, ws: Workspace,
                 out: torch.Tensor | None = None) -> torch.Tensor:
    """chamfer() for a sequence of frames on the same samples (mesh_chamfer_step):
    ps["faceA"] / ps["faceB"] (int32, required) hold the previous call's faces on entry
    (-1 = none; warm start) and this call's on return, the other entries of ps
    (baryA, dist2A, baryB, dist2B) are optional outputs, and each side's samples run
    heaviest first by the costs the previous call left in `ws` (pass the same
    Workspace every call).  Per-sample results equal chamfer()'s bit for bit; the two
    means equal it up to the order of the float64 sums."""
    SA = _f32(SA, 3, "SA")
    SB = _f32(SB, 3, "SB")
    nA, nB = SA.shape[0], SB.shape[0]
    shapes = dict(faceA=(torch.int32, (nA,)), baryA=(torch.float32, (nA, 3)), dist2A=(torch.float32, (nA,)),
                  faceB=(torch.int32, (nB,)), baryB=(torch.float32, (nB, 3)), dist2B=(torch.float32, (nB,)))
    for k, (dt, shape) in shapes.items():
        t = ps.get(k)
        if t is None:
            if k in ("faceA", "faceB"):
                raise ValueError(f"ps[{k!r}] is required")
            continue
        if not t.is_cuda or t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError(f"ps[{k!r}] must be a contiguous CUDA {dt} tensor of shape {shape}")
    buf = ws.get(lib().mesh_chamfer_step_workspace_bytes(nA, nB))
    out = torch.empty(2, dtype=torch.float64, device=SA.device) if out is None else out
    check(lib().mesh_chamfer_step(A.handle, SA.data_ptr(), nA, B.handle, SB.data_ptr(), nB, buf.data_ptr(),
                                  buf.numel(), out.data_ptr(), _ptr(ps.get("faceA")), _ptr(ps.get("baryA")),
                                  _ptr(ps.get("dist2A")), _ptr(ps.get("faceB")), _ptr(ps.get("baryB")),
                                  _ptr(ps.get("dist2B")), _stream()), "mesh_chamfer_step")
    return out


def l2_read_bandwidth(nbytes: int = 48 << 20, passes: int = 8, repeats: int = 20) -> float:
    """Sustained L2 read bandwidth of the current GPU in GB/s (mesh_probe_l2_read over an
    L2-resident buffer, CUDA events, best of `repeats` after a warm-up)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    sink = torch.empty(int(lib().mesh_probe_sink_bytes()), dtype=torch.uint8, device=dev)

    def run():
        check(lib().mesh_probe_l2_read(buf.data_ptr(), nbytes, passes, sink.data_ptr(), sink.numel(),
                                       _stream()), "mesh_probe_l2_read")

    run()
    torch.cuda.synchronize()
    best = math.inf
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b) * 1e-3)
    return nbytes * passes / best / 1e9


def chamfer_backward(A: MeshBVH, SA: torch.Tensor, B: MeshBVH, SB: torch.Tensor, g: torch.Tensor,
                     ps: dict, gSA=None, gVA=None, gSB=None, gVB=None) -> None:
    """Reverse mode of chamfer() (mesh_chamfer_backward), both directions in one launch:
    g = dL/d(out) (float64 [2] on the device), ps = the forward's per-sample faceA /
    baryA / faceB / baryB; gSA / gSB are written, gVA / gVB accumulated (each may be
    None), on the meshes' current vertex buffers."""
    SA = _f32(SA, 3, "SA")
    SB = _f32(SB, 3, "SB")
    if not g.is_cuda or g.dtype != torch.float64 or g.numel() != 2:
        raise ValueError("g must be a CUDA float64 tensor of 2 elements")
    g = g.contiguous()
    for name, t, n in (("gSA", gSA, SA.shape[0]), ("gSB", gSB, SB.shape[0])):
        if t is not None and (t.dtype != torch.float32 or tuple(t.shape) != (n, 3) or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 [{n}, 3] tensor")
    for name, t in (("gVA", gVA), ("gVB", gVB)):
        if t is not None and (t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 3
                              or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 [nV, 3] tensor")
    check(lib().mesh_chamfer_backward(A.handle, SA.data_ptr(), SA.shape[0], B.handle, SB.data_ptr(),
                                      SB.shape[0], g.data_ptr(), _ptr(ps["faceA"]), _ptr(ps["baryA"]),
                                      _ptr(ps["faceB"]), _ptr(ps["baryB"]), _ptr(gSA), _ptr(gVA),
                                      _ptr(gSB), _ptr(gVB), _stream()), "mesh_chamfer_backward")


def emd(A: torch.Tensor, B: torch.Tensor, eps_rel: float = 1e-5, max_iters: int = 1_000_000,
        ws: Workspace | None = None, want_assignment: bool = False):
    """Earth Mover's Distance of two equal-size point sets (mesh_emd): a float64
    scalar tensor within eps_rel x box diagonal of the exact minimum mean distance;
    with want_assignment also the bijection (int32) and the auction rounds used."""
    A = _f32(A, 3, "A")
    B = _f32(B, 3, "B")
    if A.shape[0] != B.shape[0]:
        raise ValueError("EMD needs equal-size point sets")
    n = A.shape[0]
    ws = Workspace(A.device) if ws is None else ws
    buf = ws.get(lib().mesh_emd_workspace_bytes(n))
    out = torch.empty(1, dtype=torch.float64, device=A.device)
    sigma = torch.empty(n, dtype=torch.int32, device=A.device) if want_assignment else None
    it = C.c_int64(0)
    check(lib().mesh_emd(A.data_ptr(), B.data_ptr(), n, float(eps_rel), int(max_iters), buf.data_ptr(),
                         buf.numel(), out.data_ptr(), _ptr(sigma), C.byref(it), _stream()), "mesh_emd")
    return (out[0], sigma, it.value) if want_assignment else out[0]


def _camera(R, t, fx, fy, cx, cy, width, height, near, background):
    cam = _abi.Camera()
    Rl = [float(x) for x in torch.as_tensor(R, dtype=torch.float64).reshape(-1).tolist()]
    tl = [float(x) for x in torch.as_tensor(t, dtype=torch.float64).reshape(-1).tolist()]
    cam.R[:] = Rl
    cam.t[:] = tl
    cam.fx, cam.fy, cam.cx, cam.cy, cam.near_z = float(fx), float(fy), float(cx), float(cy), float(near)
    cam.width, cam.height = int(width), int(height)
    cam.background[:] = [float(x) for x in background]
    return cam


def gs_render_capacity(mu, quat, scale, opacity, color, R, t, fx, fy, cx, cy, width, height,
                       max_instances: int, near=0.01, background=(0.0, 0.0, 0.0),
                       ws: Workspace | None = None, out=None, counts: torch.Tensor | None = None):
    """Gaussian-splatting render with a fixed instance capacity (mesh_gs_render_capacity):
    asynchronous, capturable in a CUDA graph.  `counts` (int32 [2] on the device, created
    if None) receives (overflow, instances); returns (image, trans, counts)."""
    mu, quat, scale = _f32(mu, 3, "mu"), _f32(quat, 4, "quat"), _f32(scale, 3, "scale")
    opacity, color = _f32(opacity, None, "opacity"), _f32(color, 3, "color")
    n = mu.shape[0]
    cam = _camera(R, t, fx, fy, cx, cy, width, height, near, background)
    if out is None:
        out = (torch.empty(height, width, 3, device=mu.device), torch.empty(height, width, device=mu.device))
    image, trans = out
    if counts is None:
        counts = torch.zeros(2, dtype=torch.int32, device=mu.device)
    ws = Workspace(mu.device) if ws is None else ws
    buf = ws.get(lib().mesh_gs_workspace_bytes(n, int(max_instances), int(width), int(height)))
    check(lib().mesh_gs_render_capacity(mu.data_ptr(), quat.data_ptr(), scale.data_ptr(), opacity.data_ptr(),
                                        color.data_ptr(), n, C.byref(cam), int(max_instances), buf.data_ptr(),
                                        buf.numel(), image.data_ptr(), _ptr(trans), counts.data_ptr(),
                                        _stream()), "mesh_gs_render_capacity")
    return image, trans, counts


def gs_render(mu, quat, scale, opacity, color, R, t, fx, fy, cx, cy, width, height, near=0.01,
              background=(0.0, 0.0, 0.0), ws: Workspace | None = None, out=None):
    """Gaussian-splatting render (mesh_gs_render): image [height, width, 3] and
    transmittance [height, width]; the workspace grows to what the view needs."""
    mu, quat, scale = _f32(mu, 3, "mu"), _f32(quat, 4, "quat"), _f32(scale, 3, "scale")
    opacity, color = _f32(opacity, None, "opacity"), _f32(color, 3, "color")
    n = mu.shape[0]
    cam = _abi.Camera()
    Rl = [float(x) for x in torch.as_tensor(R, dtype=torch.float64).reshape(-1).tolist()]
    tl = [float(x) for x in torch.as_tensor(t, dtype=torch.float64).reshape(-1).tolist()]
    cam.R[:] = Rl
    cam.t[:] = tl
    cam.fx, cam.fy, cam.cx, cam.cy, cam.near_z = float(fx), float(fy), float(cx), float(cy), float(near)
    cam.width, cam.height = int(width), int(height)
    cam.background[:] = [float(x) for x in background]
    if out is None:
        out = (torch.empty(height, width, 3, device=mu.device), torch.empty(height, width, device=mu.device))
    image, trans = out
    ws = Workspace(mu.device) if ws is None else ws
    need = C.c_size_t(lib().mesh_gs_workspace_bytes(n, 4 * n + 1, int(width), int(height)))
    for _ in range(3):
        buf = ws.get(need.value)
        st = lib().mesh_gs_render(mu.data_ptr(), quat.data_ptr(), scale.data_ptr(), opacity.data_ptr(),
                                  color.data_ptr(), n, C.byref(cam), buf.data_ptr(), buf.numel(),
                                  C.byref(need), image.data_ptr(), _ptr(trans), _stream())
        if st != 3 or need.value <= buf.numel():
            break
    check(st, "mesh_gs_render")
    return image, trans


def morton_order(P: torch.Tensor, ws: Workspace | None = None) -> torch.Tensor:
    """int32 permutation sorting the points [n, 3] by Morton key (see mesh_morton_order)."""
    P = _f32(P, 3, "P")
    n = P.shape[0]
    ws = Workspace(P.device) if ws is None else ws
    buf = ws.get(lib().mesh_morton_order_workspace_bytes(n))
    order = torch.empty(n, dtype=torch.int32, device=P.device)
    check(lib().mesh_morton_order(P.data_ptr(), n, order.data_ptr(), buf.data_ptr(), buf.numel(),
                                  _stream()), "mesh_morton_order")
    return order


def set_query_group(lanes: int) -> None:
    """Force the lanes per query of the traversal kernels (0 = automatic)."""
    check(lib().mesh_set_query_group(int(lanes)), "mesh_set_query_group")


def set_traversal(variant: int) -> None:
    """One-thread traversal variant 0..12 (see mesh_set_traversal in include/meshgs.h)."""
    check(lib().mesh_set_traversal(int(variant)), "mesh_set_traversal")


def launch_count() -> int:
    return int(lib().mesh_launch_count())
