"""ctypes declarations of the meshgs C ABI (include/meshgs.h).

Loading fails loudly: there is no CPU or Python fallback for any entry point.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

_lib = None

VP = C.c_void_p
I64 = C.c_int64
SZ = C.c_size_t

MESH_OK = 0
MESH_ERR_DEVICE = 4
DEV_INDEX_RANGE = 0x1
DEV_STACK_OVERFLOW = 0x2
DEV_DEGENERATE = 0x4
DEV_NONMANIFOLD = 0x8


class Layout(C.Structure):
    _fields_ = [("n_faces", I64), ("n_verts", I64), ("max_faces", I64), ("max_verts", I64),
                ("off_header", SZ), ("off_verts", SZ), ("off_faces", SZ), ("off_keys", SZ),
                ("off_perm", SZ), ("off_nodes", SZ), ("off_parent", SZ), ("off_tris", SZ),
                ("off_rend", SZ), ("off_iperm", SZ), ("off_adj", SZ), ("off_fnorm", SZ), ("off_xlist", SZ), ("off_wide", SZ),
                ("storage_bytes", SZ)]


class BatchLayout(C.Structure):
    _fields_ = [("n_scenes", I64), ("n_verts", I64), ("n_faces", I64), ("max_scenes", I64),
                ("max_verts", I64), ("max_faces", I64), ("off_scene", SZ), ("off_status", SZ),
                ("off_vert_off", SZ), ("off_face_off", SZ), ("off_verts", SZ), ("off_faces", SZ),
                ("off_keys", SZ), ("off_perm", SZ), ("off_nodes", SZ), ("off_parent_int", SZ),
                ("off_parent_leaf", SZ), ("off_tris", SZ), ("off_flags", SZ),
                ("storage_bytes", SZ)]


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("near_z", C.c_float), ("width", C.c_int),
                ("height", C.c_int), ("background", C.c_float * 3)]


SIGNATURES = {
    "mesh_bvh_storage_bytes": (SZ, [I64, I64]),
    "mesh_build_workspace_bytes": (SZ, [I64]),
    "mesh_bvh_create": (C.c_int, [VP, SZ, I64, I64, C.POINTER(VP)]),
    "mesh_bvh_destroy": (None, [VP]),
    "mesh_bvh_get_layout": (C.c_int, [VP, C.POINTER(Layout)]),
    "mesh_build_lbvh": (C.c_int, [VP, VP, I64, VP, I64, VP, SZ, VP]),
    "mesh_build_ploc_workspace_bytes": (SZ, [I64]),
    "mesh_build_ploc": (C.c_int, [VP, VP, I64, VP, I64, VP, SZ, VP]),
    "mesh_mapped_pointer": (C.c_int, [VP, C.POINTER(VP)]),
    "mesh_morton_order_workspace_bytes": (SZ, [I64]),
    "mesh_morton_order": (C.c_int, [VP, I64, VP, VP, SZ, VP]),
    "mesh_update_vertices": (C.c_int, [VP, VP, I64, VP]),
    "mesh_refit": (C.c_int, [VP, VP, I64, VP]),
    "mesh_refit_bind": (C.c_int, [VP, VP, I64, VP, VP, VP, I64, VP, VP, VP, VP]),
    "mesh_closest_point": (C.c_int, [VP, VP, I64, C.c_float, VP, VP, VP, VP, VP]),
    "mesh_closest_point_hinted": (C.c_int, [VP, VP, I64, C.c_float, VP, VP, VP, VP, VP, VP]),
    "mesh_closest_point_stats": (C.c_int, [VP, VP, I64, C.c_float, VP, VP]),
    "mesh_knn_project": (C.c_int, [VP, VP, I64, C.c_int, VP, C.c_float, VP, VP, VP, VP]),
    "mesh_signed_workspace_bytes": (SZ, [I64]),
    "mesh_signed_distance": (C.c_int, [VP, VP, I64, C.c_float, VP, SZ, VP, VP, VP, VP, VP]),
    "mesh_emd_workspace_bytes": (SZ, [I64]),
    "mesh_emd": (C.c_int, [VP, VP, I64, C.c_float, I64, VP, SZ, VP, VP, C.POINTER(I64), VP]),
    "mesh_gs_workspace_bytes": (SZ, [I64, I64, C.c_int, C.c_int]),
    "mesh_gs_render": (C.c_int, [VP, VP, VP, VP, VP, I64, C.POINTER(Camera), VP, SZ, C.POINTER(SZ), VP, VP, VP]),
    "mesh_gs_render_capacity": (C.c_int, [VP, VP, VP, VP, VP, I64, C.POINTER(Camera), I64, VP, SZ, VP, VP, VP, VP]),
    "mesh_contact_workspace_bytes": (SZ, [I64]),
    "mesh_contact": (C.c_int, [VP, VP, I64, C.c_float, VP, VP, VP, VP, VP, SZ, VP]),
    "mesh_set_query_group": (C.c_int, [C.c_int]),
    "mesh_set_traversal": (C.c_int, [C.c_int]),
    "mesh_bvh_set_query_config": (C.c_int, [VP, C.c_int, C.c_int]),
    "mesh_bvh_set_query_block": (C.c_int, [VP, C.c_int]),
    "mesh_bvh_set_leaf_size": (C.c_int, [VP, C.c_int]),
    "mesh_bind_gaussians": (C.c_int, [VP, VP, VP, VP, I64, VP, VP, VP, VP]),
    "mesh_interpolate": (C.c_int, [VP, VP, VP, I64, VP, VP]),
    "mesh_chamfer_workspace_bytes": (SZ, [I64, I64]),
    "mesh_chamfer": (C.c_int, [VP, VP, I64, VP, VP, I64, VP, SZ, VP, VP, VP, VP, VP, VP, VP, VP]),
    "mesh_chamfer_hinted": (C.c_int, [VP, VP, I64, VP, VP, I64, VP, SZ, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP]),
    "mesh_chamfer_step_workspace_bytes": (SZ, [I64, I64]),
    "mesh_chamfer_step": (C.c_int, [VP, VP, I64, VP, VP, I64, VP, SZ, VP, VP, VP, VP, VP, VP, VP, VP]),
    "mesh_chamfer_noalloc": (C.c_int, [VP, VP, I64, VP, VP, I64, VP, VP, VP, VP, VP, VP, VP, VP]),
    "mesh_closest_point_backward": (C.c_int, [VP, VP, I64, VP, VP, VP, VP, VP, VP]),
    "mesh_chamfer_backward": (C.c_int, [VP, VP, I64, VP, VP, I64, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP]),
    "mesh_interpolate_backward": (C.c_int, [VP, VP, VP, I64, VP, VP, VP]),
    "mesh_bind_gaussians_backward": (C.c_int, [VP, VP, VP, VP, I64, VP, VP, VP, VP, VP]),
    "mesh_batch_storage_bytes": (SZ, [I64, I64, I64]),
    "mesh_batch_workspace_bytes": (SZ, [I64, I64]),
    "mesh_batch_create": (C.c_int, [VP, SZ, I64, I64, I64, C.POINTER(VP)]),
    "mesh_batch_destroy": (None, [VP]),
    "mesh_batch_get_layout": (C.c_int, [VP, C.POINTER(BatchLayout)]),
    "mesh_batch_build": (C.c_int, [VP, I64, VP, VP, I64, VP, VP, I64, VP, SZ, VP]),
    "mesh_batch_refit": (C.c_int, [VP, VP, I64, VP]),
    "mesh_batch_closest_point": (C.c_int, [VP, VP, VP, I64, C.c_float, VP, VP, VP, VP, VP]),
    "mesh_batch_bind_gaussians": (C.c_int, [VP, VP, VP, VP, VP, I64, VP, VP, VP, VP]),
    "mesh_batch_status": (C.c_int, [VP, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), VP]),
    "mesh_bvh_status": (C.c_int, [VP, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), VP]),
    "mesh_status_string": (C.c_char_p, [C.c_int]),
    "mesh_launch_count": (C.c_uint64, []),
    "mesh_probe_sink_bytes": (SZ, []),
    "mesh_probe_l2_read": (C.c_int, [VP, SZ, C.c_int, VP, SZ, VP]),
}


def lib():
    """The loaded libmeshgs.so (built in-tree on first use if absent or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"meshgs CUDA library missing at {path}")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class MeshError(RuntimeError):
    pass


def check(status: int, what: str = "") -> None:
    if status != MESH_OK:
        msg = lib().mesh_status_string(status).decode()
        raise MeshError(f"{what}: {msg} (status {status})")


def exported_symbols() -> list[str]:
    return list(SIGNATURES)
