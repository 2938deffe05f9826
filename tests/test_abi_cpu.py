"""The C-ABI library loads and exports every entry point include/meshgs.h declares,
and its host-side size queries and argument checks work without a GPU (no
call here launches a kernel or touches device memory)."""
import ctypes as C
import os
import re

import pytest

from paper_2606_00444_gb300 import _abi
from paper_2606_00444_gb300._abi import lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "meshgs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mesh_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound():
    names = declared_functions()
    assert len(names) >= 19
    L = lib()
    for n in names:
        assert hasattr(L, n), f"{n} not exported by libmeshgs.so"
    assert set(names) == set(_abi.exported_symbols())


def test_sizes_are_monotone_and_reject_bad_input():
    L = lib()
    assert L.mesh_build_ploc_workspace_bytes(200000) > L.mesh_build_workspace_bytes(200000)
    assert L.mesh_build_ploc_workspace_bytes(-1) == 0
    s1 = L.mesh_bvh_storage_bytes(642, 1280)
    s2 = L.mesh_bvh_storage_bytes(100000, 200000)
    assert 0 < s1 < s2
    assert s2 >= 200000 * (64 + 48 + 16 + 4 + 4 + 8 + 4) + 100000 * 16
    assert L.mesh_bvh_storage_bytes(-1, 10) == 0
    assert L.mesh_build_workspace_bytes(200000) >= 200000 * 32
    assert L.mesh_build_workspace_bytes(-5) == 0
    assert L.mesh_chamfer_workspace_bytes(1 << 20, 1 << 20) >= 8 * 2 * (1 << 20) // 128
    # the ordered Chamfer keeps a 4-byte key, its sorted copy and the order per sample
    assert L.mesh_chamfer_step_workspace_bytes(10000, 10000) >= \
        L.mesh_chamfer_workspace_bytes(10000, 10000) + 3 * 4 * 20000
    assert L.mesh_chamfer_step_workspace_bytes(-1, 4) == 0
    assert L.mesh_chamfer_step_workspace_bytes(1 << 31, 1 << 31) == 0


def test_create_validates_storage_on_the_host():
    L = lib()
    h = C.c_void_p()
    need = L.mesh_bvh_storage_bytes(10, 16)
    fake = 1 << 40                                      # never dereferenced by create
    assert L.mesh_bvh_create(None, need, 10, 16, C.byref(h)) == 1          # null storage
    assert L.mesh_bvh_create(fake + 8, need, 10, 16, C.byref(h)) == 1      # misaligned
    assert L.mesh_bvh_create(fake, need - 1, 10, 16, C.byref(h)) == 3      # too small
    assert L.mesh_bvh_create(fake, need, 10, 16, C.byref(h)) == 0
    lay = _abi.Layout()
    assert L.mesh_bvh_get_layout(h, C.byref(lay)) == 0
    assert lay.max_faces == 16 and lay.storage_bytes == need
    offs = [lay.off_header, lay.off_verts, lay.off_faces, lay.off_keys, lay.off_perm,
            lay.off_nodes, lay.off_parent, lay.off_tris, lay.off_rend, lay.off_iperm, lay.off_adj, lay.off_fnorm, lay.off_xlist,
            lay.off_wide]
    assert offs == sorted(offs) and all(o % 256 == 0 for o in offs)
    # the 4-wide records: 128 bytes per internal node, the last array of the block
    assert lay.off_wide + 128 * (16 - 1) <= lay.storage_bytes
    # traversal variants 0-13, -1 = the process-wide setting; anything else is refused
    assert L.mesh_bvh_set_query_config(h, 1, 13) == 0 and L.mesh_bvh_set_query_config(h, 1, 14) == 1
    assert L.mesh_bvh_set_query_config(h, -1, -1) == 0
    assert L.mesh_set_traversal(14) == 1 and L.mesh_set_traversal(-1) == 1
    # argument errors are caught before anything is launched
    n0 = L.mesh_launch_count()
    assert L.mesh_build_lbvh(h, None, 10, None, 16, None, 0, None) == 1
    assert L.mesh_build_lbvh(h, fake, 11, fake, 16, None, 0, None) == 1     # nV > max
    assert L.mesh_build_lbvh(h, fake, 10, fake, 16, None, 0, None) == 3     # no workspace
    assert L.mesh_build_ploc(h, None, 10, None, 16, None, 0, None) == 1
    assert L.mesh_build_ploc(h, fake, 11, fake, 16, None, 0, None) == 1     # nV > max
    assert L.mesh_build_ploc(h, fake, 10, fake, 17, None, 0, None) == 1     # nF > max
    assert L.mesh_build_ploc(h, fake, 10, fake, 16, None, 0, None) == 3     # no workspace
    assert L.mesh_build_ploc(h, fake, 10, fake, 16, fake + 8, 1 << 30, None) == 3   # misaligned
    assert L.mesh_closest_point(None, fake, 4, C.c_float(1.0), None, None, None, None, None) == 1
    assert L.mesh_closest_point(h, fake, 4, C.c_float(-1.0), None, None, None, None, None) == 1
    assert L.mesh_closest_point(h, fake, 0, C.c_float(1.0), None, None, None, None, None) == 0
    assert L.mesh_bind_gaussians(h, None, None, None, 3, None, None, None, None) == 1
    assert L.mesh_chamfer(h, fake, 4, h, fake, 4, None, 0, fake, *([None] * 6), None) == 3
    # the ordered Chamfer: the face arrays (hints in, faces out) are required
    assert L.mesh_chamfer_step(h, fake, 4, h, fake, 4, fake, 1 << 30, fake, None, None, None,
                               fake, None, None, None) == 1
    assert L.mesh_chamfer_step(h, fake, 4, h, fake, 4, fake, 1 << 30, fake, fake, None, None,
                               None, None, None, None) == 1
    assert L.mesh_chamfer_step(h, fake, 4, h, fake, 4, None, 0, fake, fake, None, None,
                               fake, None, None, None) == 3
    assert L.mesh_chamfer_step(h, fake, 4, h, fake, 4, fake + 8, 1 << 30, fake, fake, None, None,
                               fake, None, None, None) == 3
    # Chamfer backward: a missing gradient seed, faces or weights; no outputs = no work
    assert L.mesh_chamfer_backward(h, fake, 4, h, fake, 4, None, fake, fake, fake, fake,
                                   fake, None, None, None, None) == 1
    assert L.mesh_chamfer_backward(h, fake, 4, h, fake, 4, fake, None, fake, fake, fake,
                                   fake, None, None, None, None) == 1
    assert L.mesh_chamfer_backward(h, fake, -1, h, fake, 4, fake, fake, fake, fake, fake,
                                   None, None, None, None, None) == 1
    assert L.mesh_chamfer_backward(h, fake, 4, h, fake, 4, fake, fake, fake, fake, fake,
                                   None, None, None, None, None) == 0
    assert L.mesh_launch_count() == n0
    L.mesh_bvh_destroy(h)


def test_status_strings():
    L = lib()
    assert L.mesh_status_string(0) == b"ok"
    for s in range(1, 5):
        assert len(L.mesh_status_string(s)) > 3
    with pytest.raises(_abi.MeshError):
        _abi.check(1, "x")
