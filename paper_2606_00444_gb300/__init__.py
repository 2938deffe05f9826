"""GB300-native per-frame dynamic-mesh update (LBVH build / refit, closest-point
queries, face-bound Gaussian rebind, Chamfer, and their gradients).

The compute path is the CUDA library ``libmeshgs.so`` behind the C ABI in
``include/meshgs.h``; this package only marshals PyTorch tensors to it.
"""
from .api import (MeshBatch, MeshBVH, Workspace, chamfer, chamfer_backward, chamfer_step, emd, gs_render,  # noqa: F401
                  gs_render_capacity, l2_read_bandwidth, launch_count, morton_order, set_query_group, set_traversal)
from ._abi import MeshError, lib  # noqa: F401
from . import autograd  # noqa: F401
from .tracking import TemporalTracker, project_template  # noqa: F401
