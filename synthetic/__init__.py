"""Seeded, synthetic inputs shared by the oracle tests and the GPU path.

Meshes, boundary conditions, load paths and random states only; no step of the
elastoplastic method is computed here.
"""
from .meshes import Mesh, structured_mesh, boundary_nodes, top_faces, N_NODES  # noqa: F401
from .problems import (Material, Problem, WORKLOADS, ELASTIC, VM_KIN, VM_ISO, DP,  # noqa: F401
                       p1_plane_vm, p2_plane_dp, q1_cube_vm, p2_tet_strip_dp, generic_box,
                       traction_load, vm_iso_material, batch_problems, l_shape_vm,
                       strip_footing_dp, prandtl_nc)
