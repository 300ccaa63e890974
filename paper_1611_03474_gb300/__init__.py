"""GB300 (sm_103a) Gaussian-surface mesher: thin Python binding of the C ABI
in include/gsmesh.h (argument marshalling only; every step runs in the
library's CUDA kernels).

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); device
tensors are passed by pointer, so inputs already resident in HBM are not
copied.  The library must be built (build.build()); there is no CPU
fallback: every call raises if the shared library is missing.
"""
from ._native import (GS_BATCH_SHARED_LEVELS, GS_BATCH_THREADS, GS_CHILD_REEXPAND, GS_CHILD_REPROJECT,
                      GS_CONFORM_CONSTRAIN, GS_CONFORM_EQUAL, GS_NORM_MAX, GS_NORM_RSS, GS_NORM_SUM,
                      GS_ORDER_BOUNDS_FIRST, GS_ORDER_LITERAL, GS_PREC_FP64, GS_PREC_MIXED, GsError, Mesh, Stats,
                      autotune_report, autotune_reset, gs_bin_atoms, gs_bin_atoms_static, gs_cube_decisions,
                      gs_eval_field, gs_eval_field_bounded, gs_mesh_backward, gs_mesh_intersections, gs_triangulate_grid, gs_volume_area,
                      library_path, load, memory_kind, mesh_gaussian_surface, mesh_gaussian_surface_batch,
                      mesh_gaussian_surface_into)

__all__ = ["GS_BATCH_SHARED_LEVELS", "GS_BATCH_THREADS", "GS_CHILD_REEXPAND", "GS_CHILD_REPROJECT",
           "GS_CONFORM_CONSTRAIN", "GS_CONFORM_EQUAL", "GS_NORM_MAX", "GS_NORM_RSS", "GS_NORM_SUM",
           "GS_ORDER_BOUNDS_FIRST", "GS_ORDER_LITERAL", "GS_PREC_FP64", "GS_PREC_MIXED", "GsError", "Mesh", "Stats",
           "autotune_report", "autotune_reset", "gs_bin_atoms", "gs_bin_atoms_static", "gs_cube_decisions",
           "gs_eval_field", "gs_eval_field_bounded", "gs_mesh_backward", "gs_mesh_intersections", "gs_triangulate_grid", "gs_volume_area",
           "library_path", "load", "memory_kind", "mesh_gaussian_surface", "mesh_gaussian_surface_batch",
           "mesh_gaussian_surface_into"]
