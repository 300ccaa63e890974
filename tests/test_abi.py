"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/gsmesh.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gsmesh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src)
    skip = {"if", "sizeof", "defined"}
    return sorted({n for n in names if n not in skip and not n.startswith("__")})


@pytest.fixture(scope="module")
def lib():
    from paper_1611_03474_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("mesh_gaussian_surface", "mesh_free", "gs_status_string", "gs_last_error", "gs_bin_atoms",
              "gs_eval_field", "gs_cube_decisions", "gs_triangulate_grid", "gs_default_options",
              "gs_mesh_backward", "gs_volume_area", "mesh_gaussian_surface_batch",
              "gs_mesh_intersections", "mesh_gaussian_surface_into"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), "missing export: " + n


def test_status_strings_without_gpu(lib):
    lib.gs_status_string.restype = ctypes.c_char_p
    assert lib.gs_status_string(0) == b"ok"
    assert lib.gs_status_string(-1) == b"invalid argument"


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    import paper_1611_03474_gb300._native as nat
    monkeypatch.setattr(nat, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(nat, "_lib", None)
    with pytest.raises(nat.GsError):
        nat.load()


def test_argument_errors_without_gpu(lib):
    """Argument validation happens before any CUDA call."""
    import numpy as np
    import paper_1611_03474_gb300 as gs
    with pytest.raises(gs.GsError) as e:
        gs.mesh_gaussian_surface(np.zeros((1, 3)), np.ones(1), -1.0, 1.0, 1e-3, 3)
    assert e.value.code == -1
    with pytest.raises(gs.GsError) as e:
        gs.mesh_gaussian_surface(np.zeros((1, 3)), np.ones(1), 0.5, 1.0, 1e-3, 21)
    assert e.value.code == -1


def test_option_and_buffer_errors_without_gpu(lib):
    """Argument errors of the mesh entry points are found on the host, before
    any device work: unknown readings, readings outside the FP64 form, and
    malformed caller-owned buffers all return GS_ERR_ARG (-1)."""
    import numpy as np
    import paper_1611_03474_gb300 as gs
    from paper_1611_03474_gb300 import _native as nat
    xyz, r = np.zeros((1, 3)), np.ones(1)
    bad = [dict(child_mode=5), dict(decision_order=3), dict(precision_norm=9),
           dict(child_mode=gs.GS_CHILD_REEXPAND, precision_mode=gs.GS_PREC_MIXED),
           dict(decision_order=gs.GS_ORDER_LITERAL, precision_mode=gs.GS_PREC_MIXED),
           dict(precision_norm=gs.GS_NORM_RSS, precision_mode=gs.GS_PREC_MIXED),
           dict(min_edge=0.0), dict(cutoff_rel=1.5)]
    for kw in bad:
        with pytest.raises(gs.GsError) as e:
            gs.mesh_gaussian_surface(xyz, r, 0.5, 1.0, 1e-3, 2, **kw)
        assert e.value.code == -1, kw
    for args in ((xyz, r, 0.0, 1.0, 1e-3, 2), (xyz, r, 0.5, 1.0, 1e-3, 21), (xyz, r, 0.5, -1.0, 1e-3, 2)):
        with pytest.raises(gs.GsError) as e:
            gs.mesh_gaussian_surface(*args)
        assert e.value.code == -1
    L = nat.load()
    opt = L.gs_default_options()
    for caps, ptrs in (((-1, 4, 0), (True, True)), ((4, 4, 0), (False, True)), ((4, 4, 0), (True, False))):
        b = nat.MeshBuffers()
        V, T = np.zeros((4, 3)), np.zeros((4, 3), np.int32)
        b.vertices = V.ctypes.data if ptrs[0] else None
        b.triangles = T.ctypes.data if ptrs[1] else None
        b.cap_vertices, b.cap_triangles, b.cap_cubes = caps
        rc = L.mesh_gaussian_surface_into(nat._ptr(xyz), nat._ptr(r), 1, 0.5, 1.0, 1e-3, 2, ctypes.byref(opt),
                                          ctypes.byref(b))
        assert rc == -1 and (b.n_vertices, b.n_triangles, b.n_cubes) == (0, 0, 0)


def test_memory_kind_without_gpu(lib):
    """A host array is not device memory (no GPU: the query fails and the
    library treats the buffer as ordinary host memory)."""
    import numpy as np
    import paper_1611_03474_gb300 as gs
    assert gs.memory_kind(np.zeros(4)) == 2
