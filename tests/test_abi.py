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
