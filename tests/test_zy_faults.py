"""Failure handling, tested without faulting the GPU: failures are injected
on the host through the GS_FAULT environment variable (a device allocation
that fails, an internal table reported full in the level loop, a host wait
past its deadline).  Each call must return the documented status, leave the
library usable (the next call gives the same mesh as before), and, for a
full table in the level loop, retry with smaller level chunks and succeed
with the same mesh."""
import os

import numpy as np
import pytest

import synth
from meshcheck import canonical_triangles

pytestmark = pytest.mark.gpu

gs = pytest.importorskip("paper_1611_03474_gb300")


@pytest.fixture()
def clean_env():
    yield
    os.environ.pop("GS_FAULT", None)


def _mesh(**kw):
    cfg = synth.config("chain100")
    return gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                    min_edge=cfg["min_edge"], **kw)


def _same(a, b):
    return (np.array_equal(np.sort(a.cube_keys), np.sort(b.cube_keys))
            and np.array_equal(canonical_triangles(a.vertex_keys, a.triangles),
                               canonical_triangles(b.vertex_keys, b.triangles)))


@pytest.mark.parametrize("spec,code", [("alloc@1", -2), ("alloc@5", -2), ("timeout", -4)])
def test_injected_failure_returns_status_and_library_recovers(clean_env, spec, code):
    ref = _mesh()
    os.environ["GS_FAULT"] = spec
    with pytest.raises(gs.GsError) as e:
        _mesh()
    assert e.value.code == code
    del os.environ["GS_FAULT"]
    assert _same(_mesh(), ref)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_capacity_in_level_loop_retries_with_smaller_chunks(clean_env, mode):
    pm = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    ref = _mesh(precision_mode=pm)
    assert ref.stats["retries"] == 0
    os.environ["GS_FAULT"] = "capacity@2"
    m = _mesh(precision_mode=pm)
    assert m.stats["retries"] == 1
    assert _same(m, ref)
