"""Launch-shape autotuner: every shape of a tuned kernel gives the same mesh
(the shapes change the tile and grid, not the sums), the tuner records one
choice per kernel and size class with a trial time per shape, and the
report works without a GPU."""
import os

import numpy as np
import pytest

import synth


def test_report_without_gpu():
    import paper_1611_03474_gb300 as gs
    gs.autotune_reset()
    assert gs.autotune_report() == []


@pytest.fixture
def restore_env():
    old = os.environ.get("GS_AUTOTUNE")
    yield
    if old is None:
        os.environ.pop("GS_AUTOTUNE", None)
    else:
        os.environ["GS_AUTOTUNE"] = old


@pytest.mark.gpu
def test_every_shape_gives_the_same_mesh(restore_env):
    import paper_1611_03474_gb300 as gs
    xyz, r = synth.globular(3000, seed=11)
    meshes = []
    for k in range(4):
        os.environ["GS_AUTOTUNE"] = "shape:%d" % k
        meshes.append(gs.mesh_gaussian_surface(xyz, r, 0.5, 1.0, 1e-3, 3, precision_mode=gs.GS_PREC_MIXED))
    for m in meshes[1:]:
        assert np.array_equal(m.vertices, meshes[0].vertices)
        assert np.array_equal(m.triangles, meshes[0].triangles)
        assert np.array_equal(m.cube_keys, meshes[0].cube_keys)
        # the FP32 values are the same bits too: the same cubes and vertices
        # go to FP64, for the same reasons
        for k in ("pair_terms", "vertex_terms", "recheck_cubes", "recheck_vertices", "recheck_bounds",
                  "recheck_rank", "estimate_fast_cubes", "vertex_mark_cubes"):
            assert m.stats[k] == meshes[0].stats[k], k


@pytest.mark.gpu
def test_tuned_choices_are_recorded(restore_env):
    import paper_1611_03474_gb300 as gs
    xyz, r = synth.globular(3000, seed=11)
    os.environ["GS_AUTOTUNE"] = "0"
    ref = gs.mesh_gaussian_surface(xyz, r, 0.5, 1.0, 1e-3, 3, precision_mode=gs.GS_PREC_MIXED)
    os.environ.pop("GS_AUTOTUNE")
    gs.autotune_reset()
    tuned = gs.mesh_gaussian_surface(xyz, r, 0.5, 1.0, 1e-3, 3, precision_mode=gs.GS_PREC_MIXED)
    again = gs.mesh_gaussian_surface(xyz, r, 0.5, 1.0, 1e-3, 3, precision_mode=gs.GS_PREC_MIXED)
    for m in (tuned, again):
        assert np.array_equal(m.vertices, ref.vertices)
        assert np.array_equal(m.triangles, ref.triangles)
        # trials send their counters to scratch: the counts are the plain run's
        assert m.stats["pair_terms"] == ref.stats["pair_terms"]
        assert m.stats["vertex_terms"] == ref.stats["vertex_terms"]
    rep = gs.autotune_report()
    kernels = {e["kernel"] for e in rep}
    assert "k_field_f32w" in kernels and "k_estimate_f32" in kernels
    assert any(k.startswith("k_accum_f32") for k in kernels)
    shapes = {"k_field_f32w": 4, "k_estimate_f32": 2}
    for e in rep:
        n = shapes.get(e["kernel"], 3)
        assert len(e["trial_ms"]) == n and 0 <= e["choice"] < n
        assert e["trial_ms"][e["choice"]] == min(e["trial_ms"])
        assert all(t > 0 for t in e["trial_ms"])
