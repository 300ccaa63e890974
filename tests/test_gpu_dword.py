"""The double-word FP32 field (each value a hi + lo float pair), which the
mixed mode runs where a vertex's FP32 bound is too wide, against the FP64
field and the oracle: the difference stays within the bound it returns, and
that bound is thousands of times below the FP32 one."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

gs = pytest.importorskip("paper_1611_03474_gb300")


@pytest.mark.parametrize("D", [0.5, 0.9])
def test_bounded_field_within_its_bound(D):
    xyz, r = synth.globular(5000, seed=3)
    rng = np.random.default_rng(int(D * 10))
    # inside atoms, in the surface shell and beyond it
    pts = xyz[rng.integers(0, len(r), 40000)] + rng.normal(0, 2.5, (40000, 3))
    phi, err = gs.gs_eval_field_bounded(xyz, r, D, 1.0, pts)
    p64 = gs.gs_eval_field(xyz, r, D, 1.0, pts)
    e = err.astype(np.float64)
    # the FP64 form's own rounding (about 1e-15 of phi) on top of the bound
    assert np.all(np.abs(phi - p64) <= e + 1e-14 * np.abs(p64))
    # about 5e-10 relative for offsets of ~100 A (a few thousand times
    # below the FP32 bound of ~1e-6)
    assert np.all(e <= 2e-9 * np.abs(p64) + 1e-300)
    assert np.abs(phi - p64).max() > 0   # the two are different evaluations
    ref = oracle.field(xyz, r, D, 1.0, pts[:3000])
    assert np.all(np.abs(phi[:3000] - ref) <= e[:3000] + 1e-14 * np.abs(ref))


def test_bounded_field_membership_at_the_cutoff():
    """Points at the cutoff distance of one atom (to 1e-7 relative either
    side): the term is in or out exactly as in the FP64 form."""
    D, c, cut = 0.5, 1.0, 1e-8
    xyz = np.array([[10.0, 20.0, 30.0], [40.0, 20.0, 30.0]])
    r = np.array([1.7, 1.5])
    R = np.sqrt(r[0] ** 2 - np.log(cut * c) / D)
    rng = np.random.default_rng(5)
    dirs = rng.normal(size=(2000, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    scale = R * (1.0 + rng.choice([-1, 1], 2000) * rng.uniform(1e-9, 1e-6, 2000))
    pts = xyz[0] + dirs * scale[:, None]
    phi, err = gs.gs_eval_field_bounded(xyz, r, D, c, pts)
    p64 = gs.gs_eval_field(xyz, r, D, c, pts)
    assert np.all(np.abs(phi - p64) <= err.astype(np.float64) + 1e-14 * np.abs(p64))
    inside = (p64 > 0).sum()
    assert 0 < inside < len(pts)   # both sides of the sphere are exercised


def test_mixed_mesh_refines_before_fp64():
    """In the mixed mesh most re-evaluated vertices stop at the double-word
    values; the mesh keeps the FP64 form's cubes and topology."""
    xyz, r = synth.globular(20000, seed=2)
    m = gs.mesh_gaussian_surface(xyz, r, 0.5, 1.0, 1e-3, 3, precision_mode=gs.GS_PREC_MIXED)
    ref = gs.mesh_gaussian_surface(xyz, r, 0.5, 1.0, 1e-3, 3)
    st = m.stats
    print("refined", st["refine_vertices"], "FP64", st["recheck_vertices"], "marked cubes",
          st["vertex_mark_cubes"], "all", st["vertex_mark_all"], "again", st["vertex_mark_fp64_cubes"])
    assert st["refine_vertices"] > 0
    assert st["recheck_vertices"] < st["refine_vertices"]
    assert np.array_equal(np.sort(m.cube_keys), np.sort(ref.cube_keys))
    assert len(m.triangles) == len(ref.triangles)
    ka, kb = np.argsort(m.vertex_keys), np.argsort(ref.vertex_keys)
    assert np.array_equal(m.vertex_keys[ka], ref.vertex_keys[kb])
    assert np.abs(m.vertices[ka] - ref.vertices[kb]).max() < 1e-5
