"""GPU parity for cubes of different sizes (section 2.3: the points of the
neighbouring cubes that lie in the current cube are taken into its loops),
through the C ABI, against the oracle: cube sets, surface-point keys and
canonical triangles bit-exact, vertices within 1e-5 A, on inputs whose
final cubes span two levels; both precision forms, the equal-size reading,
the multi-chunk level path and the gradient through constrained values."""
import numpy as np
import pytest

import oracle
import synth
from meshcheck import canonical_triangles, check_closed_manifold

pytestmark = pytest.mark.gpu

gs = pytest.importorskip("paper_1611_03474_gb300")


def _inputs(name):
    if name == "chain100":
        cfg = synth.config("chain100")
        return cfg["xyz"], cfg["r"], cfg["D"]
    if name == "chain30":
        xyz, r = synth.chain(30, seed=7)
        return xyz, r, 0.9
    xyz, r = synth.globular(1000, seed=5)
    return xyz, r, 0.5


CASES = [("chain100", 0.05, 3, 0.25), ("chain30", 0.2, 3, 0.25), ("chain30", 0.05, 4, 0.125),
         ("globular1000", 0.05, 3, 0.25), ("chain100", 0.2, 4, 0.125)]
MODES = {"fp64": "GS_PREC_FP64", "mixed": "GS_PREC_MIXED"}


def _assert_parity(m, ref):
    assert m.stats["loop_errors"] == 0
    assert np.array_equal(np.sort(m.cube_keys), ref["cube_keys"])
    assert np.array_equal(np.sort(m.vertex_keys), ref["vkeys"])
    order = np.argsort(m.vertex_keys)
    assert np.abs(m.vertices[order] - ref["vertices"]).max() < 1e-5
    assert np.array_equal(canonical_triangles(m.vertex_keys, m.triangles),
                          canonical_triangles(ref["vkeys"], ref["triangles"]))


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("name,prec,md,me", CASES)
def test_mixed_levels_parity(name, prec, md, me, mode):
    xyz, r, D = _inputs(name)
    m = gs.mesh_gaussian_surface(xyz, r, D, 1.0, prec, md, min_edge=me, precision_mode=getattr(gs, MODES[mode]))
    ref = oracle.mesh(xyz, r, D, 1.0, prec, me, md)
    st, rs = m.stats, ref["stats"]
    assert len(set((np.asarray(m.cube_keys).astype(np.int64) >> 59).tolist())) >= 2
    assert st["constrained_vertices"] == rs["constrained_vertices"] > 0
    assert st["agreement_splits"] == rs["agreement_splits"]
    assert st["conformity_splits"] == rs["conformity_splits"]
    assert st["mixed_cubes"] > 0
    _assert_parity(m, ref)
    check_closed_manifold(m.vertices, m.triangles)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_mixed_levels_small_chunks(mode):
    """debug bit 1: levels in chunks of 1000 octets, at mixed levels"""
    xyz, r, D = _inputs("globular1000")
    m = gs.mesh_gaussian_surface(xyz, r, D, 1.0, 0.05, 3, min_edge=0.25, precision_mode=getattr(gs, MODES[mode]),
                                 debug_flags=2)
    assert max(m.stats["examined"]) > 8 * 1000
    _assert_parity(m, oracle.mesh(xyz, r, D, 1.0, 0.05, 0.25, 3))


def test_mixed_form_equals_fp64_form_at_mixed_levels():
    xyz, r, D = _inputs("globular1000")
    a = gs.mesh_gaussian_surface(xyz, r, D, 1.0, 0.05, 3, precision_mode=gs.GS_PREC_FP64)
    b = gs.mesh_gaussian_surface(xyz, r, D, 1.0, 0.05, 3, precision_mode=gs.GS_PREC_MIXED)
    assert np.array_equal(np.sort(a.cube_keys), np.sort(b.cube_keys))
    assert np.array_equal(np.sort(a.vertex_keys), np.sort(b.vertex_keys))
    assert np.array_equal(canonical_triangles(a.vertex_keys, a.triangles),
                          canonical_triangles(b.vertex_keys, b.triangles))
    oa, ob = np.argsort(a.vertex_keys), np.argsort(b.vertex_keys)
    assert np.abs(a.vertices[oa] - b.vertices[ob]).max() < 1e-5


@pytest.mark.parametrize("mode", sorted(MODES))
def test_equal_size_reading_parity(mode):
    """conform_mode GS_CONFORM_EQUAL against the oracle's conform=1"""
    xyz, r, D = _inputs("chain100")
    kw = dict(min_edge=0.25, conform_mode=gs.GS_CONFORM_EQUAL)
    if mode == "mixed":
        kw["precision_mode"] = gs.GS_PREC_MIXED
    m = gs.mesh_gaussian_surface(xyz, r, D, 1.0, 0.05, 3, **kw)
    ref = oracle.mesh(xyz, r, D, 1.0, 0.05, 0.25, 3, conform=1)
    assert m.stats["conformity_splits"] == ref["stats"]["conformity_splits"] > 0
    assert m.stats["constrained_vertices"] == 0
    _assert_parity(m, ref)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_gradient_through_constrained_values(mode):
    """gs_mesh_backward against the oracle's gradient on a mesh with
    constrained vertices (loss gradient mapped by vertex key)."""
    from meshcheck import key_normal_weights, surface_loss_grad
    xyz, r = synth.chain(12, seed=3)
    D, prec, me, md = 0.5, 0.05, 0.25, 3
    pm = getattr(gs, MODES[mode])
    m = gs.mesh_gaussian_surface(xyz, r, D, 1.0, prec, md, min_edge=me, precision_mode=pm)
    assert m.stats["constrained_vertices"] > 0
    g = surface_loss_grad(m.vertices, m.triangles, key_normal_weights(m.vertex_keys))
    ga, gr, gD = gs.gs_mesh_backward(xyz, r, D, 1.0, prec, md, g, min_edge=me, precision_mode=pm)
    om = oracle.mesh(xyz, r, D, 1.0, prec, me, md)
    og = surface_loss_grad(om["vertices"], om["triangles"], key_normal_weights(om["vkeys"]))
    ox, orr, oD = oracle.mesh_grad(xyz, r, D, 1.0, prec, me, md, og)
    scale = max(np.abs(ox).max(), np.abs(orr).max(), abs(oD))
    tol = 1e-9 if mode == "fp64" else 1e-5
    assert np.abs(ga - ox).max() <= tol * scale
    assert np.abs(gr - orr).max() <= tol * scale
    assert abs(gD - oD) <= tol * max(1.0, abs(oD))
