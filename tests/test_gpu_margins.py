"""The decision-margin policy on the GPU side: gs_stats.near_threshold
counts the FP64 decisions whose margin is below 1e-10 relative.  On the
ties built on purpose (c equal to a cube's own lower bound, or to a lattice
vertex's own field value; see tests/test_oracle_margins.py) the GPU must
count them in both precision forms, as the oracle does; on ordinary inputs
neither side has any."""
import numpy as np
import pytest

import oracle
import synth
from margin_cases import ONE_ATOM, tie_on_bound, tie_on_vertex

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_tie_on_a_bound_is_counted(mode):
    import paper_1611_03474_gb300 as gs
    prec = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    xyz, r = ONE_ATOM
    c = tie_on_bound()
    m = gs.mesh_gaussian_surface(xyz, r, 0.5, c, 1e-3, 3, precision_mode=prec)
    assert m.stats["near_threshold"][0] >= 1
    assert oracle.mesh(xyz, r, 0.5, c, 1e-3, 0.25, 3)["stats"]["near"][0] >= 1


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_tie_on_a_vertex_is_counted(mode):
    import paper_1611_03474_gb300 as gs
    prec = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    xyz, r = ONE_ATOM
    c = tie_on_vertex()
    m = gs.mesh_gaussian_surface(xyz, r, 0.5, c, 1e-3, 3, precision_mode=prec)
    assert m.stats["near_threshold"][3] >= 1


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_ordinary_inputs_have_no_in_band_decisions(mode):
    import paper_1611_03474_gb300 as gs
    prec = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    xyz, r = synth.globular(2000, seed=7)
    m = gs.mesh_gaussian_surface(xyz, r, 0.5, 1.0, 1e-3, 3, precision_mode=prec)
    assert list(m.stats["near_threshold"]) == [0, 0, 0, 0]
    o = oracle.mesh(xyz, r, 0.5, 1.0, 1e-3, 0.25, 3)
    assert o["stats"]["near"] == [0, 0, 0, 0]
    assert np.array_equal(np.sort(m.cube_keys), o["cube_keys"])
