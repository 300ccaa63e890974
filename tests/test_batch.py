"""Batch form: several molecules meshed concurrently (host worker threads,
one CUDA stream each) give exactly the meshes of one-at-a-time calls."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ARGS = dict(c=1.0, precision=1e-3, max_depth=3)


@pytest.fixture(scope="module")
def mols():
    out = []
    for i, (n, D) in enumerate([(60, 0.9), (400, 0.5), (150, 0.9), (900, 0.5), (40, 0.5), (250, 0.9)]):
        xyz, r = synth.globular(n, seed=50 + i)
        out.append((xyz + 7.0 * i, r, D))
    return out


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_batch_equals_single_calls(mols, mode):
    import paper_1611_03474_gb300 as gs
    prec = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    batch = gs.mesh_gaussian_surface_batch(mols, ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                           precision_mode=prec, n_workers=3)
    assert len(batch) == len(mols)
    for (xyz, r, D), b in zip(mols, batch):
        s = gs.mesh_gaussian_surface(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["max_depth"], precision_mode=prec)
        assert np.array_equal(b.vertex_keys, s.vertex_keys)
        assert np.array_equal(b.triangles, s.triangles)
        assert np.array_equal(b.vertices, s.vertices)
        assert b.stats["n_triangles"] == s.stats["n_triangles"] > 0


def test_batch_d09_matches_oracle(mols):
    """A D = 0.9 molecule (the other decay rate of the batch workload) against
    the oracle: cube set and topology bit-exact, vertices within 1e-5 A."""
    import paper_1611_03474_gb300 as gs
    from meshcheck import canonical_triangles
    xyz, r, D = mols[0]
    b = gs.mesh_gaussian_surface_batch([mols[0], mols[4]], ARGS["c"], ARGS["precision"], ARGS["max_depth"])[0]
    o = oracle.mesh(xyz, r, D, ARGS["c"], ARGS["precision"], 0.25, ARGS["max_depth"])
    assert np.array_equal(np.sort(b.cube_keys), o["cube_keys"])
    order = np.argsort(b.vertex_keys)
    assert np.array_equal(b.vertex_keys[order], o["vkeys"])
    assert np.abs(b.vertices[order] - o["vertices"]).max() <= 1e-5
    assert np.array_equal(canonical_triangles(b.vertex_keys, b.triangles),
                          canonical_triangles(o["vkeys"], o["triangles"]))


def test_batch_rejects_bad_offsets():
    import paper_1611_03474_gb300 as gs
    with pytest.raises(gs.GsError):
        gs.mesh_gaussian_surface_batch([(np.zeros((0, 3)), np.zeros(0), 0.5)], 1.0, 1e-3, 3)
