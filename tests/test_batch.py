"""Batch form: several molecules in one call give exactly the meshes of
one-at-a-time calls, both with the shared level loop (each level's kernels
launched once over the octets of every molecule with the same D) and with
whole meshes on host worker threads; the shared loop also against the
oracle."""
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


LEVEL_KEYS = ("examined", "discarded", "accepted", "forced", "split")


def _same_mesh(b, s):
    assert np.array_equal(b.cube_keys, s.cube_keys)
    assert np.array_equal(b.vertex_keys, s.vertex_keys)
    assert np.array_equal(b.triangles, s.triangles)
    assert np.array_equal(b.vertices, s.vertices)
    assert b.stats["n_triangles"] == s.stats["n_triangles"] > 0
    for k in LEVEL_KEYS:
        assert b.stats[k] == s.stats[k], k


@pytest.mark.parametrize("batch_mode", ["shared", "threads"])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_batch_equals_single_calls(mols, mode, batch_mode):
    import paper_1611_03474_gb300 as gs
    prec = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    bm = gs.GS_BATCH_SHARED_LEVELS if batch_mode == "shared" else gs.GS_BATCH_THREADS
    batch = gs.mesh_gaussian_surface_batch(mols, ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                           precision_mode=prec, n_workers=3, batch_mode=bm)
    assert len(batch) == len(mols)
    for (xyz, r, D), b in zip(mols, batch):
        s = gs.mesh_gaussian_surface(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["max_depth"], precision_mode=prec)
        _same_mesh(b, s)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_shared_levels_small_chunks_and_coarse_cubes(mols, mode):
    """Level chunks of 1000 octets (debug bit 1), so that molecules straddle
    chunk boundaries, at a precision that accepts cubes on several levels
    (cubes of different sizes, constrained vertex values): still the meshes
    of single calls."""
    import paper_1611_03474_gb300 as gs
    prec = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    batch = gs.mesh_gaussian_surface_batch(mols, ARGS["c"], 5e-2, ARGS["max_depth"], precision_mode=prec,
                                           n_workers=2, debug_flags=2)
    coarse = 0
    for (xyz, r, D), b in zip(mols, batch):
        s = gs.mesh_gaussian_surface(xyz, r, D, ARGS["c"], 5e-2, ARGS["max_depth"], precision_mode=prec)
        _same_mesh(b, s)
        coarse += sum(b.stats["accepted"][:ARGS["max_depth"]])
    assert coarse > 0


def test_batch_single_molecule_and_duplicates(mols):
    """One molecule, and the same molecule twice in one group."""
    import paper_1611_03474_gb300 as gs
    xyz, r, D = mols[1]
    s = gs.mesh_gaussian_surface(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                 precision_mode=gs.GS_PREC_MIXED)
    for group in ([mols[1]], [mols[1], mols[1]]):
        for b in gs.mesh_gaussian_surface_batch(group, ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                                precision_mode=gs.GS_PREC_MIXED):
            _same_mesh(b, s)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_batch_two_molecules_match_oracle(mols, mode):
    """Two molecules of different D through the shared level loop against
    the oracle: cube set and topology bit-exact, vertices within 1e-5 A."""
    import paper_1611_03474_gb300 as gs
    from meshcheck import canonical_triangles
    prec = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    pair = [mols[0], mols[4]]
    batch = gs.mesh_gaussian_surface_batch(pair, ARGS["c"], ARGS["precision"], ARGS["max_depth"], precision_mode=prec)
    for (xyz, r, D), b in zip(pair, batch):
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


def test_batch_rejects_unknown_mode(mols):
    import paper_1611_03474_gb300 as gs
    with pytest.raises(gs.GsError):
        gs.mesh_gaussian_surface_batch(mols[:2], 1.0, 1e-3, 3, batch_mode=7)


def test_batch_error_names_the_molecule(mols):
    """A molecule outside the mixed form's FP32 range (D r^2 plus the cutoff
    exponent above 80) fails the whole call with GS_ERR_ARG and a message
    naming it; no mesh is returned."""
    import paper_1611_03474_gb300 as gs
    bad = list(mols[:3])
    xyz, r, _ = bad[1]
    bad[1] = (xyz, r, 40.0)
    with pytest.raises(gs.GsError) as e:
        gs.mesh_gaussian_surface_batch(bad, ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                       precision_mode=gs.GS_PREC_MIXED)
    assert e.value.code == -1 and "molecule 1" in str(e.value)
