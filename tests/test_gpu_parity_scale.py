"""Whole-mesh parity with the oracle at the sizes and code paths the
benchmark runs, on the GPU through the C ABI:
  * the 20,000-atom globular molecule, meshed whole by both sides (the
    oracle on all host cores; its output does not depend on the thread count);
  * windows of the 1,000,020-atom assembly: the method is local (every
    decision and value reads only atoms within the cutoff radius of its cube
    or point; section 3.1), so the oracle meshing the atoms within a margin
    of a window reproduces the GPU's full-size cubes, surface-point keys,
    vertex positions and triangles inside the window;
  * small inputs with the level loop cut into chunks of 1000 octets, the
    path that only the largest inputs take by default.
Bars: cube and key sets and canonical triangles bit-exact, vertices within
1e-5 A."""
import time

import numpy as np
import pytest

import oracle
import synth
from meshcheck import canonical_triangles, check_closed_manifold, window_compare, window_oracle

pytestmark = pytest.mark.gpu

gs = pytest.importorskip("paper_1611_03474_gb300")


def _mode(name):
    return gs.GS_PREC_MIXED if name == "mixed" else gs.GS_PREC_FP64


def _compare_whole(m, ref):
    assert m.stats["loop_errors"] == 0
    assert np.array_equal(np.sort(m.cube_keys), ref["cube_keys"])
    assert np.array_equal(np.sort(m.vertex_keys), ref["vkeys"])
    order = np.argsort(m.vertex_keys)
    assert np.abs(m.vertices[order] - ref["vertices"]).max() < 1e-5
    assert np.array_equal(canonical_triangles(m.vertex_keys, m.triangles),
                          canonical_triangles(ref["vkeys"], ref["triangles"]))


@pytest.fixture(scope="module")
def c2():
    cfg = synth.config("globular20k")
    threads = oracle.set_threads(0)
    t0 = time.perf_counter()
    ref = oracle.mesh(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"])
    dt = time.perf_counter() - t0
    print("oracle globular20k: %.1f s on %d threads, %d cubes, %d triangles"
          % (dt, threads, len(ref["cube_keys"]), len(ref["triangles"])))
    return cfg, ref


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_mesh_parity_globular20k(c2, mode):
    cfg, ref = c2
    m = gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                 min_edge=cfg["min_edge"], precision_mode=_mode(mode))
    assert m.stats["examined"] == ref["stats"]["examined"][:len(m.stats["examined"])]
    _compare_whole(m, ref)
    check_closed_manifold(m.vertices, m.triangles)


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
@pytest.mark.parametrize("mol", ["globular1000", "chain100_coarse"])
def test_mesh_parity_small_chunks(mode, mol):
    """debug bit 1: 1000 octets per chunk, so levels span several chunks and a
    ragged last one; the mesh must equal the oracle's."""
    if mol == "globular1000":
        xyz, r = synth.globular(1000, seed=5)
        prec = 1e-3
    else:
        cfg = synth.config("chain100")
        xyz, r = cfg["xyz"], cfg["r"]
        prec = 0.05
    kw = dict(D=0.5, c=1.0, precision=prec, max_depth=3)
    m = gs.mesh_gaussian_surface(xyz, r, kw["D"], kw["c"], kw["precision"], kw["max_depth"], min_edge=0.25,
                                 precision_mode=_mode(mode), debug_flags=2)
    assert max(m.stats["examined"]) > 8 * 1000  # at least one level spans several chunks
    ref = oracle.mesh(xyz, r, kw["D"], kw["c"], kw["precision"], 0.25, kw["max_depth"])
    _compare_whole(m, ref)


# ------------------------------------------------------------------ windows


def _window_centres(cfg, count=4, seed=3):
    """Points just outside the surface of a few units (one per unit), where
    the window holds surface cubes."""
    rng = np.random.default_rng(seed)
    xyz = cfg["xyz"]
    nu = 16667
    out = []
    for u in rng.choice(60, count, replace=False):
        unit = xyz[u * nu:(u + 1) * nu]
        cen = unit.mean(0)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        p = unit[np.argmax((unit - cen) @ d)]
        out.append(p + 1.0 * d)
    return out


def test_window_parity_assembly1m():
    """Both precision forms of the full-size assembly against the oracle's
    meshes of three windows (each computed once)."""
    cfg = synth.config("assembly1m")
    args = (cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"])
    full = {}
    for mode in ("mixed", "fp64"):
        m = gs.mesh_gaussian_surface(*args, min_edge=cfg["min_edge"], precision_mode=_mode(mode))
        full[mode] = dict(cube_keys=m.cube_keys, vkeys=m.vertex_keys, vertices=m.vertices, triangles=m.triangles)
        del m
    oracle.set_threads(0)
    tris = {"mixed": 0, "fp64": 0}
    for centre in _window_centres(cfg, count=3):
        win = window_oracle(cfg, centre)
        for mode in tris:
            tris[mode] += window_compare(full[mode], cfg, win)
    print("assembly1m windows: triangles compared", tris)


def test_window_parity_assembly1m_adaptive():
    """The adaptive path at full size: the assembly at precision 5e-2, where
    surface cubes are accepted on two levels and cubes of different sizes
    join through constrained vertex values and disagreement splits (rounds
    to a fixpoint), in the mixed form, against the oracle's meshes of two
    windows.  The splits and the 2:1 balance reach only a few cubes, so a
    14 A margin around the window keeps them local."""
    cfg = synth.config("assembly1m")
    m = gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], 5e-2, cfg["max_depth"],
                                 min_edge=cfg["min_edge"], precision_mode=_mode("mixed"))
    st = m.stats
    assert sum(st["accepted"][:cfg["max_depth"]]) > 0 and st["constrained_vertices"] > 0
    full = dict(cube_keys=m.cube_keys, vkeys=m.vertex_keys, vertices=m.vertices, triangles=m.triangles)
    del m
    oracle.set_threads(0)
    tris, coarse = 0, 0
    for centre in _window_centres(cfg, count=2, seed=5):
        win = window_oracle(cfg, centre, margin=14.0, precision=5e-2)
        coarse += sum(win["ref"]["stats"]["accepted"][:cfg["max_depth"]])
        tris += window_compare(full, cfg, win)
    assert coarse > 0
    print("assembly1m adaptive windows: triangles compared", tris)
