"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  Bars: bit-exact for integer/key work (cell lists, cube
sets, surface-point keys, triangle topology); floating point within the
stated tolerances (field values 1e-13 relative, coefficient tensors 1e-12 of
their scale, vertex positions 1e-5 A)."""
import numpy as np
import pytest

import oracle
import synth
from meshcheck import canonical_triangles, check_closed_manifold, directed_edge_defects

pytestmark = pytest.mark.gpu

gs = pytest.importorskip("paper_1611_03474_gb300")


@pytest.fixture(scope="module")
def chain100():
    return synth.config("chain100")


def test_cell_list_bit_exact(chain100):
    xyz = chain100["xyz"]
    for cell in (3.1, 1.0, 7.5):
        origin = xyz.min(0) - 2.0
        dims = np.ceil((xyz.max(0) + 2.0 - origin) / cell).astype(np.int64) + 1
        cs, pm = gs.gs_bin_atoms(xyz, cell, origin, dims)
        rs, rp = oracle.cell_list(xyz, cell, origin, dims)
        assert np.array_equal(cs, rs) and np.array_equal(pm, rp)


def test_cell_list_ragged_large():
    rng = np.random.default_rng(11)
    xyz = rng.uniform(-50, 50, (100003, 3))
    origin, cell = np.array([-51.0, -51.0, -51.0]), 3.3
    dims = np.array([32, 32, 32])
    cs, pm = gs.gs_bin_atoms(xyz, cell, origin, dims)
    rs, rp = oracle.cell_list(xyz, cell, origin, dims)
    assert np.array_equal(cs, rs) and np.array_equal(pm, rp)


def test_field_fp64_parity(chain100):
    rng = np.random.default_rng(1)
    xyz, r = chain100["xyz"], chain100["r"]
    pts = xyz[rng.integers(0, len(r), 3000)] + rng.normal(0, 2.0, (3000, 3))
    phi, g = gs.gs_eval_field(xyz, r, 0.5, 1.0, pts, grad=True)
    rphi, rg = oracle.field(xyz, r, 0.5, 1.0, pts, grad=True)
    assert np.allclose(phi, rphi, rtol=1e-13, atol=1e-300)
    assert np.allclose(g, rg, rtol=1e-12, atol=1e-14 * np.abs(rg).max())


def test_field_single_atom_exp():
    """One atom: phi(p) = exp(-D (|p - x|^2 - r^2)) exactly (Eq. 1).  Points
    at distances spanning the whole cutoff radius exercise the FP64 exponential
    over its full argument range; the bound is a few ulp."""
    rng = np.random.default_rng(7)
    D, c, r0 = 0.5, 1.0, 1.7
    xyz = np.array([[12.25, -3.5, 40.125]])
    R = np.sqrt(r0 * r0 - np.log(1e-8 * c) / D)
    dirs = rng.normal(size=(20000, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    pts = xyz + dirs * (rng.random(20000)[:, None] * 0.999 * R)
    phi = gs.gs_eval_field(xyz, np.array([r0]), D, c, pts)
    d2 = ((pts - xyz) ** 2).sum(1)
    ref = np.exp(-D * (d2 - r0 * r0))
    # the two arguments, -D d^2 (plus log w) and -D (d^2 - r^2), round
    # differently by up to half an ulp each; the exponentials, w and the
    # product add a few ulp
    u = 2.0 ** -53
    tol = (D * d2 + np.abs(D * (d2 - r0 * r0))) * u + 8 * u
    assert np.all(np.abs(phi - ref) <= tol * ref)


def _sample_cubes(cfg, rng, n_per_level=200):
    o, nroot, pad = oracle.root_grid(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["min_edge"], cfg["max_depth"])
    keys = []
    for l in range(cfg["max_depth"] + 1):
        h = cfg["min_edge"] * 2 ** (cfg["max_depth"] - l)
        centers = cfg["xyz"][rng.integers(0, len(cfg["r"]), n_per_level)] + rng.normal(0, 2.0, (n_per_level, 3))
        idx = np.floor((centers - o) / h).astype(np.int64)
        idx = np.clip(idx, 0, (nroot << l) - 1)
        for x, y, z in idx:
            keys.append(int(x) | (int(y) << 18) | (int(z) << 36) | (30 << 54) | (l << 59))
    return np.unique(np.array(keys, dtype=np.uint64))


def test_cube_tensors_and_decisions_parity(chain100):
    cfg = chain100
    keys = _sample_cubes(cfg, np.random.default_rng(2))
    A, b, d = gs.gs_cube_decisions(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"],
                                   cfg["max_depth"], keys)
    rA, rb, rd = oracle.cube_batch(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"],
                                   cfg["max_depth"], keys)
    scale = np.abs(rA).sum(1, keepdims=True) + 1e-300
    assert np.all(np.abs(A - rA) <= 1e-12 * scale)
    assert np.array_equal(d, rd)
    kept = rd != 0
    assert np.allclose(b[kept, :4], rb[kept, :4], rtol=1e-9, atol=1e-11)


def _mesh_both(cfg, **kw):
    m = gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                 min_edge=cfg["min_edge"], **kw)
    ref = oracle.mesh(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"])
    return m, ref


def _assert_mesh_parity(m, ref):
    assert np.array_equal(np.sort(m.cube_keys), ref["cube_keys"])
    assert np.array_equal(np.sort(m.vertex_keys), ref["vkeys"])
    order = np.argsort(m.vertex_keys)
    if len(order):
        assert np.abs(m.vertices[order] - ref["vertices"]).max() < 1e-5
    assert np.array_equal(canonical_triangles(m.vertex_keys, m.triangles),
                          canonical_triangles(ref["vkeys"], ref["triangles"]))


def test_mesh_parity_chain100(chain100):
    m, ref = _mesh_both(chain100)
    st = m.stats
    for l in range(chain100["max_depth"] + 1):
        assert st["examined"][l] == ref["stats"]["examined"][l]
        assert st["split"][l] == ref["stats"]["split"][l]
    assert st["loop_errors"] == 0
    _assert_mesh_parity(m, ref)
    check_closed_manifold(m.vertices, m.triangles)


def test_mesh_parity_single_atom_and_mixed_levels():
    xyz, r = np.array([[0.1, 0.2, 0.3]]), np.array([1.5])
    cfg = dict(xyz=xyz, r=r, D=0.5, c=1.0, precision=1e-3, min_edge=0.25, max_depth=3)
    _assert_mesh_parity(*_mesh_both(cfg))
    # a loose precision accepts cubes at several levels: conformity splits
    cfg2 = dict(synth.config("chain100"), precision=0.05)
    m, ref = _mesh_both(cfg2)
    _assert_mesh_parity(m, ref)
    assert m.stats["conformity_splits"] == ref["stats"]["conformity_splits"]


def _degenerate_cases():
    rng = np.random.default_rng(41)
    small = synth.config("chain100")
    base = dict(D=0.5, c=1.0, precision=1e-3, min_edge=0.25, max_depth=3)
    a, ra = synth.globular(150, seed=42)
    b, rb = synth.globular(120, seed=43)
    dup = small["xyz"][:20].copy()
    return {
        # root cubes only: every kept cube is forced at level 0
        "max_depth_0": dict(base, xyz=small["xyz"], r=small["r"], max_depth=0),
        "max_depth_1": dict(base, xyz=small["xyz"], r=small["r"], max_depth=1),
        # deeper partition with larger root cubes (h0 = 8 A)
        "max_depth_5": dict(base, xyz=small["xyz"][:30], r=small["r"][:30], max_depth=5),
        # two molecules 120 A apart in one call: two closed components
        "two_far_clusters": dict(base, xyz=np.vstack([a, b + 120.0]), r=np.concatenate([ra, rb])),
        # coincident atoms: every atom twice (the field doubles)
        "coincident_atoms": dict(base, xyz=np.vstack([dup, dup]), r=np.concatenate([small["r"][:20]] * 2)),
        # a ragged count of tiny atoms far below c: no surface anywhere
        "no_surface": dict(base, xyz=rng.uniform(0, 30, (37, 3)), r=np.full(37, 0.1), c=5.0),
        # a non-dyadic min edge
        "min_edge_0.3": dict(base, xyz=small["xyz"][:40], r=small["r"][:40], min_edge=0.3),
    }


@pytest.mark.parametrize("case", sorted(_degenerate_cases()))
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_degenerate_and_edge_inputs(case, mode):
    """Edge cases of the method against the oracle: max_depth 0 (root cubes
    only) and 1, a deep partition, disconnected components, coincident
    atoms, an input without any surface, a non-dyadic min edge."""
    cfg = _degenerate_cases()[case]
    prec = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    m, ref = _mesh_both(cfg, precision_mode=prec)
    _assert_mesh_parity(m, ref)
    assert m.stats["loop_errors"] == 0 and ref["stats"]["loop_errors"] == 0
    if case == "no_surface":
        assert len(m.triangles) == 0
    else:
        assert len(m.triangles) > 0
        check_closed_manifold(m.vertices, m.triangles)


def test_empty_surface_is_success():
    xyz, r = np.array([[0.0, 0.0, 0.0]]), np.array([1.0])
    m = gs.mesh_gaussian_surface(xyz, r, 0.5, 50.0, 1e-3, 2)
    assert len(m.triangles) == 0 and len(m.vertices) == 0


def test_non_finite_input_rejected():
    xyz = np.array([[0.0, np.nan, 0.0]])
    with pytest.raises(gs.GsError) as e:
        gs.mesh_gaussian_surface(xyz, np.array([1.5]), 0.5, 1.0, 1e-3, 2)
    assert e.value.code == -1


@pytest.mark.parametrize("seed", range(4))
def test_grid_triangulation_parity(seed):
    rng = np.random.default_rng(seed)
    vals = rng.standard_normal((9, 9, 9))
    vals[0], vals[-1], vals[:, 0], vals[:, -1], vals[:, :, 0], vals[:, :, -1] = -1, -1, -1, -1, -1, -1
    m = gs.gs_triangulate_grid(vals, 0.0)
    ref = oracle.mesh_grid(vals, 0.0)
    assert np.array_equal(np.sort(m.vertex_keys), ref["vkeys"])
    order = np.argsort(m.vertex_keys)
    assert np.abs(m.vertices[order] - ref["vertices"]).max() < 1e-12
    assert np.array_equal(canonical_triangles(m.vertex_keys, m.triangles),
                          canonical_triangles(ref["vkeys"], ref["triangles"]))
    check_closed_manifold(m.vertices, m.triangles)


def test_mixed_decisions_match_fp64_everywhere(chain100):
    """Debug mode: the mixed form also runs FP64 on every cube; no final
    decision may differ (cube sets are exact by construction)."""
    cfg = chain100
    m = gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                 min_edge=cfg["min_edge"], precision_mode=gs.GS_PREC_MIXED, debug_flags=1)
    st = m.stats
    print("recheck", st["recheck_cubes"], "of", sum(st["examined"]), "reasons", st["recheck_bounds"],
          st["recheck_precision"], st["recheck_zero"], "rank", st["recheck_rank"], "max |A32-A64|/E", st["mixed_err_ratio"],
          "band ratio", st["mixed_band_ratio"], "vertices rechecked", st["recheck_vertices"])
    assert m.mismatches == 0
    # the FP32 error stays inside the band's kappa (1.5e-6)
    assert st["mixed_err_ratio"] < 1.5e-6
    assert st["recheck_cubes"] < 0.2 * sum(st["examined"])


def test_mixed_mesh_parity_chain100(chain100):
    cfg = chain100
    m = gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                 min_edge=cfg["min_edge"], precision_mode=gs.GS_PREC_MIXED)
    ref = oracle.mesh(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"])
    _assert_mesh_parity(m, ref)


def test_field_mixed_close_to_fp64(chain100):
    rng = np.random.default_rng(4)
    xyz, r = chain100["xyz"], chain100["r"]
    pts = xyz[rng.integers(0, len(r), 2000)] + rng.normal(0, 2.0, (2000, 3))
    p32 = gs.gs_eval_field(xyz, r, 0.5, 1.0, pts, precision_mode=gs.GS_PREC_MIXED)
    p64 = oracle.field(xyz, r, 0.5, 1.0, pts)
    assert np.abs(p32 - p64).max() <= 2e-5 * max(1.0, np.abs(p64).max())


def test_mixed_decisions_match_fp64_globular():
    xyz, r = synth.globular(5000, seed=1)
    m = gs.mesh_gaussian_surface(xyz, r, 0.5, 1.0, 1e-3, 3, precision_mode=gs.GS_PREC_MIXED, debug_flags=1)
    st = m.stats
    print("globular5000 recheck", st["recheck_cubes"], "of", sum(st["examined"]), "err ratio",
          st["mixed_err_ratio"], "band ratio", st["mixed_band_ratio"])
    assert m.mismatches == 0
    assert st["mixed_err_ratio"] < 1.5e-6


def test_child_reexpansion_parity_chain100(chain100):
    """Re-expansion reading of the child tensor (FP64 form) against the oracle
    taking the same reading: same cube sets, surface points and topology."""
    cfg = chain100
    m = gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                 min_edge=cfg["min_edge"], child_mode=gs.GS_CHILD_REEXPAND)
    ref = oracle.mesh(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"],
                      child_mode=1)
    for l in range(cfg["max_depth"] + 1):
        assert m.stats["examined"][l] == ref["stats"]["examined"][l]
        assert m.stats["split"][l] == ref["stats"]["split"][l]
    _assert_mesh_parity(m, ref)
    # the holes this reading leaves (a re-expanded child's bounds describe the
    # parent's polynomial, not the field) are the oracle's too
    assert directed_edge_defects(m.triangles) == directed_edge_defects(ref["triangles"])
    with pytest.raises(gs.GsError):
        gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                 min_edge=cfg["min_edge"], child_mode=gs.GS_CHILD_REEXPAND,
                                 precision_mode=gs.GS_PREC_MIXED)


@pytest.mark.parametrize("order,norm", [(1, 0), (0, 1), (0, 2), (1, 2)])
def test_alternative_readings_parity(chain100, order, norm):
    """Literal order of steps 2-3 and the other precision-test norms (FP64
    form) against the oracle taking the same reading.  precision 0.01 makes
    the norms matter at level 2."""
    cfg = dict(chain100, precision=0.01)
    m = gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                 min_edge=cfg["min_edge"], decision_order=order, precision_norm=norm)
    ref = oracle.mesh(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"],
                      order=order, norm=norm)
    for key in ("examined", "split", "accepted", "forced"):
        assert list(m.stats[key][:cfg["max_depth"] + 1]) == list(ref["stats"][key][:cfg["max_depth"] + 1]), key
    assert m.stats["conformity_splits"] == ref["stats"]["conformity_splits"]
    _assert_mesh_parity(m, ref)
    check_closed_manifold(m.vertices, m.triangles)


def test_alternative_readings_rejected_in_mixed_form(chain100):
    """The alternative readings exist in the FP64 form only; unknown values
    are argument errors."""
    cfg = chain100
    cases = [(gs.GS_PREC_MIXED, dict(decision_order=gs.GS_ORDER_LITERAL)),
             (gs.GS_PREC_MIXED, dict(precision_norm=gs.GS_NORM_MAX)),
             (gs.GS_PREC_FP64, dict(precision_norm=7)),
             (gs.GS_PREC_FP64, dict(decision_order=3))]
    for mode, kw in cases:
        with pytest.raises(gs.GsError) as e:
            gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                     min_edge=cfg["min_edge"], precision_mode=mode, **kw)
        assert e.value.code == -1


def test_mixed_form_range_guard():
    """The FP32 form rejects inputs whose weights exp(D r^2) or cutoff factors
    leave the FP32 range (D R^2 > 80); the FP64 form meshes them."""
    xyz, r = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, 0.0]]), np.array([5.0, 5.0])
    D = 3.0   # D r^2 = 75, plus the cutoff exponent 18.4
    with pytest.raises(gs.GsError) as e:
        gs.mesh_gaussian_surface(xyz, r, D, 1.0, 1e-3, 2, min_edge=1.0, precision_mode=gs.GS_PREC_MIXED)
    assert e.value.code == -1
    with pytest.raises(gs.GsError):
        gs.gs_eval_field(xyz, r, D, 1.0, xyz, precision_mode=gs.GS_PREC_MIXED)
    m = gs.mesh_gaussian_surface(xyz, r, D, 1.0, 1e-3, 2, min_edge=1.0)
    check_closed_manifold(m.vertices, m.triangles)


def test_mesh_into_caller_buffers(chain100):
    """The caller-buffer entry point gives the library-allocated mesh bit for
    bit, into pinned host and into device buffers; buffers too small raise
    GS_ERR_CAPACITY with the sizes needed and receive nothing."""
    torch = pytest.importorskip("torch")
    cfg = chain100
    args = (cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"])
    ref = gs.mesh_gaussian_surface(*args, min_edge=cfg["min_edge"], precision_mode=gs.GS_PREC_MIXED)
    nv, nt, nc = len(ref.vertices), len(ref.triangles), len(ref.cube_keys)
    for dev in ("cpu", "cuda"):
        pin = dev == "cpu"
        V = torch.full((nv + 5, 3), -1.0, dtype=torch.float64, device=dev)
        T = torch.full((nt + 5, 3), -1, dtype=torch.int32, device=dev)
        K = torch.zeros(nv + 5, dtype=torch.int64, device=dev)
        C = torch.zeros(nc, dtype=torch.int64, device=dev)
        if pin:
            V, T, K, C = V.pin_memory(), T.pin_memory(), K.pin_memory(), C.pin_memory()
        sizes = gs.mesh_gaussian_surface_into(*args, V, T, K, C, min_edge=cfg["min_edge"],
                                              precision_mode=gs.GS_PREC_MIXED)
        assert sizes == (nv, nt, nc)
        assert np.array_equal(V[:nv].cpu().numpy(), ref.vertices)
        assert np.array_equal(T[:nt].cpu().numpy(), ref.triangles)
        assert np.array_equal(K[:nv].cpu().numpy().view(np.uint64), ref.vertex_keys)
        assert np.array_equal(C.cpu().numpy().view(np.uint64), ref.cube_keys)
        assert (V[nv:] == -1.0).all() and (T[nt:] == -1).all()
    small = torch.full((nv - 1, 3), -1.0, dtype=torch.float64)
    tri = torch.zeros((nt, 3), dtype=torch.int32)
    with pytest.raises(gs.GsError) as e:
        gs.mesh_gaussian_surface_into(*args, small, tri, min_edge=cfg["min_edge"])
    assert e.value.code == -3 and e.value.needed[:2] == (nv, nt)
    assert (small == -1.0).all()


@pytest.mark.parametrize("case", ["one_cell", "clamped_outliers"])
def test_cell_list_crowded_cells(case):
    """The cell list's time does not depend on how atoms crowd into cells
    (stable radix passes, no per-cell sort): 10^5 atoms in a single cell,
    and clamped outliers piling into the edge cells, bit-exact against the
    oracle's cell list."""
    rng = np.random.default_rng(7)
    if case == "one_cell":
        xyz = rng.uniform(0, 1, (100000, 3))
        origin, cell, dims = np.zeros(3), 2.0, np.array([1, 1, 1])
    else:
        xyz = np.concatenate([rng.uniform(-5, 5, (50000, 3)), rng.uniform(-500, 500, (60001, 3))])
        origin, cell, dims = np.array([-5.0, -5.0, -5.0]), 0.7, np.array([15, 15, 15])
    cs, pm = gs.gs_bin_atoms(xyz, cell, origin, dims)
    rs, rp = oracle.cell_list(xyz, cell, origin, dims)
    assert np.array_equal(cs, rs) and np.array_equal(pm, rp)
