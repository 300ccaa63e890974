"""Parity at the benchmark's full size (the 1,000,020-atom assembly, in the
launch configuration bench.py times) on outputs the oracle can compute one
by one, and on properties that hold at any size:
  * sampled cube tensors and decisions (brute force over all atoms);
  * sampled lattice-vertex field values;
  * the mixed-precision mesh equals the FP64 mesh (cube sets and triangle
    topology bit-exact, vertices within 1e-5 A), and is a closed,
    consistently oriented 2-manifold.
Also a whole-mesh parity check against the oracle on a 1,000-atom globular
molecule."""
import numpy as np
import pytest

import oracle
import synth
from meshcheck import canonical_triangles, check_closed_manifold

pytestmark = pytest.mark.gpu

gs = pytest.importorskip("paper_1611_03474_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def big():
    return synth.config("assembly1m")


def _keys_near_atoms(cfg, rng, n_per_level):
    o, nroot, pad = oracle.root_grid(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["min_edge"], cfg["max_depth"])
    keys = []
    for l in range(cfg["max_depth"] + 1):
        h = cfg["min_edge"] * 2 ** (cfg["max_depth"] - l)
        # surface-ish points: atoms pushed out by about their radius
        i = rng.integers(0, len(cfg["r"]), n_per_level)
        d = rng.normal(size=(n_per_level, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        p = cfg["xyz"][i] + d * (cfg["r"][i][:, None] + rng.uniform(-0.5, 1.0, (n_per_level, 1)))
        idx = np.clip(np.floor((p - o) / h).astype(np.int64), 0, (nroot << l) - 1)
        for x, y, z in idx:
            keys.append(int(x) | (int(y) << 18) | (int(z) << 36) | (30 << 54) | (l << 59))
    return np.unique(np.array(keys, dtype=np.uint64))


def test_full_size_sampled_cube_decisions(big):
    cfg = big
    keys = _keys_near_atoms(cfg, np.random.default_rng(31), 60)
    A, b, d = gs.gs_cube_decisions(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"],
                                   cfg["max_depth"], keys)
    rA, rb, rd = oracle.cube_batch(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"],
                                   cfg["max_depth"], keys)
    scale = np.abs(rA).sum(1, keepdims=True) + 1e-300
    assert np.all(np.abs(A - rA) <= 1e-12 * scale)
    assert np.array_equal(d, rd)
    assert (rd != 0).sum() > 20  # the sample reaches kept cubes


def test_full_size_sampled_field(big):
    cfg = big
    rng = np.random.default_rng(32)
    o, nroot, pad = oracle.root_grid(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["min_edge"], cfg["max_depth"])
    i = rng.integers(0, len(cfg["r"]), 400)
    p = cfg["xyz"][i] + rng.normal(0, 1.5, (400, 3))
    p = o + np.round((p - o) / cfg["min_edge"]) * cfg["min_edge"]  # lattice vertices
    phi = gs.gs_eval_field(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], p)
    ref = oracle.field(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], p)
    assert np.allclose(phi, ref, rtol=1e-13, atol=1e-300)
    p32 = gs.gs_eval_field(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], p, precision_mode=gs.GS_PREC_MIXED)
    assert np.abs(p32 - ref).max() <= 2e-6 * max(1.0, np.abs(ref).max())


def _tri_hash(keys, F):
    """order-free fingerprint of each triangle (keys rotated to the smallest), on the GPU"""
    K = torch.from_numpy(keys.astype(np.int64)).cuda()[torch.from_numpy(F.astype(np.int64)).cuda()]
    r = torch.argmin(K, dim=1)
    idx = (r[:, None] + torch.arange(3, device="cuda")[None, :]) % 3
    K = torch.gather(K, 1, idx)
    h = K[:, 0] * 1000003 + K[:, 1] * 998244353 + K[:, 2] * 1000000007
    return torch.sort(h).values


def _closed_manifold_gpu(F):
    F = torch.from_numpy(F.astype(np.int64)).cuda()
    e = torch.cat([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    fwd = e[:, 0] * (1 << 32) + e[:, 1]
    rev = e[:, 1] * (1 << 32) + e[:, 0]
    fs = torch.sort(fwd).values
    assert torch.unique(fs).numel() == fs.numel(), "a directed edge appears twice"
    rs = torch.sort(rev).values
    assert torch.equal(fs, rs), "an edge lacks its opposite"


def test_full_size_mixed_equals_fp64_and_is_manifold(big):
    cfg = big
    args = (cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"])
    m32 = gs.mesh_gaussian_surface(*args, min_edge=cfg["min_edge"], precision_mode=gs.GS_PREC_MIXED)
    m64 = gs.mesh_gaussian_surface(*args, min_edge=cfg["min_edge"], precision_mode=gs.GS_PREC_FP64)
    assert m32.stats["loop_errors"] == 0 and m64.stats["loop_errors"] == 0
    assert np.array_equal(np.sort(m32.cube_keys), np.sort(m64.cube_keys))
    assert np.array_equal(m32.vertex_keys, m64.vertex_keys)  # deterministic ids in both forms
    assert np.abs(m32.vertices - m64.vertices).max() < 1e-5
    assert torch.equal(_tri_hash(m32.vertex_keys, m32.triangles), _tri_hash(m64.vertex_keys, m64.triangles))
    _closed_manifold_gpu(m32.triangles)
    # the paper's O(N) claim, as counts: about 9e3 (cube, atom) terms per atom
    assert m32.stats["pair_terms"] < 2e4 * len(cfg["r"])


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_mesh_parity_globular1000(mode):
    xyz, r = synth.globular(1000, seed=5)
    cfg = dict(D=0.5, c=1.0, precision=1e-3, min_edge=0.25, max_depth=3)
    m = gs.mesh_gaussian_surface(xyz, r, cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                 min_edge=cfg["min_edge"],
                                 precision_mode=gs.GS_PREC_MIXED if mode == "mixed" else gs.GS_PREC_FP64)
    ref = oracle.mesh(xyz, r, cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"])
    assert np.array_equal(np.sort(m.cube_keys), ref["cube_keys"])
    assert np.array_equal(np.sort(m.vertex_keys), ref["vkeys"])
    order = np.argsort(m.vertex_keys)
    assert np.abs(m.vertices[order] - ref["vertices"]).max() < 1e-5
    assert np.array_equal(canonical_triangles(m.vertex_keys, m.triangles),
                          canonical_triangles(ref["vkeys"], ref["triangles"]))
    check_closed_manifold(m.vertices, m.triangles)
