"""Pins for the CPU oracle: each checks it against something other than
itself -- a closed form, a library routine, brute force, or an invariant the
mathematics fixes -- so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails here."""
import numpy as np
import pytest
from scipy import integrate, special

import oracle
import synth
from meshcheck import (area, check_closed_manifold, directed_edge_defects, euler_per_component,
                       key_fields, volume)


def leg(j, t):
    return special.eval_legendre(j, t)


# ---------------------------------------------------------------- section 2.2.1

@pytest.mark.parametrize("xi,a,b,D", [(0.3, -1.0, 1.0, 0.5), (2.7, 0.0, 0.25, 0.9),
                                      (-4.1, -2.0, 0.0, 0.5), (1.0, 1.0, 1.5, 0.9)])
def test_projection_matches_adaptive_quadrature(xi, a, b, D):
    """alpha_j = (2j+1)/(b-a) int_a^b f(x) L_j(t(x)) dx (orthogonal L2 projection)."""
    got = oracle.axis_projection(xi, a, b, D)
    for j in range(4):
        f = lambda x: np.exp(-D * (x - xi) ** 2) * leg(j, (2 * x - (a + b)) / (b - a))
        ref = (2 * j + 1) / (b - a) * integrate.quad(f, a, b, epsabs=1e-16, epsrel=1e-14)[0]
        assert abs(got[j] - ref) <= 1e-13, (j, got[j], ref)


def test_projection_erf_closed_form_alpha0():
    """alpha_0 = mean of f on [a,b] = sqrt(pi/D)/(2(b-a)) (erf(sqrt D (b-xi)) - erf(sqrt D (a-xi)))."""
    for xi, a, b, D in [(0.1, 0.0, 2.0, 0.5), (3.0, 0.0, 0.5, 0.9), (-1.0, -0.5, 0.0, 0.5)]:
        ref = np.sqrt(np.pi / D) / (2 * (b - a)) * (special.erf(np.sqrt(D) * (b - xi)) - special.erf(np.sqrt(D) * (a - xi)))
        assert abs(oracle.axis_projection(xi, a, b, D)[0] - ref) < 1e-14


def test_quadrature_converged_24_vs_48():
    rng = np.random.default_rng(1)
    for _ in range(200):
        D = rng.choice([0.5, 0.9])
        h = rng.choice([2.0, 1.0, 0.5, 0.25])
        a = rng.uniform(-8, 8)
        xi = rng.uniform(-8, 8)
        d = oracle.axis_projection(xi, a, a + h, D, 24) - oracle.axis_projection(xi, a, a + h, D, 48)
        assert np.abs(d).max() < 1e-14


def test_c0_correction_matches_endpoints():
    """eq condition1: the corrected cubic equals f at a and b; only L_2, L_3 change."""
    rng = np.random.default_rng(2)
    for _ in range(100):
        D = rng.choice([0.5, 0.9])
        h = rng.choice([2.0, 1.0, 0.5, 0.25])
        a = rng.uniform(-6, 6)
        xi = rng.uniform(-7, 7)
        b = a + h
        al = oracle.axis_projection(xi, a, b, D)
        at = oracle.axis_coeffs(xi, a, b, D)
        assert np.allclose(at[:2], al[:2], rtol=0, atol=1e-15)
        fa, fb = np.exp(-D * (a - xi) ** 2), np.exp(-D * (b - xi) ** 2)
        assert abs(sum(at) - fb) < 1e-15
        assert abs(at[0] - at[1] + at[2] - at[3] - fa) < 1e-15


def test_single_atom_tensor_is_rank_one_product():
    """A = e^{D r^2} alpha~ (x) beta~ (x) gamma~ for one atom (eq tensor2)."""
    xyz = np.array([[0.3, -0.2, 0.45]])
    r = np.array([1.7])
    D, c = 0.5, 1.0
    lo, h = np.array([0.5, -1.0, 0.0]), 0.5
    A, cnt = oracle.cube_tensor(xyz, r, D, c, lo, h)
    assert cnt == 1
    ax = oracle.axis_coeffs(xyz[0, 0], lo[0], lo[0] + h, D)
    ay = oracle.axis_coeffs(xyz[0, 1], lo[1], lo[1] + h, D)
    az = oracle.axis_coeffs(xyz[0, 2], lo[2], lo[2] + h, D)
    ref = np.exp(D * r[0] ** 2) * np.einsum("i,j,k->ijk", ax, ay, az)
    assert np.allclose(A, ref, rtol=1e-14, atol=0)
    b = oracle.bounds(A)
    assert b[4] == 1 and b[2] < 1e-13 * np.abs(A).sum()


def _ptilde(A, t):
    """P~ on [-1,1]^3 sample points t [n,3] (eq tensor1)."""
    Lx = np.stack([leg(j, t[:, 0]) for j in range(4)], 1)
    Ly = np.stack([leg(j, t[:, 1]) for j in range(4)], 1)
    Lz = np.stack([leg(j, t[:, 2]) for j in range(4)], 1)
    return np.einsum("ijk,ni,nj,nk->n", A.reshape(4, 4, 4), Lx, Ly, Lz)


def test_ptilde_equals_phi_at_cube_corners():
    """With the C0 correction P~ reproduces phi at the 8 corners (up to the
    cutoff difference between box and point distances, < N * 1e-8 c)."""
    cfg = synth.config("chain100")
    xyz, r = cfg["xyz"], cfg["r"]
    lo = xyz[17] + np.array([0.3, -0.8, 0.1])
    for h in (2.0, 0.5):
        A, cnt = oracle.cube_tensor(xyz, r, 0.5, 1.0, lo, h)
        corners = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], float)
        pt = _ptilde(A, 2 * corners - 1)
        ph = oracle.field(xyz, r, 0.5, 1.0, lo + h * corners)
        assert np.abs(pt - ph).max() < 100 * 1e-8


def test_svd_matches_numpy():
    rng = np.random.default_rng(3)
    for m, n in [(4, 16), (4, 4)]:
        for _ in range(50):
            X = rng.standard_normal((m, n)) * rng.choice([1e-3, 1.0, 10.0])
            s, u, v = oracle.svd_rows(X)
            ref = np.linalg.svd(X, compute_uv=False)
            assert np.allclose(s, ref, rtol=1e-13, atol=1e-14 * ref[0])
            assert np.allclose((u.T * s) @ v, X, atol=1e-13 * ref[0])
            assert np.allclose(u @ u.T, np.eye(m), atol=1e-13)


def test_cubic_bounds_brute_force():
    rng = np.random.default_rng(4)
    t = np.linspace(-1, 1, 10001)
    for _ in range(300):
        cf = rng.standard_normal(4) * rng.choice([1e-4, 1.0, 100.0], size=4)
        lo, hi = oracle.cubic_bounds(cf)
        p = sum(cf[j] * leg(j, t) for j in range(4))
        scale = np.abs(cf).sum()
        assert lo <= p.min() + 1e-12 * scale and hi >= p.max() - 1e-12 * scale
        assert p.min() - lo < 1e-6 * scale and hi - p.max() < 1e-6 * scale


def test_bounds_enclose_ptilde_on_dense_sample():
    """[L,U] contains P~ on a 33^3 sample of every cube tried (eqs bound2, bound3)."""
    cfg = synth.config("chain100")
    xyz, r = cfg["xyz"], cfg["r"]
    rng = np.random.default_rng(5)
    g = np.linspace(-1, 1, 33)
    T = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    for _ in range(12):
        i = rng.integers(len(r))
        h = rng.choice([2.0, 1.0, 0.5, 0.25])
        lo = xyz[i] + rng.uniform(-3, 1, 3)
        A, _ = oracle.cube_tensor(xyz, r, 0.5, 1.0, lo, h)
        L, U = oracle.bounds(A)[:2]
        p = _ptilde(A, T)
        tol = 1e-12 * np.abs(A).sum()
        assert L <= p.min() + tol and U >= p.max() - tol


def test_rank_rule_99_percent():
    """eq SVD3: rank = smallest j with sum_{i<=j} sigma_i >= 0.99 sum sigma."""
    rng = np.random.default_rng(6)
    for _ in range(50):
        U, _ = np.linalg.qr(rng.standard_normal((4, 4)))
        V, _ = np.linalg.qr(rng.standard_normal((16, 4)))
        s = np.sort(rng.uniform(0, 1, 4) ** 3)[::-1]
        A1 = (U * s) @ V.T
        b = oracle.bounds(A1.reshape(64))
        cs = np.cumsum(s)
        ref = int(np.argmax(cs >= 0.99 * cs[-1])) + 1
        if np.min(np.abs(cs - 0.99 * cs[-1])) > 1e-9:
            assert b[4] == ref


def test_decision_rules():
    A = np.zeros(64)
    A[0] = 1.0  # constant P~ = 1
    assert oracle.decide(A, 1.0, 1e-3, 0, 3)[0] == oracle.ACCEPT
    assert oracle.decide(A, 1.5, 1e-3, 0, 3)[0] == oracle.DISCARD
    A[16 * 2] = 0.1  # x quadratic term: high-order sum 0.1
    assert oracle.decide(A, 1.0, 1e-3, 0, 3)[0] == oracle.SPLIT
    assert oracle.decide(A, 1.0, 1e-3, 3, 3)[0] == oracle.FORCED
    assert oracle.decide(A, 1.0, 0.2, 0, 3)[0] == oracle.ACCEPT
    assert oracle.decide(np.zeros(64), 1.0, 1e-3, 0, 3)[0] == oracle.DISCARD


# ---------------------------------------------------------------- field

def test_field_single_atom_closed_form_and_cutoff():
    D, c = 0.5, 1.0
    xyz, r = np.array([[0.0, 0.0, 0.0]]), np.array([1.5])
    R2 = 1.5 ** 2 - np.log(1e-8 * c) / D
    pts = np.array([[1.0, 0.5, -0.25], [np.sqrt(R2) * (1 - 1e-9), 0, 0], [np.sqrt(R2) * (1 + 1e-9), 0, 0]])
    phi, grad = oracle.field(xyz, r, D, c, pts, grad=True)
    d2 = (pts ** 2).sum(1)
    ref = np.exp(-D * (d2 - 1.5 ** 2))
    assert abs(phi[0] - ref[0]) < 1e-15 * ref[0]
    assert np.allclose(grad[0], -2 * D * pts[0] * ref[0], rtol=1e-14)
    assert phi[1] > 0 and phi[2] == 0.0


def test_root_grid_alignment():
    cfg = synth.config("chain100")
    o, n, pad = oracle.root_grid(cfg["xyz"], cfg["r"], 0.5, 1.0, 0.25, 3)
    h0 = 2.0
    assert np.all(np.abs(o / h0 - np.round(o / h0)) == 0)
    assert np.all(o <= cfg["xyz"].min(0) - pad) and np.all(o + n * h0 >= cfg["xyz"].max(0) + pad)
    assert abs(pad - np.sqrt(1.8 ** 2 + np.log(1e8) / 0.5)) < 1e-12 or pad < 6.4


# ---------------------------------------------------------------- triangulation on exact trilinear data

def _grid_values(rng, n, c=0.0):
    v = rng.standard_normal((n + 1, n + 1, n + 1))
    v[0, :, :] = v[-1, :, :] = v[:, 0, :] = v[:, -1, :] = v[:, :, 0] = v[:, :, -1] = -1.0
    return v


def _trilinear(vals, p):
    """value of the grid's trilinear interpolant at points p [m,3] (x,y,z)."""
    i = np.minimum(np.floor(p).astype(int), np.array(vals.shape[::-1]) - 2)
    f = p - i
    out = np.zeros(len(p))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) * (f[:, 2] if dz else 1 - f[:, 2])
                out += w * vals[i[:, 2] + dz, i[:, 1] + dy, i[:, 0] + dx]
    return out


@pytest.mark.parametrize("seed", range(6))
def test_random_trilinear_grid_closed_manifold(seed):
    """Random corner values (all 256 sign cases, ambiguous faces, tunnels,
    critical points): the mesh is closed, 2-manifold and every point lies on
    the trilinear surface g = c."""
    rng = np.random.default_rng(seed)
    vals = _grid_values(rng, 7)
    m = oracle.mesh_grid(vals, 0.0)
    V, F = m["vertices"], m["triangles"]
    assert m["stats"]["loop_errors"] == 0
    assert len(F) > 0
    check_closed_manifold(V, F)
    # points on the surface: evaluate inside the cube that produced them (any
    # containing cube gives the same value on shared faces)
    g = _trilinear(vals, np.minimum(V, 7 - 1e-12))
    assert np.abs(g).max() < 1e-12
    assert volume(V, F) > 0  # outward orientation (inside = g >= c)
    types = {key_fields(k)["type"] for k in m["vkeys"]}
    assert any(t >= 20 for t in types), "no critical points exercised"


def test_all_256_sign_cases_single_cube():
    """Each of the 256 inside/outside patterns of one cube, embedded in an
    outside shell, meshes to a closed manifold."""
    rng = np.random.default_rng(7)
    for pattern in range(256):
        vals = -np.ones((4, 4, 4))
        for v in range(8):
            bx, by, bz = v & 1, (v >> 1) & 1, (v >> 2) & 1
            mag = rng.uniform(0.2, 1.0)
            vals[1 + bz, 1 + by, 1 + bx] = mag if (pattern >> v) & 1 else -mag
        m = oracle.mesh_grid(vals, 0.0)
        if pattern == 0:
            assert len(m["triangles"]) == 0
            continue
        assert m["stats"]["loop_errors"] == 0, pattern
        check_closed_manifold(m["vertices"], m["triangles"])


def _trilinear_grad(vals, p, cube):
    f = p - cube
    g = np.zeros((len(p), 3))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                v = vals[cube[:, 2] + dz, cube[:, 1] + dy, cube[:, 0] + dx]
                wx = f[:, 0] if dx else 1 - f[:, 0]
                wy = f[:, 1] if dy else 1 - f[:, 1]
                wz = f[:, 2] if dz else 1 - f[:, 2]
                g[:, 0] += v * (1 if dx else -1) * wy * wz
                g[:, 1] += v * wx * (1 if dy else -1) * wz
                g[:, 2] += v * wx * wy * (1 if dz else -1)
    return g


def test_pieces_single_valued():
    """Each piece is single-valued along x, y and z (section 2.3): no fold
    curve (where a partial derivative of g vanishes on the surface) crosses
    its interior, so every partial derivative of g keeps one sign over the
    piece.  Checked at the piece's cube-edge points, none of which lies on a
    fold."""
    rng = np.random.default_rng(8)
    vals = _grid_values(rng, 6)
    m = oracle.mesh_grid(vals, 0.0)
    V, F, piece, K = m["vertices"], m["triangles"], m["tri_piece"], m["vkeys"]
    types = np.array([key_fields(k)["type"] for k in K])
    checked = 0
    for pc in np.unique(piece):
        tri = F[piece == pc]
        vid = np.unique(tri.ravel())
        cube = np.floor(V[vid].min(0) + 1e-12).astype(int)
        ev = vid[types[vid] <= 2]
        if len(ev) < 2:
            continue
        gr = _trilinear_grad(vals, V[ev], np.tile(cube, (len(ev), 1)))
        for ax in range(3):
            d = gr[:, ax]
            big = np.abs(d) > 1e-9 * np.abs(gr).max()
            if big.sum() >= 2:
                assert np.all(d[big] > 0) or np.all(d[big] < 0), (pc, ax)
                checked += 1
    assert checked > 100


# ---------------------------------------------------------------- whole path

def _sphere_tol(D, R, h):
    """radial error bound: trilinear interpolation error h^2/8 |phi''| per axis
    over |grad phi| at the sphere (phi = c there), x1.5 margin."""
    return 1.5 * h * h / 8 * (4 * D * D * R * R + 2 * D) / (2 * D * R)


def test_single_atom_sphere():
    """One atom: the surface is the sphere of radius sqrt(r^2 - ln(c)/D)."""
    D, c, rr = 0.5, 1.0, 1.5
    xyz, r = np.array([[0.1, 0.2, 0.3]]), np.array([rr])
    m = oracle.mesh(xyz, r, D, c, 1e-3, 0.25, 3)
    V, F = m["vertices"], m["triangles"]
    check_closed_manifold(V, F)
    assert list(euler_per_component(V, F).values()) == [2]
    rad = np.linalg.norm(V - xyz[0], axis=1)
    R = np.sqrt(rr ** 2 - np.log(c) / D)
    assert np.abs(rad - R).max() < _sphere_tol(D, R, 0.25)
    assert abs(volume(V, F) - 4 / 3 * np.pi * R ** 3) / (4 / 3 * np.pi * R ** 3) < 0.02
    assert abs(area(V, F) - 4 * np.pi * R ** 2) / (4 * np.pi * R ** 2) < 0.02


def test_single_atom_sphere_other_isovalue():
    D, c, rr = 0.9, 0.5, 1.7
    xyz, r = np.array([[-0.3, 0.05, 0.2]]), np.array([rr])
    m = oracle.mesh(xyz, r, D, c, 1e-3, 0.25, 3)
    V = m["vertices"]
    check_closed_manifold(V, m["triangles"])
    R = np.sqrt(rr ** 2 - np.log(c) / D)
    assert np.abs(np.linalg.norm(V - xyz[0], axis=1) - R).max() < _sphere_tol(D, R, 0.25)


def test_two_equal_atoms_mirror_symmetry():
    """Two equal atoms mirrored in the lattice plane x = 0: the cube set and
    the vertex set are mirror images."""
    d = 1.3
    xyz = np.array([[-d, 0.37, -0.21], [d, 0.37, -0.21]])
    r = np.array([1.5, 1.5])
    m = oracle.mesh(xyz, r, 0.5, 1.0, 1e-3, 0.25, 3)
    o, n, pad = oracle.root_grid(xyz, r, 0.5, 1.0, 0.25, 3)
    assert abs(o[0] + (o[0] + n[0] * 2.0)) == 0  # grid symmetric about x = 0
    keys = m["cube_keys"].astype(np.int64)
    lvl = keys >> 59
    x = keys & 0x3FFFF
    nl = n[0] << lvl
    mirrored = (keys & ~np.int64(0x3FFFF)) | (nl - 1 - x)
    assert set(mirrored.tolist()) == set(keys.tolist())
    V = m["vertices"]
    # every surface point's mirror image is a surface point (to 1e-9 A; the
    # two sides round t and 1 - t differently)
    W = V * np.array([-1.0, 1.0, 1.0])
    order = np.lexsort(V.T[::-1])
    Vs = V[order]
    for w in W:
        k = np.searchsorted(Vs[:, 0], w[0] - 1e-9)
        found = False
        while k < len(Vs) and Vs[k, 0] <= w[0] + 1e-9:
            if np.abs(Vs[k] - w).max() < 1e-9:
                found = True
                break
            k += 1
        assert found
    check_closed_manifold(V, m["triangles"])


def test_chain100_closed_manifold_and_level_invariants():
    cfg = synth.config("chain100")
    m = oracle.mesh(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"])
    st = m["stats"]
    V, F = m["vertices"], m["triangles"]
    assert st["loop_errors"] == 0
    check_closed_manifold(V, F)
    # counts add up level by level
    for l in range(cfg["max_depth"] + 1):
        assert st["examined"][l] == st["discarded"][l] + st["accepted"][l] + st["forced"][l] + st["split"][l]
        if l + 1 <= cfg["max_depth"]:
            assert st["examined"][l + 1] == 8 * st["split"][l]
    # surface points are near phi = c (trilinear interpolation error at 0.25 A)
    phi = oracle.field(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], V)
    assert np.abs(phi - cfg["c"]).max() < 0.05
    assert volume(V, F) > 0


@pytest.mark.parametrize("c8", range(8))
def test_child_reexpansion_reproduces_parent_polynomial(c8):
    """Re-expansion reading of the child tensor (section 2.2): a cubic in each
    variable restricted to a half box is again such a cubic, so the child's
    coefficients must reproduce the parent's P~ at every point of the child
    box (t_parent = (t_child + s) / 2 with s = -1 for the lower half)."""
    rng = np.random.default_rng(40 + c8)
    A = rng.standard_normal((4, 4, 4)) * np.exp(-np.add.outer(np.add.outer(np.arange(4), np.arange(4)), np.arange(4)))
    B = oracle.child_reexpand(A, c8)
    s = np.array([1.0 if (c8 >> a) & 1 else -1.0 for a in range(3)])
    t = rng.uniform(-1, 1, (500, 3))
    ref = _ptilde(A, (t + s) / 2)
    assert np.abs(_ptilde(B, t) - ref).max() < 1e-13 * np.abs(A).sum()
    # the constant alone stays a constant; x alone halves its slope on the child
    E = np.zeros((4, 4, 4))
    E[1, 0, 0] = 1.0
    Bx = oracle.child_reexpand(E, c8)
    expect = np.zeros((4, 4, 4))
    expect[0, 0, 0], expect[1, 0, 0] = s[0] / 2, 0.5
    assert np.abs(Bx - expect).max() < 1e-15


def test_child_reexpansion_reading_leaves_holes():
    """The two readings of the child tensor (section 2.2) differ in kind: with
    the children re-projected from the atoms the chain mesh is closed; with
    the parent's polynomial re-expanded, a child's bounds describe that
    polynomial rather than phi, some surface cubes are discarded as empty and
    the mesh has open edges.  This is why the projection reading is the
    default."""
    cfg = synth.config("chain100")
    args = (cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"])
    a = oracle.mesh(*args, child_mode=0)
    b = oracle.mesh(*args, child_mode=1)
    assert directed_edge_defects(a["triangles"]) == 0
    assert directed_edge_defects(b["triangles"]) > 0
    assert b["stats"]["pair_terms"] < a["stats"]["pair_terms"]


def test_precision_norms_match_numpy():
    """The three sizes of the higher-than-linear coefficients (section 2.2.3
    leaves the norm open) against numpy's own norms of the same entries."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((4, 4, 4))
    high = A[np.maximum.outer(np.maximum.outer(np.arange(4), np.arange(4)), np.arange(4)) >= 2]
    assert high.size == 56
    assert np.isclose(oracle.high_norm(A, 0), np.linalg.norm(high, 1), rtol=1e-15)
    assert oracle.high_norm(A, 1) == np.linalg.norm(high, np.inf)
    assert np.isclose(oracle.high_norm(A, 2), np.linalg.norm(high), rtol=1e-15)
    # a trilinear tensor has no higher-order part under any norm
    T = np.zeros((4, 4, 4))
    T[:2, :2, :2] = rng.standard_normal((2, 2, 2))
    assert all(oracle.high_norm(T, n) == 0 for n in range(3))


def test_literal_decision_order():
    """Steps 2-3 of section 2.2 as printed: a child whose polynomial is
    (near) trilinear is accepted without its bound test; a root cube that
    passes the bound test is divided; a cube without atoms is discarded."""
    c, prec = 1.0, 1e-3
    A = np.zeros((4, 4, 4))
    A[0, 0, 0] = 0.2          # constant 0.2: bounds [0.2, 0.2] miss c = 1
    assert oracle.decide(A, c, prec, 1, 3)[0] == 0             # bounds first: discard
    assert oracle.decide(A, c, prec, 1, 3, order=1)[0] == 1    # literal: trilinear child, accept
    assert oracle.decide(A, c, prec, 0, 3, order=1)[0] == 0    # root: bound test
    A[1, 0, 0] = 1.0          # 0.2 + x spans [-0.8, 1.2]: straddles c
    assert oracle.decide(A, c, prec, 0, 3)[0] == 1
    assert oracle.decide(A, c, prec, 0, 3, order=1)[0] == 2    # a kept root is divided
    assert oracle.decide(A, c, prec, 2, 3, order=1)[0] == 1
    A[2, 2, 2] = 0.5          # high part over the bound: bound test, then divide or force
    assert oracle.decide(A, c, prec, 2, 3, order=1)[0] == 2
    assert oracle.decide(A, c, prec, 3, 3, order=1)[0] == 3
    assert oracle.decide(np.zeros((4, 4, 4)), c, prec, 2, 3, order=1)[0] == 0


def test_precision_norm_split_sets_are_nested():
    """max |.| <= Euclidean <= sum of |.|, so a cube split under a smaller
    norm is split under every larger one: the examined and split counts are
    ordered level by level, and each mesh stays a closed manifold."""
    cfg = dict(synth.config("chain100"), precision=0.01)
    args = (cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"])
    ms = [oracle.mesh(*args, norm=n) for n in (1, 2, 0)]
    for lo, hi in zip(ms, ms[1:]):
        assert np.all(np.asarray(lo["stats"]["split"]) <= np.asarray(hi["stats"]["split"]))
        assert np.all(np.asarray(lo["stats"]["examined"]) <= np.asarray(hi["stats"]["examined"]))
    assert sum(ms[0]["stats"]["split"]) < sum(ms[2]["stats"]["split"])
    for m in ms:
        check_closed_manifold(m["vertices"], m["triangles"])


def test_literal_order_mesh_closed():
    """Under the literal order the extra cubes are trilinear children that
    miss the surface: the surface cubes and the mesh stay closed."""
    cfg = dict(synth.config("chain100"), precision=0.01)
    args = (cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"])
    a = oracle.mesh(*args)
    b = oracle.mesh(*args, order=1)
    check_closed_manifold(b["vertices"], b["triangles"])
    assert sum(b["stats"]["accepted"][1:]) >= sum(a["stats"]["accepted"][1:])


def test_child_reexpansion_composes_over_levels():
    """Re-expanding to child c1 and then to its child c2 gives the parent's
    polynomial on that grandchild box, t_parent = ((t + s2)/2 + s1)/2."""
    rng = np.random.default_rng(77)
    A = rng.standard_normal((4, 4, 4))
    t = rng.uniform(-1, 1, (300, 3))
    for c1, c2 in ((0, 7), (5, 2), (3, 3)):
        B = oracle.child_reexpand(oracle.child_reexpand(A, c1), c2)
        s1 = np.array([1.0 if (c1 >> a) & 1 else -1.0 for a in range(3)])
        s2 = np.array([1.0 if (c2 >> a) & 1 else -1.0 for a in range(3)])
        ref = _ptilde(A, ((t + s2) / 2 + s1) / 2)
        assert np.abs(_ptilde(B, t) - ref).max() < 1e-13 * np.abs(A).sum()


def test_corner_straddle_implies_keep():
    """The first passes of the estimate rest on the bounds enclosing P~: a cube
    whose corner values of P~ (L_n(+-1) = (+-1)^n, so signed coefficient
    sums) straddle c has L <= min corner and max corner <= U, so the bound
    test keeps it.  Checked on the oracle's tensors, bounds and decisions for
    cubes of every level around the chain."""
    cfg = synth.config("chain100")
    rng = np.random.default_rng(5)
    o, nroot, pad = oracle.root_grid(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["min_edge"], cfg["max_depth"])
    keys = []
    for l in range(cfg["max_depth"] + 1):
        h = cfg["min_edge"] * 2 ** (cfg["max_depth"] - l)
        centres = cfg["xyz"][rng.integers(0, len(cfg["r"]), 400)] + rng.normal(0, 1.5, (400, 3))
        idx = np.clip(np.floor((centres - o) / h).astype(np.int64), 0, (nroot << l) - 1)
        keys += [int(x) | (int(y) << 18) | (int(z) << 36) | (30 << 54) | (l << 59) for x, y, z in idx]
    keys = np.unique(np.array(keys, dtype=np.uint64))
    A, b, d = oracle.cube_batch(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"],
                                cfg["max_depth"], keys)
    s = np.array([[1.0 if (v >> a) & 1 else -1.0 for a in range(3)] for v in range(8)])
    j = np.arange(4)
    corners = np.einsum("qjkl,vj,vk,vl->qv", A.reshape(-1, 4, 4, 4), s[:, :1] ** j, s[:, 1:2] ** j, s[:, 2:] ** j)
    lo, hi = corners.min(1), corners.max(1)
    tot = np.abs(A).sum(1)
    straddle = (hi - cfg["c"] > 1e-12 * tot) & (cfg["c"] - lo > 1e-12 * tot)
    assert straddle.sum() > 100 and (~straddle).sum() > 100
    assert np.all(d[straddle] != 0)                                   # never discarded
    assert np.all(b[straddle, 0] <= lo[straddle] + 1e-12 * tot[straddle])
    assert np.all(hi[straddle] <= b[straddle, 1] + 1e-12 * tot[straddle])
    # and the decision is the one the first passes take without the SVD
    t = np.arange(64)
    high_mask = ((t >> 4) >= 2) | (((t >> 2) & 3) >= 2) | ((t & 3) >= 2)
    high = np.abs(A[:, high_mask]).sum(1)
    level = (keys >> np.uint64(59)).astype(int)
    expect = np.where(high <= cfg["precision"], 1, np.where(level >= cfg["max_depth"], 3, 2))
    assert np.array_equal(d[straddle], expect[straddle])


def test_threaded_oracle_equals_single_thread():
    """The oracle's parallel loops (cube tensors and decisions, lattice
    values, per-cube triangulation) give the same mesh, cube set and
    statistics on 1 thread and on several: each cube's or point's result
    depends on it alone and results are collected in input order."""
    cfg = synth.config("chain100")
    args = (cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], 0.05, cfg["min_edge"], cfg["max_depth"])
    try:
        oracle.set_threads(1)
        one = oracle.mesh(*args)
        if oracle.set_threads(4) < 2:
            pytest.skip("oracle built without OpenMP")
        many = oracle.mesh(*args)
    finally:
        oracle.set_threads(0)
    for k in ("vertices", "vkeys", "triangles", "cube_keys", "pre_keys", "lattice_keys", "lattice_phi"):
        assert np.array_equal(one[k], many[k]), k
    assert one["stats"] == many["stats"]
