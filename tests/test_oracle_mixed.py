"""Pins of the oracle's reading of section 2.3 for cubes of different sizes
(the points of the neighbouring cubes that lie in the current cube are taken
into its loops).  Reading: accepted cubes keep their sizes, except that
cubes sharing a face or an edge differ by at most one level and a lattice
vertex whose field value and coarser-cube interpolant lie on different sides
of c splits the coarser cube; vertices on a coarser cube's face or edge take
its interpolant (constrained values).  The checks below use only the
oracle's outputs (cube keys, lattice keys, field and constrained values,
mesh) and mathematics that holds for any correct implementation:
continuity of the piecewise trilinear function, g = c at every surface
point in every cube holding it, the closed-manifold invariants, and
adaptivity (coarse surface cubes remain)."""
import numpy as np
import pytest

import oracle
import synth
from meshcheck import check_closed_manifold, directed_edge_defects

TYPE_CUBE = 30


def _decode(keys):
    k = np.asarray(keys, dtype=np.uint64).astype(np.int64)
    return np.stack([k & 0x3FFFF, (k >> 18) & 0x3FFFF, (k >> 36) & 0x3FFFF], 1), (k >> 59)


def _ckey(x, y, z, l):
    return int(x) | (int(y) << 18) | (int(z) << 36) | (TYPE_CUBE << 54) | (int(l) << 59)


class Field:
    """The piecewise trilinear function of the final cubes: each cube's
    trilinear interpolant (eq linear1) of the constrained values at its
    corners."""

    def __init__(self, m, md):
        self.md = md
        self.cubes = set(int(k) for k in m["cube_keys"])
        lk = np.asarray(m["lattice_keys"]).astype(np.int64)
        self.val = dict(zip(lk.tolist(), m["lattice_psi"].tolist()))
        self.phi = dict(zip(lk.tolist(), m["lattice_phi"].tolist()))

    def corner(self, X):
        return self.val[int(X[0]) | (int(X[1]) << 18) | (int(X[2]) << 36) | (31 << 54)]

    def g(self, q, l, f):
        """cube q (level-l indices) at local coordinates f in [0,1]^3"""
        s = 1 << (self.md - l)
        tot = 0.0
        for v in range(8):
            b = [(v >> a) & 1 for a in range(3)]
            w = 1.0
            for a in range(3):
                w *= f[a] if b[a] else 1.0 - f[a]
            tot += w * self.corner([(q[a] + b[a]) * s for a in range(3)])
        return tot

    def holders(self, U):
        """final cubes whose closed box holds the point at finest-lattice
        coordinates U: (indices, level, local coordinates)"""
        out = []
        for l in range(self.md + 1):
            s = 1 << (self.md - l)
            cand = []
            for a in range(3):
                u = U[a] / s
                fl = np.floor(u)
                cand.append([int(fl)] + ([int(fl) - 1] if u == fl else []))
            for x in cand[0]:
                for y in cand[1]:
                    for z in cand[2]:
                        if _ckey(x, y, z, l) in self.cubes:
                            q = (x, y, z)
                            out.append((q, l, [U[a] / s - q[a] for a in range(3)]))
        return out


def _mesh(name, prec, md=3, me=0.25, conform=0):
    if name == "chain100":
        cfg = synth.config("chain100")
        xyz, r, D = cfg["xyz"], cfg["r"], cfg["D"]
    elif name == "chain30":
        xyz, r = synth.chain(30, seed=7)
        D = 0.9
    else:
        xyz, r = synth.globular(1000, seed=5)
        D = 0.5
    m = oracle.mesh(xyz, r, D, 1.0, prec, me, md, conform=conform)
    o, _, _ = oracle.root_grid(xyz, r, D, 1.0, me, md)
    return m, o


CASES = [("chain100", 0.05, 3, 0.25), ("chain30", 0.2, 3, 0.25), ("chain30", 0.05, 4, 0.125)]


@pytest.mark.parametrize("name,prec,md,me", CASES)
def test_mixed_levels_closed_manifold_and_coarse_cubes_kept(name, prec, md, me):
    """Meshes whose final cubes span two levels are closed 2-manifolds with
    no loop errors, and surface cubes of the coarser level remain (the
    equal-size reading splits every one of them)."""
    m, _ = _mesh(name, prec, md, me)
    st = m["stats"]
    assert st["loop_errors"] == 0
    check_closed_manifold(m["vertices"], m["triangles"])
    F = Field(m, md)
    idx, lvl = _decode(m["cube_keys"])
    levels = sorted(set(lvl.tolist()))
    assert len(levels) >= 2
    coarse_surface = 0
    for q, l in zip(idx, lvl):
        if l == levels[-1]:
            continue
        s = 1 << (md - l)
        g = [F.corner([(q[a] + ((v >> a) & 1)) * s for a in range(3)]) for v in range(8)]
        coarse_surface += (min(g) < 1.0 <= max(g))
    assert coarse_surface >= 100
    assert st["constrained_vertices"] > 0
    # the equal-size reading splits every coarse cube next to a finer one
    eq, _ = _mesh(name, prec, md, me, conform=1)
    assert eq["stats"]["conformity_splits"] > st["conformity_splits"] + st["agreement_splits"]
    assert directed_edge_defects(eq["triangles"]) == 0


@pytest.mark.parametrize("name,prec,md,me", CASES[:2])
def test_constrained_field_is_continuous_across_mixed_faces(name, prec, md, me):
    """Two final cubes of different levels that share a face region have
    the same trilinear values on it (at the finer face's corners, centre and
    random points): the constrained values make g continuous.  Free
    vertices keep the field value."""
    m, _ = _mesh(name, prec, md, me)
    F = Field(m, md)
    rng = np.random.default_rng(2)
    idx, lvl = _decode(m["cube_keys"])
    pairs = 0
    for q, l in zip(idx.tolist(), lvl.tolist()):
        if l == 0:
            continue
        for a in range(3):
            for sd in (0, 1):
                # the coarser cube across this face, if any
                n = list(q)
                n[a] += 1 if sd else -1
                if min(n) < 0:
                    continue
                p = [v >> 1 for v in n]
                if _ckey(*p, l - 1) not in F.cubes:
                    continue
                for _ in range(4):
                    f = rng.uniform(0, 1, 3)
                    f[a] = float(sd)
                    s = 1 << (md - l)
                    U = [(q[b] + f[b]) * s for b in range(3)]
                    S = 2 * s
                    fc = [U[b] / S - p[b] for b in range(3)]
                    assert abs(F.g(q, l, f) - F.g(p, l - 1, fc)) < 1e-12
                pairs += 1
    assert pairs > 50
    # constrained vertices are exactly those off the corners of the coarsest
    # cube touching them; all others keep phi
    diff = np.flatnonzero(m["lattice_psi"] != m["lattice_phi"])
    assert 0 < len(diff) <= m["stats"]["constrained_vertices"]


@pytest.mark.parametrize("name,prec,md,me", CASES[:2])
def test_surface_points_on_every_holding_cube_level_set(name, prec, md, me):
    """Every mesh vertex satisfies g = c (to rounding) in every final cube
    whose closed box holds it: edge points, the finer neighbours' points taken
    into a coarser cube's face curve and the coarser neighbour's extreme
    points taken into a finer cube's all lie on the shared level curve."""
    m, o = _mesh(name, prec, md, me)
    F = Field(m, md)
    U = (m["vertices"] - o) / me
    worst, multi = 0.0, 0
    for i in range(len(U)):
        hs = F.holders(U[i])
        assert hs, "a surface point outside every final cube"
        if len({h[1] for h in hs}) > 1:
            multi += 1
        for q, l, f in hs:
            worst = max(worst, abs(F.g(q, l, f) - 1.0))
    assert worst < 1e-9
    assert multi > 100  # points shared by cubes of two levels were checked


def test_no_sign_disagreement_left():
    """After the splits no constrained value lies on the other side of c from
    the field value at its vertex, and the splits did happen (the chain at
    precision 0.05 has such vertices before them)."""
    m, _ = _mesh("chain100", 0.05)
    c = 1.0
    assert np.all((m["lattice_psi"] >= c) == (m["lattice_phi"] >= c))
    assert m["stats"]["agreement_splits"] > 0


def test_mixed_levels_mirror_symmetry():
    """Two equal atoms mirrored in the lattice plane x = 0, at a precision
    that accepts cubes on two levels: the cube sets are mirror images and
    every surface point has its mirror image among the surface points."""
    d = 1.3
    xyz = np.array([[-d, 0.37, -0.21], [d, 0.37, -0.21]])
    r = np.array([1.5, 1.5])
    m = oracle.mesh(xyz, r, 0.5, 1.0, 0.05, 0.25, 3)
    o, n, _ = oracle.root_grid(xyz, r, 0.5, 1.0, 0.25, 3)
    assert o[0] + (o[0] + n[0] * 2.0) == 0
    keys = m["cube_keys"].astype(np.int64)
    lvl = keys >> 59
    assert len(set(lvl.tolist())) >= 2
    x = keys & 0x3FFFF
    mirrored = (keys & ~np.int64(0x3FFFF)) | ((n[0] << lvl) - 1 - x)
    assert set(mirrored.tolist()) == set(keys.tolist())
    V = m["vertices"]
    W = V * np.array([-1.0, 1.0, 1.0])
    order = np.lexsort(V.T[::-1])
    Vs = V[order]
    for w in W:
        j = np.searchsorted(Vs[:, 0], w[0] - 1e-9)
        k = j
        found = False
        while k < len(Vs) and Vs[k, 0] <= w[0] + 1e-9:
            if np.abs(Vs[k] - w).max() < 1e-9:
                found = True
                break
            k += 1
        assert found
    check_closed_manifold(V, m["triangles"])


def test_gradient_through_constrained_values():
    """The oracle's gradient on a mesh with constrained vertices against
    central differences of the same loss (components whose +-h meshes change
    cubes or topology are skipped): the adjoint of a constrained value is
    passed to the corners it interpolates."""
    from meshcheck import key_normal_weights, surface_loss, surface_loss_grad
    xyz, r = synth.chain(12, seed=3)
    D, prec, me, md = 0.5, 0.05, 0.25, 3

    def run(x, rr, DD):
        return oracle.mesh(x, rr, DD, 1.0, prec, me, md)

    m = run(xyz, r, D)
    assert m["stats"]["constrained_vertices"] > 0
    W = key_normal_weights(m["vkeys"])
    gx, gr, gD = oracle.mesh_grad(xyz, r, D, 1.0, prec, me, md, surface_loss_grad(m["vertices"], m["triangles"], W))
    same = lambda a, b: (np.array_equal(a["vkeys"], b["vkeys"]) and np.array_equal(a["triangles"], b["triangles"])
                         and np.array_equal(a["cube_keys"], b["cube_keys"]))
    h = 1e-6
    rng = np.random.default_rng(1)
    checked = 0
    for i in rng.choice(len(r), 6, replace=False):
        for q in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[i, q] += h
            xm[i, q] -= h
            mp, mm = run(xp, r, D), run(xm, r, D)
            if not (same(mp, m) and same(mm, m)):
                continue
            fd = (surface_loss(mp["vertices"], mp["triangles"], W) - surface_loss(mm["vertices"], mm["triangles"], W)) / (2 * h)
            assert abs(fd - gx[i, q]) <= 2e-6 * max(1.0, abs(gx[i, q])), (i, q, fd, gx[i, q])
            checked += 1
    assert checked >= 8
