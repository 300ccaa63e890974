"""Mesh invariants used as pins: closed 2-manifold (every edge in exactly two
triangles, with opposite orientations), one link loop per vertex, Euler
characteristic per connected component, outward orientation, areas/volumes."""
from collections import defaultdict

import numpy as np


def key_fields(k):
    k = int(k)
    return dict(x=k & 0x3FFFF, y=(k >> 18) & 0x3FFFF, z=(k >> 36) & 0x3FFFF,
                type=(k >> 54) & 31, level=k >> 59)


def directed_edge_defects(F):
    """Count directed edges whose multiplicity is not 1 or whose reverse is missing."""
    F = np.asarray(F, dtype=np.int64)
    if len(F) == 0:
        return 0
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    key = e[:, 0] * (1 << 32) + e[:, 1]
    rkey = e[:, 1] * (1 << 32) + e[:, 0]
    u, cnt = np.unique(key, return_counts=True)
    bad = int((cnt != 1).sum())
    missing = int((~np.isin(rkey, u)).sum())
    return bad + missing


def link_defects(F, nv):
    """Vertices whose neighbourhood is not a single closed loop (condition b)."""
    nxt = defaultdict(list)
    for a, b, c in np.asarray(F, dtype=np.int64):
        nxt[a].append((b, c))
        nxt[b].append((c, a))
        nxt[c].append((a, b))
    bad = 0
    for v, pairs in nxt.items():
        succ = {}
        dup = False
        for p, q in pairs:
            if p in succ:
                dup = True
            succ[p] = q
        if dup:
            bad += 1
            continue
        start = pairs[0][0]
        cur, steps = start, 0
        while True:
            cur = succ.get(cur)
            steps += 1
            if cur is None or steps > len(pairs):
                break
            if cur == start:
                break
        if cur != start or steps != len(pairs):
            bad += 1
    return bad


def components(F, nv):
    parent = np.arange(nv)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b, c in np.asarray(F, dtype=np.int64):
        for p, q in ((a, b), (b, c)):
            rp, rq = find(p), find(q)
            if rp != rq:
                parent[rp] = rq
    roots = np.array([find(i) for i in range(nv)])
    return roots


def euler_per_component(V, F):
    F = np.asarray(F, dtype=np.int64)
    roots = components(F, len(V))
    used = np.zeros(len(V), bool)
    used[F.ravel()] = True
    out = {}
    froot = roots[F[:, 0]]
    for r in np.unique(froot):
        tri = F[froot == r]
        verts = np.unique(tri.ravel())
        e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
        e = np.sort(e, axis=1)
        ne = len(np.unique(e[:, 0] * (1 << 32) + e[:, 1]))
        out[int(r)] = len(verts) - ne + len(tri)
    return out


def volume(V, F):
    V = np.asarray(V)
    F = np.asarray(F, dtype=np.int64)
    return float(np.einsum("ij,ij->i", V[F[:, 0]], np.cross(V[F[:, 1]], V[F[:, 2]])).sum() / 6.0)


def area(V, F):
    V = np.asarray(V)
    F = np.asarray(F, dtype=np.int64)
    return float(np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1).sum() / 2.0)


def canonical_triangles(keys, F):
    """Triangles as key triples rotated to start at the smallest key, sorted."""
    K = np.asarray(keys, dtype=np.uint64)[np.asarray(F, dtype=np.int64)]
    r = np.argmin(K, axis=1)
    idx = (r[:, None] + np.arange(3)[None, :]) % 3
    K = np.take_along_axis(K, idx, axis=1)
    order = np.lexsort((K[:, 2], K[:, 1], K[:, 0]))
    return K[order]


def check_closed_manifold(V, F):
    assert directed_edge_defects(F) == 0, "edge not shared by exactly two oppositely oriented triangles"
    assert link_defects(F, len(V)) == 0, "vertex link is not a single loop"


# ---------------------------------------------------------------- differentiation
def key_normal_weights(keys, seed=0):
    """w_v ~ N(0,1)^3 per vertex, drawn from a counter-based hash of the
    vertex key (so that two meshes with the same keys get the same weights
    whatever their vertex order): splitmix64 of (key, seed, axis), Box-Muller."""
    k = np.asarray(keys, dtype=np.uint64)
    M = np.uint64(0xFFFFFFFFFFFFFFFF)

    def mix(x):
        x = (x + np.uint64(0x9E3779B97F4A7C15)) & M
        x = ((x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & M
        x = ((x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & M
        return x ^ (x >> np.uint64(31))

    out = np.zeros((len(k), 3))
    with np.errstate(over="ignore"):
        for q in range(3):
            a = mix(k ^ mix(np.uint64(seed * 6 + 2 * q)))
            b = mix(k ^ mix(np.uint64(seed * 6 + 2 * q + 1)))
            u1 = ((a >> np.uint64(11)).astype(np.float64) + 0.5) / 2.0 ** 53
            u2 = ((b >> np.uint64(11)).astype(np.float64) + 0.5) / 2.0 ** 53
            out[:, q] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return out


def surface_loss(vertices, triangles, W):
    """L = sum_v W_v . p_v + enclosed volume + surface area (plain numpy)."""
    v, t = np.asarray(vertices), np.asarray(triangles)
    p0, p1, p2 = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    vol = np.einsum("ij,ij->", p0, np.cross(p1, p2)) / 6.0
    area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1).sum()
    return float((W * v).sum() + vol + area)


def surface_loss_grad(vertices, triangles, W):
    """dL/dp of surface_loss: W + sum over triangles of (p_{k+1} x p_{k+2})/6
    + n_hat x (p_{k+2} - p_{k+1})/2 at each corner k."""
    v, t = np.asarray(vertices), np.asarray(triangles)
    g = np.array(W, dtype=np.float64, copy=True)
    p0, p1, p2 = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    nh = n / np.linalg.norm(n, axis=1)[:, None]
    for k in range(3):
        a, b = v[t[:, (k + 1) % 3]], v[t[:, (k + 2) % 3]]
        np.add.at(g, t[:, k], np.cross(a, b) / 6.0 + 0.5 * np.cross(nh, b - a))
    return g


# ---------------------------------------------------------------- windows
TYPE_CUBE = 30


def key_shift(keys, shift, max_depth):
    """Keys of a sub-problem moved to the full problem's lattice: shift is the
    difference of the two root origins in finest-lattice units (a multiple of
    2^max_depth).  Cube keys hold coordinates at their own level, point keys
    finest-lattice coordinates."""
    k = np.asarray(keys, dtype=np.uint64).astype(np.int64)
    x, y, z = k & 0x3FFFF, (k >> 18) & 0x3FFFF, (k >> 36) & 0x3FFFF
    typ, lvl = (k >> 54) & 31, (k >> 59) & 31
    sh = np.where(typ == TYPE_CUBE, max_depth - lvl, 0)
    x = x + (shift[0] >> sh)
    y = y + (shift[1] >> sh)
    z = z + (shift[2] >> sh)
    assert (x < (1 << 18)).all() and (y < (1 << 18)).all() and (z < (1 << 18)).all()
    return (x | (y << 18) | (z << 36) | (typ << 54) | (lvl << 59)).astype(np.uint64)


def cube_boxes(keys, origin, min_edge, max_depth):
    k = np.asarray(keys, dtype=np.uint64).astype(np.int64)
    xyz = np.stack([k & 0x3FFFF, (k >> 18) & 0x3FFFF, (k >> 36) & 0x3FFFF], 1).astype(np.float64)
    h = min_edge * 2.0 ** (max_depth - ((k >> 59) & 31)).astype(np.float64)
    lo = origin + xyz * h[:, None]
    return lo, lo + h[:, None]


def window_oracle(cfg, centre, half=6.0, margin=10.0, precision=None):
    """The oracle's mesh of the atoms within `margin` of the window
    [centre - half, centre + half]^3, with the shift of its root origin to
    the whole problem's (finest-lattice units).  precision: the config's
    unless given."""
    import oracle
    md, me = cfg["max_depth"], cfg["min_edge"]
    o_full, _, _ = oracle.root_grid(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], me, md)
    lo_w, hi_w = centre - half, centre + half
    sel = np.all((cfg["xyz"] >= lo_w - margin) & (cfg["xyz"] <= hi_w + margin), axis=1)
    sx, sr = np.ascontiguousarray(cfg["xyz"][sel]), np.ascontiguousarray(cfg["r"][sel])
    ref = oracle.mesh(sx, sr, cfg["D"], cfg["c"], cfg["precision"] if precision is None else precision, me, md)
    assert ref["stats"]["loop_errors"] == 0
    o_sub, _, _ = oracle.root_grid(sx, sr, cfg["D"], cfg["c"], me, md)
    shift = np.round((o_sub - o_full) / me).astype(np.int64)
    assert np.all(shift % (1 << md) == 0) and np.all(shift >= 0)
    return dict(ref=ref, shift=shift, origin=o_full, centre=centre, half=half)


def window_compare(full, cfg, win, inner=5.0, min_cubes=100, min_tris=500):
    """Locality check (section 3.1: every cube decision and field value reads
    only atoms within the cutoff radius): the oracle's mesh of a window's
    atoms plus a margin (window_oracle) must give the same cubes inside the
    window, and inside the inner window [centre - inner, centre + inner]^3
    the same surface-point keys, positions within 1e-5 A and triangles, as
    `full` (dict cube_keys, vkeys, vertices, triangles: the whole problem's
    mesh).  A margin >= root cube edge + largest cutoff radius covers every
    ancestor's and neighbour's atoms.  Returns the number of triangles
    compared."""
    md, me = cfg["max_depth"], cfg["min_edge"]
    ref, shift, o_full = win["ref"], win["shift"], win["origin"]
    centre, half = win["centre"], win["half"]
    lo_w, hi_w = centre - half, centre + half
    # cubes inside the window
    glo, ghi = cube_boxes(full["cube_keys"], o_full, me, md)
    ginside = np.all((glo >= lo_w) & (ghi <= hi_w), axis=1)
    rkeys = key_shift(ref["cube_keys"], shift, md)
    rlo, rhi = cube_boxes(rkeys, o_full, me, md)
    rinside = np.all((rlo >= lo_w) & (rhi <= hi_w), axis=1)
    assert ginside.sum() >= min_cubes
    assert np.array_equal(np.sort(full["cube_keys"][ginside]), np.sort(rkeys[rinside])), "cubes differ"
    # surface points inside the inner window
    gv, gkeys = full["vertices"], np.asarray(full["vkeys"], dtype=np.uint64)
    gin = np.all((gv > centre - inner) & (gv < centre + inner), axis=1)
    rvk = key_shift(ref["vkeys"], shift, md)
    rin = np.all((ref["vertices"] > centre - inner) & (ref["vertices"] < centre + inner), axis=1)
    gk, rk = gkeys[gin], rvk[rin]
    only = np.setxor1d(gk, rk)
    if len(only):  # allowed only on the inner window's boundary
        pos = np.concatenate([gv[np.isin(gkeys, only)], ref["vertices"][np.isin(rvk, only)]])
        d = np.minimum(np.abs(pos - (centre - inner)), np.abs(pos - (centre + inner))).min(1)
        assert d.max() < 1e-5, "surface points differ inside the window"
    common = np.intersect1d(gk, rk)
    go = np.argsort(gkeys, kind="stable")
    gi = go[np.searchsorted(gkeys[go], common)]
    ro = np.argsort(rvk, kind="stable")
    ri = ro[np.searchsorted(rvk[ro], common)]
    assert np.array_equal(gkeys[gi], common) and np.array_equal(rvk[ri], common)
    assert np.abs(gv[gi] - ref["vertices"][ri]).max() < 1e-5
    # triangles whose three points lie in the common inner set (the whole
    # mesh's triangles are cut to the inner window first)
    gt = np.asarray(full["triangles"])
    gt = gt[gin[gt].all(axis=1)]
    gct = canonical_triangles(gkeys, gt)
    rct = canonical_triangles(rvk, ref["triangles"])
    gct = gct[np.all(np.isin(gct, common), axis=1)]
    rct = rct[np.all(np.isin(rct, common), axis=1)]
    assert len(gct) >= min_tris
    assert np.array_equal(gct, rct), "triangles differ inside the window"
    return len(gct)
