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
