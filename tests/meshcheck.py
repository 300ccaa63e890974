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
