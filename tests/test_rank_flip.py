"""The rank-flip allowance of the mixed estimate, checked directly: when a
99% rank rule of the two-level SVD (section 2.2.2, eqs SVD3-SVD7) sits at its
threshold, the bounds L and U under either rank differ by less than 0.36 of
the sum of the outer singular values S.  The mixed form treats a decision as
final when its margin exceeds the FP32 band by 0.4 S.

The bounds here are a numpy restatement of the two-level estimate (exact
1-D cubic ranges, 4-corner interval products, residual sum) with the ranks
given, independent of both the oracle and the CUDA path."""
import numpy as np
import pytest


def cubic_range(c):
    """Exact min and max over [-1,1] of sum_j c_j L_j(t)."""
    p = np.array([c[0] - c[2] / 2, c[1] - 1.5 * c[3], 1.5 * c[2], 2.5 * c[3]])   # 1, t, t^2, t^3
    ts = [-1.0, 1.0]
    r = np.roots([3 * p[3], 2 * p[2], p[1]]) if abs(p[3]) > 0 else (
        np.array([-p[1] / (2 * p[2])]) if abs(p[2]) > 0 else np.array([]))
    ts += [float(x.real) for x in np.atleast_1d(r) if abs(x.imag) < 1e-12 and -1 < x.real < 1]
    v = [p[0] + p[1] * t + p[2] * t * t + p[3] * t ** 3 for t in ts]
    return min(v), max(v)


def bounds(A, outer_rank, inner_ranks):
    A1 = A.reshape(4, 16)
    U, s, Vt = np.linalg.svd(A1)
    M = m = 0.0
    At = np.zeros((4, 4, 4))
    for i in range(outer_rank):
        W, d, Zt = np.linalg.svd(Vt[i].reshape(4, 4))
        Myz = myz = 0.0
        for k in range(inner_ranks[i]):
            ly, hy = cubic_range(W[:, k])
            lz, hz = cubic_range(Zt[k])
            prods = [hy * hz, hy * lz, ly * hz, ly * lz]
            Myz += d[k] * max(prods)
            myz += d[k] * min(prods)
            At += s[i] * d[k] * np.einsum("a,b,c->abc", U[:, i], W[:, k], Zt[k])
        lx, hx = cubic_range(U[:, i])
        prods = [hx * Myz, hx * myz, lx * Myz, lx * myz]
        M += s[i] * max(prods)
        m += s[i] * min(prods)
    R = np.abs(A - At).sum()
    return m - R, M + R, s.sum()


def rank99(s):
    acc, tot = 0.0, s.sum()
    for j, x in enumerate(s):
        acc += x
        if acc >= 0.99 * tot:
            return j + 1
    return len(s)


def orthonormal(rng, n, k):
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return q[:, :k]


def tensor(rng, sig, inner_sig):
    """A with outer singular values sig and, for each outer term, inner
    singular values inner_sig[i] (scaled to a unit Frobenius norm)."""
    U = orthonormal(rng, 4, 4)
    rows = []
    for i in range(4):
        W, Z = orthonormal(rng, 4, 4), orthonormal(rng, 4, 4)
        d = np.asarray(inner_sig[i], float)
        d = d / np.linalg.norm(d)
        rows.append((W * d) @ Z.T)
    # the outer right vectors must be orthonormal: orthogonalise the
    # flattened inner matrices (keeps each one's shape up to a small mix)
    V, _ = np.linalg.qr(np.stack([r.ravel() for r in rows], 1))
    V = V * np.sign(np.sum(V * np.stack([r.ravel() for r in rows], 1), 0))
    return (U * np.asarray(sig, float)) @ V.T


@pytest.mark.parametrize("seed", range(40))
def test_rank_flip_moves_bounds_less_than_allowance(seed):
    rng = np.random.default_rng(seed)
    # outer: the rule at j sits exactly on the 99% threshold
    j = int(rng.integers(1, 4))
    head = rng.uniform(0.2, 1.0, j)
    tail = rng.uniform(0.1, 1.0, 4 - j)
    sig = np.concatenate([np.sort(head)[::-1] * 0.99 / head.sum(), np.sort(tail)[::-1] * 0.01 / tail.sum()])
    sig = np.sort(sig)[::-1]
    inner = [np.sort(rng.uniform(0.01, 1.0, 4))[::-1] for _ in range(4)]
    A = tensor(rng, sig * rng.uniform(0.5, 5.0), inner).reshape(4, 4, 4)
    U, s, Vt = np.linalg.svd(A.reshape(4, 16))
    r = rank99(s)
    inner_r = [rank99(np.linalg.svd(Vt[i].reshape(4, 4), compute_uv=False)) for i in range(4)]
    L0, U0, S = bounds(A, r, inner_r)
    flipped = 0
    for alt in {max(1, r - 1), min(4, r + 1)} - {r}:
        if abs(s[:alt].sum() - s[:r].sum()) > 0.011 * S:
            continue   # that rule is not at its threshold: no flip to bound
        flipped += 1
        L1, U1, _ = bounds(A, alt, inner_r)
        assert abs(L1 - L0) <= 0.36 * S and abs(U1 - U0) <= 0.36 * S, (r, alt)
    assert flipped >= 1   # the constructed rule at j is at its threshold
    # inner: put one kept term's inner rule on its threshold and flip it
    i = int(rng.integers(0, r))
    d = np.linalg.svd(Vt[i].reshape(4, 4), compute_uv=False)
    for alt in {max(1, inner_r[i] - 1), min(4, inner_r[i] + 1)} - {inner_r[i]}:
        moved = abs(d[:alt].sum() - d[:inner_r[i]].sum()) / d.sum()
        if moved > 0.011:
            continue   # that rule is not at its threshold: no flip to bound
        ir = list(inner_r)
        ir[i] = alt
        L1, U1, _ = bounds(A, r, ir)
        assert abs(L1 - L0) <= 0.36 * S and abs(U1 - U0) <= 0.36 * S
