"""The FP32 filters of the triangulation, checked on the CPU.  The CUDA file
that holds them is compiled without FMA contraction, so numpy's float32
operations (one rounding each) reproduce their arithmetic.

- Orientation (ear clipping, section 2.3): when the FP32 value of
  (b-a)_i (c-a)_j - (b-a)_j (c-a)_i clears its bound, its sign is the FP64
  predicate's.
- Fold-root screen: the FP32 screen of a fold quadratic answers "no root"
  only where the FP64 solver finds none.
- Newell normal of a piece (its projection axis): every FP32 component lies
  within n (1e-6 + 1.5e-7 n) of the FP64 one, so the axis and sign chosen
  when the largest leads by twice that are the FP64 choice.
- Edge-point and fold-root marks of the mixed vertex field: the first-order
  criteria that leave a surface point to FP32 keep it within the 1e-5 A bar;
  the face-saddle criterion keeps the saddle decision.
- The estimate's FP32 first pass (additions only, so no contraction can
  apply): its corner values of P~ lie within 64 dA + 4e-6 sum|A| of the
  FP64 ones.
- The double-word vertex term stays within its stated bound.
- The warp box filter of the field kernels keeps every atom one of the
  warp's vertices accepts, and the double-word field's FP32 screen never
  drops an FP64 member."""
import numpy as np
import pytest

f32 = np.float32


def orient64(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def orient32_filtered(a, b, c):
    qa = [f32(a[0]), f32(b[0]), f32(c[0])]
    qb = [f32(a[1]), f32(b[1]), f32(c[1])]
    d1, d2 = f32(qa[1] - qa[0]), f32(qb[2] - qb[0])
    d3, d4 = f32(qb[1] - qb[0]), f32(qa[2] - qa[0])
    p1, p2 = f32(d1 * d2), f32(d3 * d4)
    vv = f32(p1 - p2)
    err = f32(f32(4e-7) * f32(f32(f32(abs(d1) + abs(d2)) + abs(d3)) + abs(d4))
              + f32(f32(3e-7) * f32(abs(p1) + abs(p2)))) + f32(1e-13)
    return 1 if vv > err else (-1 if vv < -err else 0)


@pytest.mark.parametrize("seed", range(4))
def test_orientation_filter_agrees_with_fp64(seed):
    rng = np.random.default_rng(seed)
    decided = 0
    for k in range(20000):
        a, b = rng.random(2), rng.random(2)
        if k % 2:
            # near-collinear: c on the line ab, moved off it by 1e-9 .. 1e-4
            t = rng.uniform(-0.5, 1.5)
            n = np.array([-(b - a)[1], (b - a)[0]])
            c = a + t * (b - a) + n * rng.choice([-1, 1]) * 10 ** rng.uniform(-9, -4)
            c = np.clip(c, 0, 1)
        else:
            c = rng.random(2)
        s32 = orient32_filtered(a, b, c)
        if s32:
            decided += 1
            o = orient64(a, b, c)
            assert (o > 0) == (s32 > 0) and o != 0
    assert decided > 10000


@pytest.mark.parametrize("seed", range(3))
def test_newell_normal_fp32_bound(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(600):
        n = int(rng.integers(3, 97))
        if rng.random() < 0.5:
            P = rng.random((n, 3))
        else:
            # nearly planar polygons with two components of similar size
            u, v = rng.standard_normal(3), rng.standard_normal(3)
            P = 0.5 + 0.3 * (np.outer(np.cos(np.linspace(0, 6.2, n)), u) +
                             np.outer(np.sin(np.linspace(0, 6.2, n)), v)) + 1e-6 * rng.standard_normal((n, 3))
            P = np.clip(P, 0, 1)
        Q = P.astype(f32)
        M = np.zeros(3, f32)
        N = np.zeros(3)
        for i in range(n):
            p, q = Q[i], Q[(i + 1) % n]
            M[0] = f32(M[0] + f32(f32(p[1] - q[1]) * f32(p[2] + q[2])))
            M[1] = f32(M[1] + f32(f32(p[2] - q[2]) * f32(p[0] + q[0])))
            M[2] = f32(M[2] + f32(f32(p[0] - q[0]) * f32(p[1] + q[1])))
            pd, qd = P[i], P[(i + 1) % n]
            N += [(pd[1] - qd[1]) * (pd[2] + qd[2]), (pd[2] - qd[2]) * (pd[0] + qd[0]),
                  (pd[0] - qd[0]) * (pd[1] + qd[1])]
        errM = n * (1e-6 + 1.5e-7 * n)
        assert np.all(np.abs(M.astype(np.float64) - N) <= errM)


def _faces(g, a):
    ua, va = (1, 2) if a == 0 else ((0, 2) if a == 1 else (0, 1))
    lo, up = [], []
    for k in range(4):
        b = [0, 0, 0]
        b[ua], b[va] = k & 1, k >> 1
        b[a] = 0
        lo.append(g[b[0] + 2 * b[1] + 4 * b[2]])
        b[a] = 1
        up.append(g[b[0] + 2 * b[1] + 4 * b[2]])
    return lo, up


def _coeffs(lo, up, c, T):
    lo = [T(x) for x in lo]
    up = [T(x) for x in up]
    p0 = T(lo[0] - c) if c is not None else lo[0]
    p1, p2 = T(lo[1] - lo[0]), T(lo[2] - lo[0])
    p3 = T(T(T(lo[3] - lo[1]) - lo[2]) + lo[0])
    d = [T(up[k] - lo[k]) for k in range(4)]
    q0, q1, q2 = d[0], T(d[1] - d[0]), T(d[2] - d[0])
    q3 = T(T(T(d[3] - d[1]) - d[2]) + d[0])
    A2 = T(T(p1 * q3) - T(p3 * q1))
    A1 = T(T(T(T(p0 * q3) + T(p1 * q2)) - T(p2 * q1)) - T(p3 * q0))
    A0 = T(T(p0 * q2) - T(p2 * q0))
    return (p0, p1, p2, p3), (q0, q1, q2, q3), (A2, A1, A0)


def screen32(g, c, a):
    gc = [f32(x - c) for x in g]
    lo, up = _faces(gc, a)
    (p0, p1, p2, p3), (q0, q1, q2, q3), (A2, A1, A0) = _coeffs(lo, up, None, f32)
    terms = [p1 * q3, p3 * q1, p0 * q3, p1 * q2, p2 * q1, p3 * q0, p0 * q2, p2 * q0]
    mag = f32(0)
    for t in terms:
        mag = f32(mag + abs(f32(t)))
    if not mag > 1e-30:
        return True
    if abs(A2) <= f32(1e-3) * mag:
        return True
    disc = f32(f32(A1 * A1) - f32(f32(f32(4) * A2) * A0))
    scale = f32(f32(A1 * A1) + f32(4) * abs(f32(A2 * A0)))
    if disc < f32(-1e-3) * scale:
        return False
    if disc <= f32(1e-3) * scale:
        return True
    sq = np.sqrt(disc, dtype=f32)
    w = f32(f32(-0.5) * f32(A1 + sq)) if A1 >= 0 else f32(f32(-0.5) * f32(A1 - sq))
    if w == 0:
        return True
    u1, u2 = f32(w / A2), f32(A0 / w)
    return (-0.01 < u1 < 1.01) or (-0.01 < u2 < 1.01)


def solve64_has_root(g, c, a):
    """The FP64 fold solver's root test (roots u, v in [0,1] satisfying both
    fold equations), restated in numpy."""
    lo, up = _faces(g, a)
    (p0, p1, p2, p3), (q0, q1, q2, q3), (A2, A1, A0) = _coeffs(lo, up, c, np.float64)
    if q0 == q1 == q2 == q3 == 0:
        return False
    us = []
    if A2 == 0:
        if A1 != 0:
            us.append(-A0 / A1)
    else:
        disc = A1 * A1 - 4 * A2 * A0
        if disc >= 0:
            sq = np.sqrt(disc)
            w = -0.5 * (A1 + sq) if A1 >= 0 else -0.5 * (A1 - sq)
            us += [w / A2, A0 / w] if w != 0 else [0.0]
    sp, sq_ = abs(p0) + abs(p1) + abs(p2) + abs(p3), abs(q0) + abs(q1) + abs(q2) + abs(q3)
    for u in us:
        if not (0 < u < 1):
            continue
        for num, den in ((q0 + q1 * u, q2 + q3 * u), (p0 + p1 * u, p2 + p3 * u)):
            if den == 0:
                continue
            v = -num / den
            if 0 < v < 1 and abs(p0 + p1 * u + p2 * v + p3 * u * v) <= 1e-9 * sp and \
                    abs(q0 + q1 * u + q2 * v + q3 * u * v) <= 1e-9 * sq_:
                return True
    return False


@pytest.mark.parametrize("seed", range(3))
def test_fold_screen_never_misses_a_root(seed):
    """The FP32 screen answers 'no root' only where the FP64 solver finds
    none: random corner values, corner values differing by 1e-6 of their
    size, and cubes built around a fold root of chosen position."""
    rng = np.random.default_rng(200 + seed)
    c, found = 1.0, 0
    for k in range(6000):
        kind = k % 3
        if kind == 0:
            g = c + rng.uniform(-1, 1, 8)
        elif kind == 1:
            g = c + 1e-6 * rng.uniform(-1, 1, 8) * 10 ** rng.uniform(-2, 2)
        else:
            # g = A(u,v) + s B(u,v) with B = (u - u0)(...) style zero near (u0, v0)
            u0, v0, s0 = rng.random(3)
            g = np.empty(8)
            cu, cv, cs = rng.standard_normal(3)
            for v in range(8):
                x, y, z = v & 1, (v >> 1) & 1, v >> 2
                g[v] = c + cu * (x - u0) + cv * (y - v0) * (z - s0) * rng.uniform(0.5, 2) + cs * (x - u0) * (y - v0)
        for a in range(3):
            if solve64_has_root(g, c, a):
                found += 1
                assert screen32(g, c, a), (g.tolist(), a)
    assert found > 100


def _corner_range(a, T):
    """Corner values of P~ as the estimate's first pass sums them
    (x pairs, then y pairs, then z pairs), in type T."""
    a = [T(x) for x in a]
    lo, hi = None, None
    for sx in (0, 1):
        bx = []
        for kl in range(16):
            e, o = T(a[kl] + a[32 + kl]), T(a[16 + kl] + a[48 + kl])
            bx.append(T(e + o) if sx else T(e - o))
        for sy in (0, 1):
            cz = []
            for l in range(4):
                e, o = T(bx[l] + bx[8 + l]), T(bx[4 + l] + bx[12 + l])
                cz.append(T(e + o) if sy else T(e - o))
            e, o = T(cz[0] + cz[2]), T(cz[1] + cz[3])
            for v in (T(e - o), T(e + o)):
                lo = v if lo is None else min(lo, v)
                hi = v if hi is None else max(hi, v)
    return lo, hi


@pytest.mark.parametrize("seed", range(3))
def test_corner_sums_within_the_first_pass_margin(seed):
    """The FP32 first pass keeps a cube when its FP32 corner values straddle
    c by 64 dA + 4e-6 sum|A|: with every FP32 entry within dA of the FP64
    one, the FP32 corner range lies within that margin of the FP64 range."""
    rng = np.random.default_rng(300 + seed)
    for _ in range(3000):
        A = rng.standard_normal(64) * np.exp(-rng.uniform(0, 6, 64))
        tot = np.abs(A).sum()
        dA = 1.6e-6 * tot * rng.uniform(0.01, 1)
        A32 = (A + rng.uniform(-1, 1, 64) * dA).astype(f32)   # entries off by <= dA (+ their rounding)
        dA_eff = dA + 6e-8 * np.abs(A).max()
        lo32, hi32 = _corner_range(A32, f32)
        lo64, hi64 = _corner_range(A, np.float64)
        m = 64 * dA_eff + 4e-6 * tot
        assert abs(float(lo32) - lo64) <= m and abs(float(hi32) - hi64) <= m


@pytest.mark.parametrize("D", [0.5, 0.9])
def test_vertex_term_bound_covers_argument_rounding(D):
    """Mixed vertex field: each FP32 term t = 2^(-D log2e (d^2 - r^2)) is
    taken to err by at most t (3e-7 + 3e-7 D (d^2 + r^2)).  The exponent's
    FP32 rounding is reproduced here (two-float offsets from the origin, d^2
    with or without FMA contraction, d^2 - r^2, the scaled exponent); the
    hardware ex2 adds its documented 2^-22 and the result's rounding.  Rare
    far terms (D d^2 ~ 10, where the rounding of D log2e itself counts)
    reach about 0.84 of the bound; the test holds every case within it."""
    rng = np.random.default_rng(int(D * 10))
    origin = np.array([-7.0, -3.0, -11.0])
    nDl2e = f32(-D * 1.4426950408889634)
    worst = 0.0
    for _ in range(20000):
        x = rng.uniform(0, 300, 3)
        r = rng.choice([1.2, 1.7, 1.55, 1.52, 1.8])
        R = np.sqrt(r * r - np.log(1e-8) / D)
        dvec = rng.normal(size=3)
        p = x + dvec / np.linalg.norm(dvec) * rng.uniform(0, R)
        ph, xh = (p - origin).astype(f32), (x - origin).astype(f32)
        pl = ((p - origin) - ph.astype(np.float64)).astype(f32)
        xl = ((x - origin) - xh.astype(np.float64)).astype(f32)
        d = [f32(f32(ph[a] - xh[a]) + f32(pl[a] - xl[a])) for a in range(3)]
        r2 = f32(r * r)
        d2_plain = f32(f32(f32(d[0] * d[0]) + f32(d[1] * d[1])) + f32(d[2] * d[2]))
        d2_fma = f32(np.float64(d[2]) * d[2] + np.float64(f32(np.float64(d[1]) * d[1] + np.float64(f32(d[0] * d[0])))))
        exact = -D * 1.4426950408889634 * (np.sum((p - x) ** 2) - r * r)
        bound = 3e-7 + 3e-7 * D * (float(d2_plain) + r * r)
        for d2 in (d2_plain, d2_fma):
            arg = f32(nDl2e * f32(d2 - r2))
            rel = np.log(2) * abs(float(arg) - exact) + 2.0 ** -22 + 2.0 ** -24
            worst = max(worst, rel / bound)
            assert rel <= bound
    assert worst > 0.05   # the cases reach a sizeable share of the bound


def test_edge_point_mark_criterion_is_sound():
    """Mixed vertex marks: an edge point t = (c - g0)/(g1 - g0) is left to FP32
    when h ((1 - t) e0 + t e1) / |g1 - g0|, inflated by 1%, is at most
    8e-6 A (e0, e1 the corners' error bounds).  Then the point moves by less
    than the 1e-5 A bar for any corner errors within the bounds: the exact
    worst case over the four sign combinations of the errors is checked."""
    rng = np.random.default_rng(17)
    h, c, tol = 0.25, 1.0, 8e-6
    checked = 0
    for _ in range(200000):
        g0 = c - 10 ** rng.uniform(-7, 0)
        g1 = c + 10 ** rng.uniform(-7, 0)
        if rng.random() < 0.5:
            g0, g1 = g1, g0
        e0, e1 = (10 ** rng.uniform(-9, -5, 2))
        t = (c - g0) / (g1 - g0)
        first = 1.01 * h * ((1 - t) * e0 + t * e1) / abs(g1 - g0)
        if first > tol or max(e0, e1) >= abs(g1 - g0) / 2:
            continue
        checked += 1
        moves = [abs((c - (g0 + s0 * e0)) / ((g1 + s1 * e1) - (g0 + s0 * e0)) - t) * h
                 for s0 in (-1, 1) for s1 in (-1, 1)]
        assert max(moves) < 1e-5
    assert checked > 20000


def _fold_roots64(g, c, a):
    """(u, v) fold roots of axis a in the open face square, FP64."""
    lo, up = _faces(g, a)
    (p0, p1, p2, p3), (q0, q1, q2, q3), (A2, A1, A0) = _coeffs(lo, up, c, np.float64)
    us = []
    if A2 == 0:
        if A1 != 0:
            us.append(-A0 / A1)
    else:
        disc = A1 * A1 - 4 * A2 * A0
        if disc >= 0:
            sq = np.sqrt(disc)
            w = -0.5 * (A1 + sq) if A1 >= 0 else -0.5 * (A1 - sq)
            us += [w / A2, A0 / w] if w != 0 else [0.0]
    out = []
    for u in us:
        if not 0 < u < 1:
            continue
        denB, denA = q2 + q3 * u, p2 + p3 * u
        den, num = (denB, q0 + q1 * u) if abs(denB) >= abs(denA) else (denA, p0 + p1 * u)
        if den != 0 and 0 < -num / den < 1:
            out.append((u, -num / den))
    return out, (p0, p1, p2, p3), (q0, q1, q2, q3), (A2, A1, A0)


def test_fold_root_mark_criterion_is_sound():
    """Mixed vertex marks for fold roots: when the first-order bound
    h (|du| + |dv|) from J^-1 of the corner errors (inflated 1%) is within
    8e-6 A, the root is at least 4 error radii inside the face square and not
    a near-double root, corner errors within their bounds move the root by
    less than 1e-5 A (checked over random sign patterns, root re-solved in
    FP64)."""
    rng = np.random.default_rng(23)
    h, c, tol, a = 0.25, 1.0, 8e-6, 0
    checked = 0
    for _ in range(4000):
        g = c + rng.uniform(-1, 1, 8) * 10 ** rng.uniform(-2, 0)
        roots, (p0, p1, p2, p3), (q0, q1, q2, q3), (A2, A1, A0) = _fold_roots64(g, c, a)
        if not roots:
            continue
        scale = A1 * A1 + 4 * abs(A2 * A0)
        if A2 != 0 and abs(A1 * A1 - 4 * A2 * A0) <= 1e-4 * scale:
            continue   # near-double root: every corner goes to FP64
        e = 10 ** rng.uniform(-10, -6, 8)
        lo_i = [0, 2, 4, 6]   # axis 0: corner index of (u, v) = (y, z) on the x = 0 face
        up_i = [1, 3, 5, 7]
        for u, v in roots:
            w4 = [(1 - u) * (1 - v), u * (1 - v), (1 - u) * v, u * v]
            J11, J12, J21, J22 = p1 + p3 * v, p2 + p3 * u, q1 + q3 * v, q2 + q3 * u
            det = abs(J11 * J22 - J12 * J21)
            if det == 0:
                continue
            bu = bv = 0.0
            for q in range(4):
                slo, sup = 1.01 * w4[q] * e[lo_i[q]], 1.01 * w4[q] * e[up_i[q]]
                bu += ((abs(J22) + abs(J12)) * slo + abs(J12) * sup) / det
                bv += ((abs(J21) + abs(J11)) * slo + abs(J11) * sup) / det
            if h * (bu + bv) > tol or min(u, 1 - u) <= 4 * bu + 1e-5 or min(v, 1 - v) <= 4 * bv + 1e-5:
                continue
            checked += 1
            for _ in range(24):
                gp = g + rng.choice([-1.0, 1.0], 8) * e
                rp, *_ = _fold_roots64(gp, c, a)
                assert rp, "the root vanished"
                move = min(np.hypot(up_ - u, vp - v) for up_, vp in rp) * h
                assert move < 1e-5
    assert checked > 300


def test_face_saddle_mark_criterion_is_sound():
    """Mixed vertex marks for diagonal faces: when |h_s - c| exceeds
    4 amp sum(e), amp = 2 sum|h| / |h0 - h1 - h2 + h3|, the saddle decision
    h_s < c is the same under corner errors within e (corner signs
    themselves are settled by the first recheck round).  Checked at all 16
    corner-error sign patterns and at 4 random interior error vectors per
    face."""
    rng = np.random.default_rng(29)
    c, checked = 1.0, 0
    patterns = np.array([[1.0 if (k >> b) & 1 else -1.0 for b in range(4)] for k in range(16)])
    for _ in range(50000):
        s = rng.choice([-1.0, 1.0])
        h = c + s * np.array([1, -1, -1, 1]) * 10 ** rng.uniform(-6, 0, 4)   # diagonal pattern
        e = 10 ** rng.uniform(-10, -5, 4)
        if np.any(np.abs(h - c) <= 2 * e):
            continue
        den = h[0] - h[1] - h[2] + h[3]
        hs = (h[0] * h[3] - h[1] * h[2]) / den
        amp = 2 * np.abs(h).sum() / abs(den)
        if abs(hs - c) <= 4 * amp * e.sum():
            continue
        checked += 1
        hp = h + np.vstack([patterns, rng.uniform(-1.0, 1.0, (4, 4))]) * e
        denp = hp[:, 0] - hp[:, 1] - hp[:, 2] + hp[:, 3]
        hsp = (hp[:, 0] * hp[:, 3] - hp[:, 1] * hp[:, 2]) / denp
        assert np.all((hsp < c) == (hs < c))
    assert checked > 10000


def _dw_term(ph, pl, ah, al, fr2, lr2, Kh, Kl, L2h, L2l, tab):
    """One double-word term 2^(K (r^2 - d^2)) in the steps the mixed mode's
    vertex re-evaluation takes (numpy float32 rounds each operation as the
    GPU does; an FMA is the exact product plus the addend, rounded once)."""
    def add(a, b): return f32(f32(a) + f32(b))
    def sub(a, b): return f32(f32(a) - f32(b))
    def mul(a, b): return f32(f32(a) * f32(b))
    def fma(a, b, c): return f32(np.float64(f32(a)) * np.float64(f32(b)) + np.float64(f32(c)))
    def two_sum(a, b):
        s = add(a, b)
        bb = sub(s, a)
        return s, add(sub(a, sub(s, bb)), sub(b, bb))
    def two_prod(a, b):
        p = mul(a, b)
        return p, fma(a, b, -p)
    sd = [two_sum(ph[a], -ah[a]) for a in range(3)]
    lo = [add(sd[a][1], sub(pl[a], al[a])) for a in range(3)]
    sq = [two_prod(sd[a][0], sd[a][0]) for a in range(3)]
    q = [fma(add(add(sd[a][0], sd[a][0]), lo[a]), lo[a], sq[a][1]) for a in range(3)]
    u1 = two_sum(sq[0][0], sq[1][0])
    u2 = two_sum(u1[0], sq[2][0])
    d2l = add(add(u1[1], u2[1]), add(add(q[0], q[1]), q[2]))
    z = two_sum(fr2, -u2[0])
    zl = add(z[1], sub(lr2, d2l))
    yh = mul(Kh, z[0])
    yl = fma(Kh, zl, fma(Kl, z[0], fma(Kh, z[0], -yh)))
    n = f32(np.rint(yh))
    f = sub(yh, n)
    j = f32(np.rint(mul(f, 64)))
    g = two_sum(sub(f, mul(j, f32(1 / 64))), yl)
    sh = mul(L2h, g[0])
    sl = fma(L2h, g[1], fma(L2l, g[0], fma(L2h, g[0], -sh)))
    qq = fma(sh, fma(sh, fma(sh, f32(1 / 120), f32(1 / 24)), f32(1 / 6)), f32(0.5))
    Q = fma(sh, sl, mul(mul(sh, sh), qq))
    eh = add(f32(1), sh)
    el = add(sub(sh, sub(eh, f32(1))), add(sl, Q))
    th, tl = tab[int(j) + 32]
    p = mul(th, eh)
    pl2 = fma(th, el, fma(tl, eh, fma(th, eh, -p)))
    sc = f32(2.0 ** int(n))
    return np.longdouble(mul(p, sc)) + np.longdouble(mul(pl2, sc))


@pytest.mark.parametrize("D", [0.5, 0.9])
def test_double_word_term_within_its_bound(D):
    """The double-word vertex term stays within its stated bound
    D u^2 (90 R L + 120 R^2) + 2e-11 (u = 2^-24, L the vertex's largest
    offset from the origin, R the cutoff radius) of the exact term, taken in
    extended precision from the FP64 coordinates.  The random cases reach a
    few percent of it."""
    if np.finfo(np.longdouble).eps > 1e-18:
        pytest.skip("needs an extended-precision long double")
    ld = np.longdouble
    tab = []
    for j in range(-32, 33):
        v = ld(2) ** (ld(j) / 64)
        h = f32(v)
        tab.append((h, f32(v - ld(h))))
    K = D * 1.4426950408889634074
    Kh = f32(K)
    Kl = f32(K - np.float64(Kh))
    L2h = f32(0.6931471805599453094)
    L2l = f32(0.6931471805599453094 - np.float64(L2h))
    rng = np.random.default_rng(int(D * 100))
    origin = np.array([-3.0, -5.0, -7.0])
    worst = 0.0
    for _ in range(3000):
        x = rng.uniform(0, 600, 3)
        r = rng.choice([1.2, 1.7, 1.55, 1.52, 1.8])
        R = np.sqrt(r * r - np.log(1e-8) / D)
        dv = rng.normal(size=3)
        p = x + dv / np.linalg.norm(dv) * rng.uniform(0, R)
        rp, ra = p - origin, x - origin
        ph, ah = rp.astype(f32), ra.astype(f32)
        pl = (rp - ph.astype(np.float64)).astype(f32)
        al = (ra - ah.astype(np.float64)).astype(f32)
        rr = r * r
        fr2 = f32(rr)
        lr2 = f32(rr - np.float64(fr2))
        t = _dw_term(ph, pl, ah, al, fr2, lr2, Kh, Kl, L2h, L2l, tab)
        d2 = sum((ld(p[a]) - ld(x[a])) ** 2 for a in range(3))
        exact = np.exp(-ld(D) * (d2 - ld(r) * ld(r)))
        L = float(np.abs(ph).max())
        bound = D * 2.0 ** -48 * (90 * R * L + 120 * R * R) + 2e-11
        rel = abs(float((t - exact) / exact))
        worst = max(worst, rel / bound)
        assert rel <= bound
    assert worst > 0.01


def _split2(x):
    """offsets from the origin as hi + lo floats, as the kernels store them"""
    h = x.astype(f32)
    return h, (x - h.astype(np.float64)).astype(f32)


@pytest.mark.parametrize("scale", [100.0, 60000.0])
def test_warp_box_filter_keeps_every_accepted_atom(scale):
    """The field kernels stage an atom for a warp only if its cutoff sphere
    reaches the box of the warp's vertices (hi parts only; gaps lowered by
    1e-3 A + 4e-7 |x|, sphere grown by 1% + 0.01 A^2).  Every atom that one
    of the warp's vertices accepts, by the FP32 test of the FP32 field or by
    the FP64 membership of the FP64 and double-word fields, must pass."""
    rng = np.random.default_rng(int(scale))
    kept = rejected = 0
    for _ in range(300):
        centre = rng.uniform(0.2 * scale, scale, 3)
        verts = centre + rng.uniform(0, 2.5, (32, 3))
        R2 = rng.uniform(20.0, 60.0)
        dirs = rng.normal(size=(64, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        atoms = centre + 1.25 + dirs * rng.uniform(0.0, np.sqrt(R2) + 3.0, 64)[:, None]
        ph, pl = _split2(verts)
        ah, al = _split2(atoms)
        lo, hi = ph.min(axis=0), ph.max(axis=0)
        fR2 = f32(R2)
        for k in range(len(atoms)):
            g2 = f32(0)
            for a in range(3):
                x = ah[k, a]
                gap = max(f32(lo[a] - x), f32(x - hi[a]))
                slack = f32(np.float64(f32(4e-7)) * np.float64(abs(x)) + np.float64(f32(1e-3)))
                g = max(f32(0), f32(gap - slack))
                g2 = f32(g2 + f32(g * g))
            passes = g2 <= f32(np.float64(fR2) * np.float64(f32(1.01)) + np.float64(f32(0.01)))
            d = (ph - ah[k]).astype(f32) + (pl - al[k]).astype(f32)
            d2_32 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]).astype(f32)
            d2_64 = ((verts - atoms[k]) ** 2).sum(axis=1)
            accepted = bool(np.any(d2_32 <= fR2) or np.any(d2_64 <= R2))
            if accepted:
                assert passes
            kept += passes
            rejected += not passes
    assert rejected > 0.1 * (kept + rejected)   # the filter does drop atoms out of reach


def test_double_word_screen_never_drops_a_member():
    """The double-word field screens a candidate with the FP32 distance from
    the two-float offsets: beyond R^2 (1 + 1e-5) + 1e-5 it is out, below
    R^2 (1 - 1e-5) - 1e-5 it is in, and between the exact FP64 test decides.
    So no FP64 member is screened out and every atom taken without the FP64
    test is an FP64 member, for offsets up to thousands of A."""
    rng = np.random.default_rng(11)
    for scale in (50.0, 5000.0):
        for _ in range(20000):
            atom = rng.uniform(0.2 * scale, scale, 3)
            R2 = rng.uniform(20.0, 60.0)
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            d = np.sqrt(R2) * (1.0 + rng.choice([-1, 1]) * 10.0 ** rng.uniform(-9, -3))
            p = atom + u * d
            ph, pl = _split2(p)
            ah, al = _split2(atom)
            f = (ph - ah).astype(f32) + (pl - al).astype(f32)
            f2 = f32(f32(f32(f[0] * f[0]) + f32(f[1] * f[1])) + f32(f[2] * f[2]))
            fR2 = f32(R2)
            member = ((p - atom) ** 2).sum() <= R2
            out = f2 > f32(f32(fR2 * f32(1.0 + 1e-5)) + f32(1e-5))
            sure_in = f2 < f32(f32(fR2 * f32(1.0 - 1e-5)) - f32(1e-5))
            assert not (member and out)
            assert not (sure_in and not member)
