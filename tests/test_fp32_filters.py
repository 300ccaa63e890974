"""The FP32 filters of the triangulation, checked on the CPU.  The CUDA file
that holds them is compiled without FMA contraction, so numpy's float32
operations (one rounding each) reproduce their arithmetic.

- Orientation (ear clipping, section 2.3): when the FP32 value of
  (b-a)_i (c-a)_j - (b-a)_j (c-a)_i clears its bound, its sign is the FP64
  predicate's.
- Newell normal of a piece (its projection axis): every FP32 component lies
  within n (1e-6 + 1.5e-7 n) of the FP64 one, so the axis and sign chosen
  when the largest leads by twice that are the FP64 choice."""
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
