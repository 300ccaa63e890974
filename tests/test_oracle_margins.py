"""The decision-margin policy on the oracle side: decisions whose margin is
below 1e-10 relative are counted per kind (bound test, precision test, rank
rule, vertex sign), and the resolve mode takes them again in quad precision.

Pins of the quad path against arithmetic that does not share its code:
mpmath at 40 digits for the 1-D coefficients (the projection integral and
the endpoint conditions written out) and for the field sum; the FP64
bounds for the quad bounds (same definition, another precision).  Ties are
built on purpose: c set to a cube's own lower bound L, and to a lattice
vertex's own field value, which the counts must catch."""
import numpy as np
import pytest

import oracle
import synth
from margin_cases import ONE_ATOM, tie_on_bound, tie_on_vertex

mpmath = pytest.importorskip("mpmath")
pytestmark = pytest.mark.skipif(not oracle.have_quad(), reason="no binary128 type in this compiler")
mpmath.mp.dps = 40


def _mp_axis_coeffs(xi, a, b, D):
    """Legendre projection of exp(-D (x - xi)^2) on [a, b] (eqs poly2_1 ..
    poly3), then L_2, L_3 corrections that make the cubic equal f at both
    ends (L_j(1) = 1, L_j(-1) = (-1)^j)."""
    xi, a, b, D = (mpmath.mpf(v) for v in (xi, a, b, D))
    m, hh = (a + b) / 2, (b - a) / 2
    f = lambda x: mpmath.exp(-D * (x - xi) ** 2)
    leg = [lambda t: 1, lambda t: t, lambda t: (3 * t * t - 1) / 2, lambda t: (5 * t ** 3 - 3 * t) / 2]
    al = [(2 * j + 1) / mpmath.mpf(2) * mpmath.quad(lambda t: f(m + hh * t) * leg[j](t), [-1, 1]) for j in range(4)]
    top = f(b) - (al[0] + al[1] + al[2] + al[3])
    bot = f(a) - (al[0] - al[1] + al[2] - al[3])
    return [al[0], al[1], al[2] + (top + bot) / 2, al[3] + (top - bot) / 2]


@pytest.mark.parametrize("xi,a,b,D", [(0.3, -0.5, 1.5, 0.5), (2.7, 0.0, 0.25, 0.9), (-1.1, -2.0, 0.0, 0.5),
                                      (0.05, 0.0, 2.0, 0.9)])
def test_quad_axis_coeffs_match_mpmath(xi, a, b, D):
    hi, lo = oracle.axis_coeffs_quad(xi, a, b, D)
    ref = _mp_axis_coeffs(xi, a, b, D)
    scale = max(abs(float(v)) for v in ref)
    for j in range(4):
        err = abs(mpmath.mpf(hi[j]) + mpmath.mpf(lo[j]) - ref[j])
        assert err < 1e-28 * scale, (j, float(err))
    # and the FP64 oracle agrees with both to FP64 rounding
    d = oracle.axis_coeffs(xi, a, b, D)
    assert np.abs(d - hi).max() < 1e-14 * scale


def test_quad_field_matches_mpmath():
    xyz, r = synth.globular(40, seed=3)
    D, c = 0.5, 1.0
    rng = np.random.default_rng(1)
    pts = xyz[rng.integers(0, 40, 12)] + rng.normal(0, 1.5, (12, 3))
    hi, lo = oracle.field_quad(xyz, r, D, c, pts)
    R2 = r * r + (-np.log(1e-8 * c)) / D
    for k, p in enumerate(pts):
        s = mpmath.mpf(0)
        for i in range(len(r)):
            dx, dy, dz = p[0] - xyz[i, 0], p[1] - xyz[i, 1], p[2] - xyz[i, 2]
            if dx * dx + dy * dy + dz * dz > R2[i]:   # the FP64 cutoff test decides membership
                continue
            d2 = sum((mpmath.mpf(p[a]) - mpmath.mpf(xyz[i, a])) ** 2 for a in range(3))
            s += mpmath.exp(-mpmath.mpf(D) * (d2 - mpmath.mpf(r[i]) ** 2))
        assert abs(mpmath.mpf(hi[k]) + mpmath.mpf(lo[k]) - s) < 1e-30 * (1 + s)


def test_quad_bounds_agree_with_fp64_bounds():
    xyz, r = synth.globular(200, seed=4)
    rng = np.random.default_rng(2)
    for _ in range(20):
        lo = np.floor(xyz[rng.integers(0, 200)] / 2.0) * 2.0 + rng.integers(-1, 2, 3) * 2.0
        A, _ = oracle.cube_tensor(xyz, r, 0.5, 1.0, lo, 2.0)
        b64 = oracle.bounds(A)
        bq = oracle.bounds_quad(A.reshape(-1))
        tot = np.abs(A).sum()
        assert abs(bq[0] - b64[0]) < 1e-12 * tot and abs(bq[1] - b64[1]) < 1e-12 * tot
        assert bq[3] == b64[4]


def test_ordinary_inputs_have_no_in_band_decisions():
    xyz, r = synth.globular(300, seed=1)
    m = oracle.mesh(xyz, r, 0.5, 1.0, 1e-3, 0.25, 3)
    assert m["stats"]["near"] == [0, 0, 0, 0]
    q = oracle.mesh(xyz, r, 0.5, 1.0, 1e-3, 0.25, 3, resolve=True)
    assert q["stats"]["resolved_cubes"] == 0 and q["stats"]["resolved_vertices"] == 0
    assert np.array_equal(m["cube_keys"], q["cube_keys"]) and np.array_equal(m["triangles"], q["triangles"])


def test_tie_on_a_bound_is_counted_and_resolved():
    xyz, r = ONE_ATOM
    c = tie_on_bound()
    m = oracle.mesh(xyz, r, 0.5, c, 1e-3, 0.25, 3)
    assert m["stats"]["near"][0] >= 1
    q = oracle.mesh(xyz, r, 0.5, c, 1e-3, 0.25, 3, resolve=True)
    assert q["stats"]["resolved_cubes"] >= 1


def test_tie_on_a_vertex_is_counted_and_resolved():
    xyz, r = ONE_ATOM
    c = tie_on_vertex()
    m = oracle.mesh(xyz, r, 0.5, c, 1e-3, 0.25, 3)
    assert m["stats"]["near"][3] >= 1
    q = oracle.mesh(xyz, r, 0.5, c, 1e-3, 0.25, 3, resolve=True)
    assert q["stats"]["resolved_vertices"] >= 1
    # the quad value of that vertex lies within FP64 rounding of c
    hi, lo = oracle.field_quad(xyz, r, 0.5, c, np.array([[1.0, 1.0, 1.0]]))
    assert abs(hi[0] - c) <= 4e-16 * c
