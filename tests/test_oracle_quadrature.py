"""Pins of the oracle's quadrature pieces (Sec. II.C "Integral evaluation").

* Dunavant rules: exact on every monomial up to the rule's degree (the
  defining property of the 1/3/4- and 19/25/37-point rules), and not exact
  one degree above (so a truncated or mis-copied table is caught).
* Self-panel integral: the closed form against (a) the textbook value for the
  centroid of an equilateral triangle and (b) an independent Duffy-transformed
  adaptive integration on random triangles and points.
"""
from math import factorial

import numpy as np
import pytest
from scipy.integrate import quad

DEGREE = {1: 1, 3: 2, 4: 3, 19: 9, 25: 10, 37: 13}


def _monomial_exact(a, b):
    # integral of x^a y^b over the triangle (0,0),(1,0),(0,1)
    return factorial(a) * factorial(b) / factorial(a + b + 2)


@pytest.mark.parametrize("K", sorted(DEGREE))
def test_dunavant_exactness(oracle, K):
    bary, w = oracle.quad_rule(K)
    assert bary.shape == (K, 3)
    assert np.allclose(bary.sum(1), 1.0, atol=1e-15)
    assert abs(w.sum() - 1.0) < 1e-14
    x, y = bary[:, 1], bary[:, 2]
    deg = DEGREE[K]
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            q = 0.5 * np.sum(w * x ** a * y ** b)
            assert abs(q - _monomial_exact(a, b)) <= 5e-14 * _monomial_exact(a, b) + 1e-16, (K, a, b)
    # one degree higher must fail for at least one monomial (the rule's degree is sharp)
    errs = [abs(0.5 * np.sum(w * x ** a * y ** (deg + 1 - a)) - _monomial_exact(a, deg + 1 - a))
            / _monomial_exact(a, deg + 1 - a) for a in range(deg + 2)]
    assert max(errs) > 1e-10


def test_dunavant_rule_symmetry(oracle):
    # symmetric rules: the point set is invariant under permutation of barycentrics
    for K in DEGREE:
        bary, w = oracle.quad_rule(K)
        key = {tuple(np.round(p, 12)) for p in bary}
        for perm in [(1, 0, 2), (2, 1, 0), (0, 2, 1)]:
            assert {tuple(np.round(p[list(perm)], 12)) for p in bary} == key


def test_unknown_rule_rejected(oracle):
    with pytest.raises(ValueError):
        oracle.quad_rule(7)


def test_self_integral_equilateral_closed_form(oracle):
    # centroid of an equilateral triangle of side a: int 1/|c-y| dA = sqrt(3) a ln(2+sqrt(3))
    a = 1.7
    v0 = np.array([0.0, 0.0, 0.0]); v1 = np.array([a, 0.0, 0.0]); v2 = np.array([a / 2, a * np.sqrt(3) / 2, 0.0])
    c = (v0 + v1 + v2) / 3
    exact = np.sqrt(3) * a * np.log(2 + np.sqrt(3)) / (4 * np.pi)
    assert abs(oracle.self_V(v0, v1, v2, c) - exact) < 1e-14 * exact


def _duffy_self(v, x):
    """int_T 1/|x-y| dA by three Duffy-mapped sub-triangles (x, a, b):
    y = x + u[(a-x) + t(b-a)], dA = u |(a-x)x(b-a)| du dt, |x-y| = u |(a-x)+t(b-a)|,
    so the u-integral is trivial and t is integrated adaptively (scipy quad,
    split at the foot of the perpendicular where the integrand peaks)."""
    tot = 0.0
    for e in range(3):
        a, b = v[e], v[(e + 1) % 3]
        cr = np.linalg.norm(np.cross(a - x, b - a))
        foot = float(np.clip(-np.dot(a - x, b - a) / np.dot(b - a, b - a), 0.0, 1.0))
        f = lambda t: 1.0 / np.linalg.norm((a - x) + t * (b - a))
        tot += cr * quad(f, 0.0, 1.0, points=[foot], epsabs=0, epsrel=1e-13, limit=200)[0]
    return tot / (4 * np.pi)


def test_self_integral_random_triangles(oracle):
    rng = np.random.default_rng(7)
    for _ in range(50):
        v = rng.normal(size=(3, 3))
        lam = rng.dirichlet([2, 2, 2])
        x = lam @ v
        ref = _duffy_self(v, x)
        got = oracle.self_V(v[0], v[1], v[2], x)
        assert abs(got - ref) < 1e-10 * abs(ref), (got, ref)
