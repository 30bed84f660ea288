"""Pins of the oracle's quadratic fibers (App. B.1 constraint; intersection
as the raised cubic) against closed forms, brute force and the
paper's figure (CPU only)."""
import os

import numpy as np
import pytest

import oracle as O
from tests import _geom as G
from tests.test_oracle_traversal import aimed_ray

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def quad_eval(q, u):
    """Quadratic Bezier by de Casteljau (two rounds of linear interpolation)."""
    a = (1 - u) * q[0] + u * q[1]
    b = (1 - u) * q[1] + u * q[2]
    return (1 - u) * a + u * b


def cubic_bernstein(c, u):
    v = 1 - u
    return v ** 3 * c[0] + 3 * u * v * v * c[1] + 3 * u * u * v * c[2] + u ** 3 * c[3]


def random_quadratic(g, valid=None):
    while True:
        q = np.concatenate([g.uniform(-1, 1, (3, 3)), g.uniform(0.01, 0.1, (3, 1))], axis=1)
        if valid is None or O.valid_quadratic(q) == valid:
            return q


def test_elevation_is_the_same_curve():
    # the raised cubic evaluates to the quadratic at every parameter, all four
    # components (position and radius)
    g = np.random.default_rng(1)
    for _ in range(200):
        q = random_quadratic(g)
        c = O.elevate_quadratics(q[None])[0]
        for u in np.linspace(0, 1, 33):
            np.testing.assert_allclose(cubic_bernstein(c, u), quad_eval(q, u), atol=1e-14)


def test_golden_figure():
    rows = np.loadtxt(os.path.join(GOLD, "fig_quadratic_constraint.txt"))
    q, prods = rows[:3], rows[3, :3]
    p0, p1, p2 = q[:, :3]
    np.testing.assert_allclose([np.dot(p1 - p0, p1 - p2), np.dot(p1 - p0, p2 - p0), np.dot(p1 - p2, p0 - p2)],
                               prods)
    assert O.valid_quadratic(q)
    # moving p1 out of the band through p2's plane breaks the constraint
    q2 = q.copy()
    q2[1, 0] = 5.0
    assert not O.valid_quadratic(q2)


def _halves(q):
    """Control points of the two halves (de Casteljau at u = 1/2), the split
    point and the tangent there."""
    l1, r1 = (q[0] + q[1]) / 2, (q[1] + q[2]) / 2
    s = (l1 + r1) / 2
    return np.stack([q[0], l1, s]), np.stack([s, r1, q[2]]), s, q[2] - q[0]


def _separated(q):
    L, R, s, t = _halves(q[:, :3])
    return np.all((L - s) @ t <= 1e-15) and np.all((R - s) @ t >= -1e-15)


def test_constraint_separates_the_halves_and_is_kept_by_them():
    # App. B.1: the constraint puts each half's control points on its own
    # side of the plane through the split point orthogonal to the split
    # tangent, and both halves meet the constraint again (so every nested
    # subcurve does)
    g = np.random.default_rng(2)
    for _ in range(3000):
        q = random_quadratic(g, valid=True)
        assert _separated(q)
        L, R, _, _ = _halves(q[:, :3])
        for h in (L, R):
            assert O.valid_quadratic(np.concatenate([h, np.zeros((3, 1))], axis=1))


def test_constraint_is_sufficient_not_necessary():
    # halves can be separated while the constraint fails (the
    # lemma's one-sided conditions do not combine into it)
    q = np.array([[0.0, 0, 0, 0], [1.0, 0, 0, 0], [0.5, 1, 0, 0]])
    assert not O.valid_quadratic(q)
    assert _separated(q)


def test_valid_quadratic_raises_to_a_valid_cubic():
    # with a = p1 - p0, b = p2 - p1, each of the five cubic inequalities of
    # the raised curve is a non-negative combination of |a|^2, |b|^2 and
    # <a, b> >= 0: a valid quadratic is never pre-split
    g = np.random.default_rng(3)
    for _ in range(3000):
        q = random_quadratic(g, valid=True)
        assert O.valid_cubic(O.elevate_quadratics(q[None])[0])


@pytest.mark.parametrize("depth", [0, 4, 11, 19])
def test_straight_quadratic_is_the_capped_cylinder(depth):
    # p1 at the chord's midpoint, constant radius: the fiber is the capped
    # cylinder at every depth
    g = np.random.default_rng(4 + depth)
    n_hit = 0
    for _ in range(150):
        A = g.uniform(-1, 1, 3)
        B = A + g.standard_normal(3)
        r = g.uniform(0.05, 0.3)
        q = np.array([[*A, r], [*(A + B) / 2, r], [*B, r]])
        c = O.elevate_quadratics(q[None])[0]
        ray = aimed_ray(g, A + g.uniform(-0.2, 1.2) * (B - A) + 1.5 * r * g.uniform(-1, 1, 3))
        h = O.intersect(ray, c, depth)
        ref = G.capped_cylinder_entry(ray[:3], ray[3:6], A, B, r)
        if ref is None:
            assert not h.hit
            continue
        assert h.hit and abs(h.t - ref) <= 1e-11 * max(1.0, ref)
        n_hit += 1
    assert n_hit > 30


def test_quadratic_traversal_equals_brute_force_over_leaves():
    # the traversal of a raised quadratic returns the nearest of its 2^d leaf
    # cylinders (the plain definition of the depth-d fiber)
    g = np.random.default_rng(5)
    depth = 7
    for _ in range(60):
        q = random_quadratic(g, valid=True)
        c = O.elevate_quadratics(q[None])[0]
        target = quad_eval(q[:, :3], g.uniform(0, 1)) + 0.05 * g.uniform(-1, 1, 3)
        ray = aimed_ray(g, target)
        h = O.intersect(ray, c, depth)
        best = None
        for leaf in range(1 << depth):
            lh = O.leaf_hit(ray, c, depth, leaf)
            if lh is not None and (best is None or lh[0] < best[0]):
                best = lh
        if best is None:
            assert not h.hit
        else:
            assert h.hit and abs(h.t - best[0]) <= 1e-12 * max(1.0, best[0])
