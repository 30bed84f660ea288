"""Pins of the oracle's hit normal (App. C: the hit point minus its
projection onto the hit leaf's axis, or the outward end-disk normal for a
hit on an end disk -- one on or beyond the segment's end plane)
against closed forms, the limit surface and invariants (CPU only)."""
import numpy as np
import pytest

import oracle as O
from paper_1811_03374_gb300 import inputs as I
from tests import _geom as G
from tests.test_oracle_traversal import aimed_ray, straight_cp

SIZE = O.ROOT_SIZE


def _normal_of_hit(ray, cp, depth):
    h = O.intersect(ray, cp, depth)
    if not h.hit:
        return None
    n, kind, u = O.normal(ray, cp, h.leaf, SIZE >> depth, h.t)
    return h, n, kind, u


@pytest.mark.parametrize("depth", [0, 3, 9, 16, 22])
def test_straight_cylinder_normal_is_radial(depth):
    # Every leaf of a straight constant-radius fiber has the fiber's axis as
    # its own: a lateral hit's normal is the textbook cylinder normal, the
    # hit point minus its projection onto the axis, over the radius.
    g = np.random.default_rng(2000 + depth)
    n_lat = 0
    for _ in range(300):
        A = g.uniform(-1, 1, 3)
        B = A + g.standard_normal(3)
        r = g.uniform(0.05, 0.3)
        cp = straight_cp(A, B, r)
        ray = aimed_ray(g, A + g.uniform(0.05, 0.95) * (B - A) + 1.2 * r * g.uniform(-1, 1, 3))
        res = _normal_of_hit(ray, cp, depth)
        if res is None:
            continue
        h, n, kind, u = res
        if kind != 1:
            continue
        x = ray[:3] + h.t * ray[3:6]
        a = (B - A) / np.linalg.norm(B - A)
        radial = (x - A) - np.dot(x - A, a) * a
        rho = np.linalg.norm(radial)
        # the hit point minus its projection onto the axis, normalised; on the
        # lateral surface that vector is r long (a ray entering through an end
        # disk whose projection lands a rounding away from u = 0 or 1 is
        # lateral by the paper's exact test, inside the cylinder)
        # (a depth-d leaf's chord c(u1) - c(u0) carries a relative FP64 error
        # of about 2^-52 / 2^-d, 1e-9 at depth 22)
        np.testing.assert_allclose(n, radial / rho, atol=1e-8)
        if abs(rho - r) <= 1e-10:
            n_lat += 1
    assert n_lat > 60


@pytest.mark.parametrize("depth", [0, 5, 14])
def test_end_disk_normal_is_the_outward_axis(depth):
    # A ray entering through the flat end disk at u = 0 (u = 1) gets the
    # normal p0 - p1 (p3 - p2), normalised: minus (plus) the axis direction.
    g = np.random.default_rng(3000 + depth)
    n_cap = [0, 0]
    for _ in range(200):
        A = g.uniform(-1, 1, 3)
        B = A + g.standard_normal(3)
        a = (B - A) / np.linalg.norm(B - A)
        r = g.uniform(0.1, 0.3)
        cp = straight_cp(A, B, r)
        end = g.integers(0, 2)
        P, out = (A, -a) if end == 0 else (B, a)
        # a point on the disk, approached from outside through the disk
        e = np.cross(a, g.standard_normal(3))
        e /= np.linalg.norm(e)
        q = P + 0.7 * r * g.uniform() * e
        w = -out + 0.3 * np.cross(out, e)
        w /= np.linalg.norm(w)
        ray = G.ray7(q - 2.0 * w, w)
        res = _normal_of_hit(ray, cp, depth)
        assert res is not None
        h, n, kind, u = res
        assert kind == 2 + end and abs(u - end) <= 1e-9
        np.testing.assert_allclose(n, out, atol=1e-12)
        assert abs(h.t - 2.0) <= 1e-9
        n_cap[end] += 1
    assert min(n_cap) > 50


def test_curved_normal_converges_to_the_limit_surface():
    # At depth 22 the leaf axis is the curve's tangent to within 2^-22 of the
    # parameter: the normal is the radial direction of the limit surface's
    # circle through the hit, (x - c(u)) orthogonalised against c'(u).
    case = I.sweep_case("moderate", 400, forced_hits=True)
    checked = 0
    for i in range(400):
        ray = O.ray7_from_packed(case["rays"][i])
        cp = case["cps"][i].astype(np.float64)
        if not O.valid_cubic(cp):
            continue
        res = _normal_of_hit(ray, cp, 22)
        if res is None or res[2] != 1:
            continue
        h, n, kind, u = res
        x = ray[:3] + h.t * ray[3:6] / np.linalg.norm(ray[3:6])  # the packed direction is FP32
        c = I.bezier(cp[None], np.array([u]))[0, :3]
        tg = I.bezier_tangent(cp[None], np.array([u]))[0, :3]
        tg /= np.linalg.norm(tg)
        v = (x - c) - np.dot(x - c, tg) * tg
        if np.linalg.norm(x - c) < 0.5 * np.max(cp[:, 3]):
            continue  # hit through an end plane, near the axis
        # the leaf chord turns from the tangent by about 2^-22 times the
        # curvature, and the axis point lies within O(2^-44) of c(u)
        ang = np.arccos(np.clip(np.dot(n, v / np.linalg.norm(v)), -1, 1))
        assert ang <= 1e-6, (i, ang)
        checked += 1
    assert checked > 300


def test_normal_invariants():
    # unit length; front-facing entries; rigid-motion covariance; reversal
    g = np.random.default_rng(7)
    case = I.sweep_case("curved", 300, forced_hits=True)
    Rm, _ = np.linalg.qr(g.standard_normal((3, 3)))
    shift = g.uniform(-3, 3, 3)
    front = tot = 0
    for i in range(300):
        ray = O.ray7_from_packed(case["rays"][i])
        cp = case["cps"][i].astype(np.float64)
        for depth in (6, 15):
            res = _normal_of_hit(ray, cp, depth)
            if res is None:
                continue
            h, n, kind, u = res
            assert abs(np.linalg.norm(n) - 1.0) <= 1e-12
            tot += 1
            front += np.dot(n, ray[3:6]) <= 1e-12
            # rigid motion of ray and curve
            cp2 = cp.copy()
            cp2[:, :3] = cp[:, :3] @ Rm.T + shift
            ray2 = np.concatenate([Rm @ ray[:3] + shift, Rm @ ray[3:6], ray[6:]])
            h2, n2, kind2, u2 = _normal_of_hit(ray2, cp2, depth)
            assert kind2 == kind and h2.leaf == h.leaf
            np.testing.assert_allclose(n2, Rm @ n, atol=1e-8)
            # reversed control points: the same surface point, u -> 1 - u
            cpr = cp[::-1].copy()
            hr, nr, kindr, ur = _normal_of_hit(ray, cpr, depth)
            assert {1: 1, 2: 3, 3: 2}[kind] == kindr
            np.testing.assert_allclose(nr, n, atol=1e-8)
    assert tot > 300
    # an entry point faces the ray, except where the ray enters a leaf through
    # one of its planes (inside the leaf cylinder)
    assert front >= 0.9 * tot, (front, tot)
