"""Pins of the oracle's limit-surface hit and its implicit-function gradient
dt/d(control points, radii) (CPU only)."""
import numpy as np
import pytest

import oracle as O
from tests import _geom as G


def forced_hit(g, jitter=0.2):
    for _ in range(100):
        cp = G.random_valid_cubic(g, jitter=jitter, rmin=0.02, rmax=0.06)
        if not O.thick_ok(cp):
            continue
        u = g.uniform(0.15, 0.85)
        c = G.curve_eval(cp, u)
        w = g.standard_normal(3)
        w /= np.linalg.norm(w)
        tgt = c[:3] + 0.5 * c[3] * g.uniform(-1, 1, 3)
        ray = G.ray7(tgt - 3.0 * w, w)
        kind, t, uu = O.limit_hit(ray, cp, 20000)
        if kind == 1:
            return cp, ray, t, uu
    raise RuntimeError("no lateral hit")


def _straight(A, B, rk):
    return np.concatenate([np.stack([A + k / 3 * (B - A) for k in range(4)]),
                           np.asarray(rk, float).reshape(4, 1)], 1)


def test_limit_hit_straight_cylinder_closed_form():
    # constant radius: the limit surface is the capped cylinder itself
    A, B, r = np.array([0.0, 0, 0]), np.array([2.0, 0, 0]), 0.3
    cp = _straight(A, B, [r] * 4)
    ray = G.ray7([0.2, 0.1, 4.0], [0.3, 0.05, -1.0])
    kind, t, u = O.limit_hit(ray, cp, 10000)
    ref = G.capped_cylinder_entry(ray[:3], ray[3:6], A, B, r)
    assert kind == 1
    assert abs(t - ref) < 1e-13
    x = ray[:3] + t * ray[3:6]
    assert abs(u - x[0] / 2.0) < 1e-12
    # end disk: a ray along the axis enters through the disk at u = 0
    kind, t, u = O.limit_hit(G.ray7([-1.0, 0.05, 0.0], [1.0, 0, 0]), cp, 10000)
    assert kind == 2 and abs(t - 1.0) < 1e-14 and u == 0.0


@pytest.mark.parametrize("seed", range(6))
def test_limit_hit_point_lies_on_the_sweep(seed):
    # G1 = G2 = 0 at the returned (t, u): the point is in the normal plane of
    # c(u) at distance r(u).
    g = np.random.default_rng(700 + seed)
    cp, ray, t, u = forced_hit(g)
    x = ray[:3] + t * ray[3:6]
    c = G.curve_eval(cp, u)
    dc = G.curve_deriv(cp, u)
    assert abs(np.dot(x - c[:3], dc[:3])) < 1e-12
    assert abs(np.linalg.norm(x - c[:3]) - c[3]) < 1e-12
    # and no earlier point of the ray is inside the swept solid (dense check)
    ts = np.linspace(0, t, 4001)[:-1]
    us = np.linspace(0, 1, 2001)
    C = G.curve_eval(cp, us)
    D = G.curve_deriv(cp, us)
    for tt in ts[::40]:
        p = ray[:3] + tt * ray[3:6]
        rel = p - C[:, :3]
        in_plane = np.abs(np.einsum("ij,ij->i", rel, D[:, :3])) < 1e-3 * np.linalg.norm(D[:, :3], axis=1)
        assert not np.any(in_plane & (np.linalg.norm(rel, axis=1) < C[:, 3] * (1 - 1e-3)))


def _fd_grad(ray, cp, h=1e-6):
    grad = np.zeros((4, 4))
    for k in range(4):
        for a in range(4):
            cpp, cpm = cp.copy(), cp.copy()
            cpp[k, a] += h
            cpm[k, a] -= h
            kp, tp, _ = O.limit_hit(ray, cpp, 20000)
            km, tm, _ = O.limit_hit(ray, cpm, 20000)
            assert kp == 1 and km == 1
            grad[k, a] = (tp - tm) / (2 * h)
    return grad


@pytest.mark.parametrize("seed", range(6))
def test_ift_gradient_matches_central_differences(seed):
    g = np.random.default_rng(800 + seed)
    cp, ray, t, u = forced_hit(g)
    grad = O.grad_t(ray, cp, t, u)
    fd = _fd_grad(ray, cp)
    err = np.linalg.norm(grad - fd) / np.linalg.norm(fd)
    assert err < 1e-6


@pytest.mark.parametrize("seed", range(6))
def test_gradient_homogeneity_and_translation(seed):
    # t is homogeneous of degree one in (p_k - o, r_k):
    #   sum_k <dt/dp_k, p_k - o> + dt/dr_k r_k = t,
    # and moving the fiber along the ray by e moves the hit by e:
    #   sum_k <dt/dp_k, w> = 1.
    g = np.random.default_rng(900 + seed)
    cp, ray, t, u = forced_hit(g)
    grad = O.grad_t(ray, cp, t, u)
    o, w = ray[:3], ray[3:6]
    euler = np.sum(grad[:, :3] * (cp[:, :3] - o)) + np.sum(grad[:, 3] * cp[:, 3])
    assert abs(euler - t) < 1e-10 * t
    assert abs(np.sum(grad[:, :3] @ w) - 1.0) < 1e-10


def test_gradient_straight_cylinder_closed_form():
    # Constant-radius straight fiber: growing r_k by e moves the surface
    # outward along the normal n by B_k(u) e, so the hit moves by
    # dt/dr_k = -B_k(u) / <-w, n>; translating the fiber along the ray moves
    # the hit by the same amount (sum_k dt/dp_k . w = 1).
    A, B = np.array([0.0, 0, 0]), np.array([2.0, 0, 0])
    cp = _straight(A, B, [0.3] * 4)
    ray = G.ray7([0.2, 0.1, 4.0], [0.3, 0.05, -1.0])
    kind, t, u = O.limit_hit(ray, cp, 20000)
    assert kind == 1
    grad = O.grad_t(ray, cp, t, u)
    x = ray[:3] + t * ray[3:6]
    n = np.array([0.0, x[1], x[2]]) / np.hypot(x[1], x[2])
    Bu = np.array([(1 - u) ** 3, 3 * u * (1 - u) ** 2, 3 * u * u * (1 - u), u ** 3])
    np.testing.assert_allclose(grad[:, 3], -Bu / np.dot(-ray[3:6], n), rtol=1e-10)
    assert abs(grad[:, :3].sum(axis=0) @ ray[3:6] - 1.0) < 1e-10


def test_gradient_end_disk():
    # End-disk hit at u = 0: t = <c(0) - o, c'(0)> / <w, c'(0)>; only p0 and
    # p1 enter, radii not at all.
    A, B = np.array([0.0, 0, 0]), np.array([2.0, 0, 0])
    cp = np.concatenate([np.stack([A + k / 3 * (B - A) for k in range(4)]), np.full((4, 1), 0.3)], 1)
    ray = G.ray7([-1.0, 0.05, 0.1], [1.0, 0, 0])
    kind, t, u = O.limit_hit(ray, cp, 10000)
    assert kind == 2
    grad = O.grad_t(ray, cp, t, u)
    np.testing.assert_allclose(grad[:, 3], 0.0, atol=0)
    np.testing.assert_allclose(grad[2:, :3], 0.0, atol=1e-15)
    # moving p0 along the ray moves the disk plane: dt/dp0 . w = 1 here
    assert abs(grad[0, :3] @ ray[3:6] - 1.0) < 1e-12
