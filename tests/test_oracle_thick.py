"""Pins of the oracle's end-plane check for thick fibers (Sec. 3.4, Fig. 7):
the exact polynomial criterion against dense sampling of the
distance the cross-sections keep from the end planes, straight fibers of any
radius, monotonicity in the radius, and the end-curvature limit (CPU only)."""
import numpy as np
import pytest

import oracle as O


def margin(cp, n=20001):
    """min over u of (distance of c(u) inside an end plane) - rbar sin(theta),
    theta the angle between c'(u) and the plane's normal, sampled densely
    (the end point itself, where both vanish, left out)."""
    P = cp[:, :3]
    rbar = cp[:, 3].max()
    u = np.linspace(0, 1, n)[:, None]
    v = 1 - u
    c = v ** 3 * P[0] + 3 * u * v * v * P[1] + 3 * u * u * v * P[2] + u ** 3 * P[3]
    t = v * v * (P[1] - P[0]) + 2 * u * v * (P[2] - P[1]) + u * u * (P[3] - P[2])
    tn = t / np.linalg.norm(t, axis=1, keepdims=True)
    out = []
    for nrm, p, sgn, sl in ((P[3] - P[2], P[3], 1, slice(0, n - 1)), (P[1] - P[0], P[0], -1, slice(1, n))):
        nh = nrm / np.linalg.norm(nrm)
        h = sgn * ((p - c) @ nh) - rbar * np.linalg.norm(np.cross(tn, nh), axis=1)
        out.append(h[sl].min())
    return min(out)


def bent(g, jitter=0.35, rmax=0.8):
    A = g.uniform(-1, 1, 3)
    B = A + g.standard_normal(3)
    L = np.linalg.norm(B - A)
    P = np.stack([A + k / 3 * (B - A) for k in range(4)])
    P[1:3] += jitter * L * g.uniform(-1, 1, (2, 3))
    r = np.full((4, 1), g.uniform(0.0, rmax) * L)
    return np.concatenate([P, r], axis=1)


def test_exact_check_matches_dense_sampling():
    g = np.random.default_rng(21)
    n = 0
    outcomes = set()
    for _ in range(1000):
        cp = bent(g)
        if not O.valid_cubic(cp):
            continue
        ok = O.thick_ok(cp)
        m = margin(cp)
        if abs(m) < 1e-6:
            continue  # tangent to a plane: below the sampling's resolution
        assert ok == (m >= 0), (cp.tolist(), m)
        outcomes.add(ok)
        n += 1
    assert n > 600 and outcomes == {True, False}


def test_straight_fibers_of_any_radius_pass():
    g = np.random.default_rng(22)
    for _ in range(200):
        A = g.uniform(-1, 1, 3)
        B = A + g.standard_normal(3)
        P = np.stack([A + k / 3 * (B - A) for k in range(4)])
        cp = np.concatenate([P, np.full((4, 1), g.uniform(0, 10))], axis=1)
        assert O.thick_ok(cp)


def test_monotone_in_the_radius():
    g = np.random.default_rng(23)
    for _ in range(300):
        cp = bent(g, rmax=0.0)
        if not O.valid_cubic(cp):
            continue
        res = []
        for r in np.linspace(0, 1.0, 21):
            cp[:, 3] = r
            res.append(O.thick_ok(cp))
        # once cropped, a thicker fiber stays cropped
        if False in res:
            assert not any(res[res.index(False):]), res


def test_end_curvature_limit():
    # near u = 1 the condition becomes rbar * curvature(1) <= 1: a curve
    # straight but for a tight end bend passes just below that radius and
    # fails just above it
    P = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0], [2.4, 0.3, 0]])
    d1 = 3 * (P[3] - P[2])
    d2 = 6 * (P[3] - 2 * P[2] + P[1])
    kappa = np.linalg.norm(np.cross(d1, d2)) / np.linalg.norm(d1) ** 3
    r_lim = 1.0 / kappa
    cp = np.concatenate([P, np.zeros((4, 1))], axis=1)
    assert O.valid_cubic(cp)
    cp[:, 3] = 0.999 * r_lim
    m_below = margin(cp)
    cp[:, 3] = 1.001 * r_lim
    assert not O.thick_ok(cp)
    cp[:, 3] = 0.999 * r_lim
    assert O.thick_ok(cp) == (m_below >= 0)
