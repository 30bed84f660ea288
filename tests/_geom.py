"""Textbook geometry for pinning the oracle (numpy, float64, world frame).

Nothing here follows the paper's unit-ray formulation: curves are evaluated
through their power-basis matrix, cylinders and cones are solved as quadratics
in world coordinates, planes by signed distances.  These are the independent
references the oracle is checked against.
"""
import numpy as np

# Bernstein -> power basis: c(u) = sum_j u^j * (M @ P)[j]
BEZ_M = np.array([[1, 0, 0, 0], [-3, 3, 0, 0], [3, -6, 3, 0], [-1, 3, -3, 1]], dtype=np.float64)


def curve_eval(cp, u):
    """cp [4, k] control rows; u scalar or array -> points [..., k]."""
    coef = BEZ_M @ np.asarray(cp, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    return sum(np.multiply.outer(u ** j, coef[j]) for j in range(4))


def curve_deriv(cp, u):
    coef = BEZ_M @ np.asarray(cp, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    return sum(j * np.multiply.outer(u ** (j - 1), coef[j]) for j in range(1, 4))


def subcurve(cp, u0, u1):
    """Control points of the restriction of the cubic to [u0, u1], from the
    blossom: the control points are the values at the sub-interval's ends plus
    tangent thirds (c(u0), c(u0) + h c'(u0)/3, c(u1) - h c'(u1)/3, c(u1))."""
    h = u1 - u0
    a, b = curve_eval(cp, u0), curve_eval(cp, u1)
    da, db = curve_deriv(cp, u0), curve_deriv(cp, u1)
    return np.stack([a, a + h * da / 3.0, b - h * db / 3.0, b])


def ray_infinite_cylinder(o, w, A, axis, r):
    """Entry/exit t of the ray o + t w (any t) with the infinite cylinder of
    radius r around the line A + s axis; None if it misses."""
    a = axis / np.linalg.norm(axis)
    m = o - A
    wp = w - np.dot(w, a) * a
    mp = m - np.dot(m, a) * a
    qa, qb, qc = np.dot(wp, wp), 2 * np.dot(wp, mp), np.dot(mp, mp) - r * r
    if qa == 0.0:
        return (-np.inf, np.inf) if qc < 0 else None
    disc = qb * qb - 4 * qa * qc
    if disc < 0:
        return None
    s = np.sqrt(disc)
    return ((-qb - s) / (2 * qa), (-qb + s) / (2 * qa))


def halfspace_interval(o, w, P, n, keep_positive):
    """t-interval where sign(<o + t w - P, n>) is kept (>= 0 if keep_positive)."""
    f0, f1 = np.dot(o - P, n), np.dot(w, n)
    sgn = 1.0 if keep_positive else -1.0
    f0, f1 = sgn * f0, sgn * f1
    if f1 == 0.0:
        return (-np.inf, np.inf) if f0 >= 0 else (np.inf, -np.inf)
    t = -f0 / f1
    return (t, np.inf) if f1 > 0 else (-np.inf, t)


def capped_cylinder_entry(o, w, A, B, r, nA=None, nB=None, tmax=np.inf):
    """Entry t >= 0 into the cylinder of radius r around segment A-B, cropped
    by the plane through A with normal nA (kept side towards B) and the plane
    through B with normal nB (kept side towards A).  Default normals: the
    axis (a right cylinder)."""
    axis = B - A
    if nA is None:
        nA = axis
    if nB is None:
        nB = axis
    c = ray_infinite_cylinder(o, w, A, axis, r)
    if c is None:
        return None
    s0 = halfspace_interval(o, w, A, nA, True)
    s1 = halfspace_interval(o, w, B, nB, False)
    lo = max(c[0], s0[0], s1[0], 0.0)
    hi = min(c[1], s0[1], s1[1], tmax)
    if lo > hi:
        return None
    return lo


def cone_frustum_entry(o, w, A, B, rA, rB):
    """First t >= 0 where the ray enters the solid cone frustum around A-B with
    radius rA at A and rB at B (flat end disks)."""
    L = np.linalg.norm(B - A)
    a = (B - A) / L
    m = o - A
    al, be = np.dot(a, w), np.dot(a, m)
    k = (rB - rA) / L
    r0 = rA + k * be
    qa = 1 - al * al - k * k * al * al
    qb = 2 * (np.dot(m, w) - al * be - k * al * r0)
    qc = np.dot(m, m) - be * be - r0 * r0
    cands = []
    if qa != 0.0:
        disc = qb * qb - 4 * qa * qc
        if disc >= 0:
            for t in ((-qb - np.sqrt(disc)) / (2 * qa), (-qb + np.sqrt(disc)) / (2 * qa)):
                s = be + al * t
                if t >= 0 and 0 <= s <= L and rA + k * s >= 0:
                    cands.append(t)
    for P, rr in ((A, rA), (B, rB)):
        if al != 0.0:
            t = np.dot(P - o, a) / al
            x = o + t * w
            if t >= 0 and np.dot(x - P, x - P) <= rr * rr:
                cands.append(t)
    return min(cands) if cands else None


def ray7(o, w, tmax=np.inf):
    w = np.asarray(w, dtype=np.float64)
    w = w / np.linalg.norm(w)
    return np.array([o[0], o[1], o[2], w[0], w[1], w[2], tmax], dtype=np.float64)


def random_valid_cubic(g, jitter=0.3, rmin=0.01, rmax=0.05, max_tries=1000):
    """Random cubic satisfying the five inequalities, found by rejection; the
    check here is written from the inequalities directly."""
    for _ in range(max_tries):
        p0 = g.uniform(-1, 1, 3)
        d = g.standard_normal(3)
        d /= np.linalg.norm(d)
        p3 = p0 + d * g.uniform(0.5, 2.0)
        p1 = p0 + (p3 - p0) / 3 + jitter * g.standard_normal(3)
        p2 = p0 + 2 * (p3 - p0) / 3 + jitter * g.standard_normal(3)
        P = np.stack([p0, p1, p2, p3])
        ok = all(np.dot(a, b) >= 0 for a, b in [
            (P[2] - P[0], P[1] - P[0]), (P[3] - P[1], P[1] - P[0]), (P[3] - P[1], P[3] - P[2]),
            (P[2] - P[0], P[3] - P[2]), (P[2] - P[0], P[3] - P[1])])
        if ok:
            r = g.uniform(rmin, rmax, (4, 1))
            return np.concatenate([P, r], axis=1)
    raise RuntimeError("no valid cubic found")
