"""Pins of the oracle's traversal (the method's whole hot path in FP64)
against closed forms, brute force over leaves, the limit surface and
invariants (CPU only)."""
import numpy as np
import pytest

import oracle as O
from tests import _geom as G

SIZE = O.ROOT_SIZE


def straight_cp(A, B, rA, rB=None):
    rB = rA if rB is None else rB
    pts = np.stack([A + k / 3.0 * (B - A) for k in range(4)])
    rad = np.array([rA + k / 3.0 * (rB - rA) for k in range(4)])[:, None]
    return np.concatenate([pts, rad], axis=1)


def aimed_ray(g, target, dist=5.0):
    w = g.standard_normal(3)
    w /= np.linalg.norm(w)
    return G.ray7(target - dist * w, w)


@pytest.mark.parametrize("depth", [0, 1, 2, 5, 8, 13, 18, 22])
def test_straight_cylinder_is_exact_at_every_depth(depth):
    # A straight, constant-radius fiber: every node's bounding cylinder is
    # the fiber itself and every plane is orthogonal to the axis, so every
    # depth must return the textbook ray / capped-cylinder entry.
    g = np.random.default_rng(1000 + depth)
    n_hit = 0
    for _ in range(200):
        A = g.uniform(-1, 1, 3)
        B = A + g.standard_normal(3)
        r = g.uniform(0.05, 0.3)
        cp = straight_cp(A, B, r)
        target = A + g.uniform(-0.2, 1.2) * (B - A) + 1.5 * r * g.uniform(-1, 1, 3)
        ray = aimed_ray(g, target)
        h = O.intersect(ray, cp, depth)
        ref = G.capped_cylinder_entry(ray[:3], ray[3:6], A, B, r)
        if ref is None:
            assert not h.hit
            continue
        assert h.hit
        n_hit += 1
        assert abs(h.t - ref) <= 1e-11 * max(1.0, ref)
        x = ray[:3] + h.t * ray[3:6]
        u_ref = np.clip(np.dot(x - A, B - A) / np.dot(B - A, B - A), 0, 1)
        assert abs(h.u - u_ref) <= 1e-10
    assert n_hit > 40


def test_fig5_four_cases():
    # Fig. 5: a cylinder along x partitioned by the plane x = 0.  The ray
    # entering left and leaving right visits (left, right), hits the left
    # half; the mirrored ray hits the right half; a ray meeting only the
    # right half never visits the left; a ray passing by visits neither.
    cp = straight_cp(np.array([-1.0, 0, 0]), np.array([1.0, 0, 0]), 0.5)
    down = np.array([0.0, 0, -1.0])

    def ray_through(a, b):
        a, b = np.asarray(a, float), np.asarray(b, float)
        return G.ray7(a, b - a)

    h = O.intersect(ray_through([-2, 0, 2], [1, 0, -2]), cp, 1)   # left, right
    assert h.hit and h.leaf == 0 and h.backtracks == 0
    h = O.intersect(ray_through([2, 0, 2], [-1, 0, -2]), cp, 1)   # right, left
    assert h.hit and h.leaf == SIZE // 2 and h.backtracks == 0
    h = O.intersect(G.ray7([0.5, 0, 2], down), cp, 1)             # right only
    assert h.hit and h.leaf == SIZE // 2
    h = O.intersect(ray_through([-5, 0, 2], [3, 0, 4.5]), cp, 1)  # neither
    assert not h.hit and h.nodes == 1


@pytest.mark.parametrize("depth", [0, 2, 4, 7, 10])
def test_tapered_fiber_hits_leaf_cylinder_of_larger_end_radius(depth):
    # Straight axis, radius linear in u: a leaf's conservative radius is the
    # larger of its two end radii, so a lateral hit lies exactly that far
    # from the axis, on the leaf whose axial range contains it.
    g = np.random.default_rng(2000 + depth)
    checked = 0
    for _ in range(300):
        A = g.uniform(-1, 1, 3)
        B = A + 2.0 * g.standard_normal(3)
        rA, rB = g.uniform(0.05, 0.4, 2)
        cp = straight_cp(A, B, rA, rB)
        target = A + g.uniform(0.05, 0.95) * (B - A) + 0.3 * g.uniform(-1, 1, 3)
        ray = aimed_ray(g, target)
        h = O.intersect(ray, cp, depth)
        if not h.hit:
            continue
        x = ray[:3] + h.t * ray[3:6]
        ax = (B - A) / np.linalg.norm(B - A)
        s = np.dot(x - A, ax) / np.linalg.norm(B - A)
        rho = np.linalg.norm((x - A) - np.dot(x - A, ax) * ax)
        n = 1 << depth
        leaf = h.leaf * n // SIZE
        u0, u1 = leaf / n, (leaf + 1) / n
        if not (u0 + 1e-9 < s < u1 - 1e-9):
            continue  # end-cap hit of the leaf
        r_leaf = max(rA + u0 * (rB - rA), rA + u1 * (rB - rA))
        assert abs(rho - r_leaf) < 1e-10
        checked += 1
    assert checked > 30


def test_tapered_fiber_converges_to_cone():
    # Limit surface of a straight tapered fiber: the cone frustum.  The
    # depth-d hit lies on leaf cylinders at most |rB - rA| 2^-d wider.
    g = np.random.default_rng(31)
    for _ in range(60):
        A = g.uniform(-1, 1, 3)
        B = A + 2.0 * g.standard_normal(3)
        rA, rB = g.uniform(0.05, 0.4, 2)
        cp = straight_cp(A, B, rA, rB)
        target = A + g.uniform(0.1, 0.9) * (B - A) + 0.3 * min(rA, rB) * g.uniform(-1, 1, 3)
        ray = aimed_ray(g, target)
        ref = G.cone_frustum_entry(ray[:3], ray[3:6], A, B, rA, rB)
        assert ref is not None
        ax = (B - A) / np.linalg.norm(B - A)
        sin_ray_axis = np.linalg.norm(np.cross(ray[3:6], ax))
        for depth in (6, 10, 14, 18, 22):
            h = O.intersect(ray, cp, depth)
            assert h.hit
            assert h.t <= ref + 1e-12  # leaf cylinders contain the cone
            # the hit lies between the cone and the cone widened by the leaf's
            # radius spread, so the ray travels at most that spread over the
            # sine of its angle to the axis
            bound = abs(rB - rA) * 2.0 ** -depth / max(sin_ray_axis, 1e-3)
            assert ref - h.t <= 4 * bound + 1e-12


def _brute_force(ray, cp, depth):
    """Closest entry over all 2^depth leaf volumes, each built from its
    definition: the sub-curve's chord, radius = farthest inner control point
    from the chord + largest control radius, end planes normal to the
    sub-curve's end tangents."""
    o, w = ray[:3], ray[3:6]
    n = 1 << depth
    best = None
    for i in range(n):
        P = G.subcurve(cp, i / n, (i + 1) / n)
        A, B = P[0, :3], P[3, :3]
        ax = B - A
        ax_u = ax / np.linalg.norm(ax)
        dist = max(np.linalg.norm((P[k, :3] - A) - np.dot(P[k, :3] - A, ax_u) * ax_u) for k in (1, 2))
        r = dist + P[:, 3].max()
        t = G.capped_cylinder_entry(o, w, A, B, r, P[1, :3] - P[0, :3], P[3, :3] - P[2, :3])
        if t is not None and (best is None or t < best[0]):
            best = (t, i)
    return best


@pytest.mark.parametrize("depth", [0, 1, 3, 6, 8])
def test_traversal_equals_brute_force_over_leaves(depth):
    # Disjoint bounding volumes visited near-first (Sec. 3.2): the first leaf
    # the traversal reaches is the closest leaf volume overall.  Rays whose
    # closest leaf hit lies in the slack of an ancestor's cylinder may differ;
    # their share is bounded.
    g = np.random.default_rng(3000 + depth)
    n, agree, both_hit = 0, 0, 0
    for _ in range(150):
        cp = G.random_valid_cubic(g, jitter=0.25, rmin=0.02, rmax=0.08)
        target = G.curve_eval(cp, g.uniform(0, 1))[:3] + 0.1 * g.uniform(-1, 1, 3)
        ray = aimed_ray(g, target)
        h = O.intersect(ray, cp, depth)
        bf = _brute_force(ray, cp, depth)
        n += 1
        if (bf is None) == (not h.hit):
            if bf is None:
                agree += 1
            elif abs(h.t - bf[0]) <= 1e-10 * max(1, bf[0]):
                agree += 1
                both_hit += 1
                assert h.leaf == bf[1] * (SIZE >> depth)
    assert both_hit > 30
    assert agree >= 0.97 * n


def test_traversal_converges_to_limit_surface():
    # Sec. 3.2: the cylinders' limit surface; depth-d error shrinks at least
    # geometrically and is below 1e-6 r at depth 22.
    g = np.random.default_rng(41)
    got = 0
    for _ in range(40):
        cp = G.random_valid_cubic(g, jitter=0.2, rmin=0.02, rmax=0.06)
        if not O.thick_ok(cp):
            continue
        u = g.uniform(0.2, 0.8)
        c = G.curve_eval(cp, u)
        tgt = c[:3] + 0.5 * c[3] * g.uniform(-1, 1, 3)
        ray = aimed_ray(g, tgt)
        kind, tl, ul = O.limit_hit(ray, cp, 20000)
        if kind != 1:
            continue
        errs = []
        for depth in (8, 12, 16, 20, 22):
            h = O.intersect(ray, cp, depth)
            assert h.hit
            errs.append(abs(h.t - tl))
        if errs[0] > 1e-3:
            continue  # silhouette-adjacent at coarse depth
        got += 1
        # taper and curvature errors of the leaf cylinders shrink as 2^-d and
        # 4^-d: with radii <= 0.06 and rays well inside the silhouette the
        # error stays below 2^-d at every depth
        for depth, e in zip((8, 12, 16, 20, 22), errs):
            assert e <= 2.0 ** -depth
        assert errs[-1] < 1e-5 * cp[:, 3].min()
        h = O.intersect(ray, cp, 22)
        assert abs(h.u - ul) < 1e-5
    assert got > 10


@pytest.mark.parametrize("depth", [2, 8, 16])
def test_reversed_curve_gives_same_t_and_mirrored_u(depth):
    # The construction is symmetric in the curve direction: reversing the
    # control points maps every leaf, radius and plane onto itself.
    g = np.random.default_rng(5000 + depth)
    checked = 0
    for _ in range(100):
        cp = G.random_valid_cubic(g, jitter=0.3)
        target = G.curve_eval(cp, g.uniform(0, 1))[:3] + 0.05 * g.uniform(-1, 1, 3)
        ray = aimed_ray(g, target)
        a = O.intersect(ray, cp, depth)
        b = O.intersect(ray, cp[::-1].copy(), depth)
        assert a.hit == b.hit
        if a.hit:
            checked += 1
            assert abs(a.t - b.t) <= 1e-9 * max(1, a.t)
            assert abs(a.u - (1 - b.u)) <= 1e-9
    assert checked > 20


def test_rigid_motion_invariance():
    # Results depend only on the relative geometry of ray and curve.
    g = np.random.default_rng(61)
    for _ in range(50):
        cp = G.random_valid_cubic(g, jitter=0.3)
        target = G.curve_eval(cp, g.uniform(0, 1))[:3] + 0.05 * g.uniform(-1, 1, 3)
        ray = aimed_ray(g, target)
        q, _ = np.linalg.qr(g.standard_normal((3, 3)))
        if np.linalg.det(q) < 0:
            q[:, 0] *= -1
        shift = g.uniform(-10, 10, 3)
        cp2 = cp.copy()
        cp2[:, :3] = cp[:, :3] @ q.T + shift
        ray2 = G.ray7(q @ ray[:3] + shift, q @ ray[3:6])
        a, b = O.intersect(ray, cp, 10), O.intersect(ray2, cp2, 10)
        assert a.hit == b.hit
        if a.hit:
            assert abs(a.t - b.t) <= 1e-9 * max(1, a.t)
            assert abs(a.u - b.u) <= 1e-9


def test_closest_equals_min_over_pairs():
    # Per-ray closest hit is the minimum over the ray's per-pair hits, ties to
    # the earlier candidate.
    from paper_1811_03374_gb300 import inputs as I
    case = I.tiny_case(n_ray=2048)
    pc = O.presplit(case["cps"])
    cl = O.closest(case, 8, pc)
    pr = O.pairs(case, 8, pc)
    tp = pr["t"].reshape(2048, 16)
    ref = tp.min(axis=1)
    np.testing.assert_array_equal(ref, cl["t"])
    hit = np.isfinite(cl["t"])
    np.testing.assert_array_equal(cl["seg"][hit], np.argmin(tp, axis=1)[hit])
    assert cl["counters"]["tests"] == 2048 * len(pc["seg"])


def test_node_counts_of_a_direct_hit():
    # A hit found without backtracking tests exactly depth + 1 nodes.
    cp = straight_cp(np.array([-1.0, 0, 0]), np.array([1.0, 0, 0]), 0.5)
    for depth in (0, 3, 9, 17):
        h = O.intersect(G.ray7([0.3, 0.1, 5.0], [0, 0, -1.0]), cp, depth)
        assert h.hit and h.nodes == depth + 1 and h.descents == depth and h.backtracks == 0
        assert abs(h.t - (5.0 - np.sqrt(0.25 - 0.01))) < 1e-14
