"""Pins of the FP64 oracle's building blocks against textbook definitions and
values printed in the paper's figures (CPU only)."""
import os

import numpy as np
import pytest

import oracle as O
from tests import _geom as G

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLD, name))


def test_fig3_curve_is_valid():
    # Fig. 3 draws an ordinary curve in the (p, d, t0, t1) representation.
    assert O.valid_cubic(_load("fig3_representation.txt"))


def test_fig4_loop_is_invalid():
    # Fig. 4: the loop, which violates the constraints, must be rejected.
    cp = _load("fig4_loop.txt")
    assert not O.valid_cubic(cp)
    P = cp[:, :3]
    assert np.dot(P[2] - P[0], P[1] - P[0]) == -4.0


def test_cubic_lemma_split_point_and_tangent():
    # App. B.2: s = (p0 + 3p1 + 3p2 + p3)/8, t = 3/4 (-p0 - p1 + p2 + p3).
    g = _load("fig_cubic_split.txt")
    cp, s, t = g[:4], g[4], g[5]
    node = O.node_at(cp, 0, O.ROOT_SIZE)
    left = O.subdivide(node, 0)
    right = O.subdivide(node, 1)
    # left child ends at the split point, right child starts there
    np.testing.assert_allclose(left[0] + left[1], s, atol=1e-15)
    np.testing.assert_allclose(right[0], s, atol=1e-15)
    # tangent at the split: left.t1 == right.t0 == t_c == (u1 - u0)/3 * c'(1/2)
    # with u1 - u0 = 1/2 for a child, i.e. t / 6
    np.testing.assert_allclose(left[3], t / 6.0, atol=1e-15)
    np.testing.assert_allclose(right[2], t / 6.0, atol=1e-15)


def _node_to_cp(node):
    p, d, t0, t1 = node
    return np.stack([p, p + t0, p + d - t1, p + d])


@pytest.mark.parametrize("seed", range(5))
def test_subdivision_rules_give_the_half_curves(seed):
    # Sec. 3.1: the (p, d, t0, t1) children are the curve restricted to
    # [0, 1/2] and [1/2, 1]; compared with the power-basis restriction.
    g = np.random.default_rng(seed)
    cp = np.concatenate([g.uniform(-2, 2, (4, 3)), g.uniform(0, 0.1, (4, 1))], axis=1)
    node = O.node_at(cp, 0, O.ROOT_SIZE)
    for go_right, (u0, u1) in ((0, (0.0, 0.5)), (1, (0.5, 1.0))):
        child = _node_to_cp(O.subdivide(node, go_right))
        np.testing.assert_allclose(child, G.subcurve(cp, u0, u1), atol=1e-14)
    # repeated: a random path down to depth 12 equals the dyadic sub-curve
    start, size = 0, O.ROOT_SIZE
    for lvl in range(12):
        gr = int(g.integers(0, 2))
        node = O.subdivide(node, gr)
        size //= 2
        start += gr * size
    u0, u1 = start / O.ROOT_SIZE, (start + size) / O.ROOT_SIZE
    np.testing.assert_allclose(_node_to_cp(node), G.subcurve(cp, u0, u1), atol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_node_recompute_matches_subcurve(seed):
    # Sec. 3.3 backtracking recomputation: node of (start, size).
    g = np.random.default_rng(100 + seed)
    cp = np.concatenate([g.uniform(-2, 2, (4, 3)), g.uniform(0, 0.1, (4, 1))], axis=1)
    for depth in (1, 5, 13, 22):
        size = O.ROOT_SIZE >> depth
        start = int(g.integers(0, 1 << depth)) * size
        node = O.node_at(cp, start, size)
        u0, u1 = start / O.ROOT_SIZE, (start + size) / O.ROOT_SIZE
        np.testing.assert_allclose(_node_to_cp(node), G.subcurve(cp, u0, u1), atol=1e-13)


def test_split_half_is_restriction():
    g = np.random.default_rng(7)
    cp = np.concatenate([g.uniform(-2, 2, (4, 3)), g.uniform(0, 0.1, (4, 1))], axis=1)
    L, R = O.split_half(cp)
    u = np.linspace(0, 1, 33)
    np.testing.assert_allclose(G.curve_eval(L, u), G.curve_eval(cp, u / 2), atol=1e-14)
    np.testing.assert_allclose(G.curve_eval(R, u), G.curve_eval(cp, 0.5 + u / 2), atol=1e-14)


@pytest.mark.parametrize("seed", range(20))
def test_unit_ray_cylinder_matches_world_solve(seed):
    # App. A: unit ray along +z from the origin vs a textbook quadratic.
    g = np.random.default_rng(200 + seed)
    p = g.uniform(-1, 1, 3)
    a = g.standard_normal(3)
    r = g.uniform(0.05, 1.0)
    got = O.cylinder(p, a, r)
    ref = G.ray_infinite_cylinder(np.zeros(3), np.array([0, 0, 1.0]), p, a, r)
    if ref is None:
        assert got is None
    else:
        assert got is not None
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)


def test_unit_ray_cylinder_axis_parallel_to_ray():
    # App. A special case g = 0: distance is |p_xy|; outside, a miss.
    assert O.cylinder([0.1, 0.0, 3.0], [0, 0, 2.0], 0.2) == (-np.inf, np.inf)
    assert O.cylinder([0.3, 0.0, 3.0], [0, 0, 2.0], 0.2) is None


@pytest.mark.parametrize("seed", range(10))
def test_conservative_radius_bounds_the_fiber(seed):
    # Sec. 3.3: the bounding cylinder contains every point of the curve
    # dilated by its radius; equality for a straight constant-radius fiber.
    g = np.random.default_rng(300 + seed)
    cp = G.random_valid_cubic(g)
    node = O.node_at(cp, 0, O.ROOT_SIZE)
    rc = O.cons_radius(node)
    u = np.linspace(0, 1, 2001)
    c = G.curve_eval(cp, u)
    A, B = cp[0, :3], cp[3, :3]
    ax = (B - A) / np.linalg.norm(B - A)
    rel = c[:, :3] - A
    dist = np.linalg.norm(rel - np.outer(rel @ ax, ax), axis=1)
    assert np.all(dist + c[:, 3] <= rc + 1e-12)
    straight = np.stack([A + k / 3 * (B - A) for k in range(4)])
    cps = np.concatenate([straight, np.full((4, 1), 0.07)], axis=1)
    assert abs(O.cons_radius(O.node_at(cps, 0, O.ROOT_SIZE)) - 0.07) < 1e-14


@pytest.mark.parametrize("seed", range(10))
def test_slab_is_region_between_end_planes(seed):
    # Sec. 3.3: [t_min, t_max] = ray points between the start plane (normal
    # t0 through p) and the end plane (normal t1 through p + d), t >= 0.
    g = np.random.default_rng(400 + seed)
    node = g.standard_normal((4, 4))
    ok, lo, hi = O.slab(node, 50.0)
    ts = np.linspace(-1, 60, 20001)
    x = np.outer(ts, [0, 0, 1.0])
    p, d, t0, t1 = node[0, :3], node[1, :3], node[2, :3], node[3, :3]
    inside = ((x - p) @ t0 >= 0) & ((x - p - d) @ t1 <= 0) & (ts >= 0) & (ts <= 50.0)
    if not inside.any():
        assert not ok or hi - lo < 0.01
    else:
        assert ok
        assert abs(ts[inside].min() - lo) < 0.01 and abs(ts[inside].max() - hi) < 0.01


def test_slab_plane_parallel_to_ray():
    # a plane parallel to the ray constrains nothing unless the
    # ray is on its excluded side, which empties the interval.
    node = np.array([[0, 0, 1, 0], [0, 0, 2, 0], [1, 0, 0, 0], [0, 0, 1, 0]], float)
    node[0, 0] = -0.5  # start plane x = -0.5 with normal +x: origin kept
    ok, lo, hi = O.slab(node, 10.0)
    assert ok and lo == 0.0 and abs(hi - 3.0) < 1e-15
    node[0, 0] = 0.5   # start plane x = 0.5: origin excluded
    assert not O.slab(node, 10.0)[0]


def test_ray_frame_is_rigid():
    # Sec. 3.3 ray-centric frame: distances to the origin and along the ray
    # are preserved; the ray maps to +z.
    g = np.random.default_rng(9)
    cp = np.concatenate([g.uniform(-2, 2, (4, 3)), g.uniform(0, 0.1, (4, 1))], axis=1)
    o, w = g.uniform(-3, 3, 3), g.standard_normal(3)
    w /= np.linalg.norm(w)
    Q = O.to_ray_frame(G.ray7(o, w), cp)
    rel = cp[:, :3] - o
    np.testing.assert_allclose(np.linalg.norm(Q[:, :3], axis=1), np.linalg.norm(rel, axis=1), rtol=1e-14)
    np.testing.assert_allclose(Q[:, 2], rel @ w, atol=1e-14)
    np.testing.assert_allclose(Q[:, 3], cp[:, 3], atol=0)
    # pairwise distances preserved
    for i in range(4):
        for j in range(4):
            assert abs(np.linalg.norm(Q[i, :3] - Q[j, :3]) - np.linalg.norm(rel[i] - rel[j])) < 1e-13


@pytest.mark.parametrize("seed", range(30))
def test_lemma_validity_is_preserved_by_bisection(seed):
    # App. B.2, second lemma: halves of a valid cubic are valid, recursively.
    g = np.random.default_rng(500 + seed)
    cp = G.random_valid_cubic(g, jitter=0.6)
    assert O.valid_cubic(cp)
    stack = [cp]
    for _ in range(4):
        nxt = []
        for c in stack:
            L, R = O.split_half(c)
            assert O.valid_cubic(L) and O.valid_cubic(R)
            nxt += [L, R]
        stack = nxt


@pytest.mark.parametrize("seed", range(30))
def test_lemma_valid_halves_are_separated_by_split_plane(seed):
    # App. B.2, first lemma: the control points of the two halves lie on
    # opposite sides of the plane through s orthogonal to the split tangent.
    g = np.random.default_rng(600 + seed)
    cp = G.random_valid_cubic(g, jitter=0.6)
    L, R = O.split_half(cp)
    P = cp[:, :3]
    s = (P[0] + 3 * P[1] + 3 * P[2] + P[3]) / 8
    t = 0.75 * (-P[0] - P[1] + P[2] + P[3])
    assert np.all((L[:, :3] - s) @ t <= 1e-12)
    assert np.all((R[:, :3] - s) @ t >= -1e-12)


def test_presplit_pieces_tile_each_segment():
    # pieces are dyadic sub-curves covering [0, 1] in order.
    from paper_1811_03374_gb300 import inputs as I
    case = I.tiny_case()
    pc = O.presplit(case["cps"])
    for s in range(case["cps"].shape[0]):
        b, e = pc["begin"][s], pc["begin"][s + 1]
        assert e > b
        lo = 0.0
        for k in range(b, e):
            lv, off = pc["level"][k], pc["off"][k]
            u0, u1 = off / 2.0 ** lv, (off + 1) / 2.0 ** lv
            assert u0 == lo
            lo = u1
            np.testing.assert_allclose(pc["cp"][k], G.subcurve(case["cps"][s].astype(np.float64), u0, u1),
                                       atol=1e-12)
            if pc["flags"][k] == 0:
                assert O.valid_cubic(pc["cp"][k])
        assert lo == 1.0


def test_thick_check_flags_tight_bends_only():
    # Sec. 3.4 / Fig. 6: the same curve passes with a thin radius and fails
    # once the radius exceeds what the end planes allow.
    cp = _load("fig_cubic_split.txt")[:4].copy()
    cp[:, 3] = 0.1
    assert O.thick_ok(cp)
    # at u = 0 the end plane lies <p3 - p0, t1^> = 27 / |(3, -3.5)| = 5.86 away
    # while the cross-section reaches r * sin(angle(t0, t1)) = 0.988 r towards
    # it, so a radius of 6.5 crosses the end plane
    cp[:, 3] = 6.5
    assert not O.thick_ok(cp)
