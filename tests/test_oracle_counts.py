"""Pins of the oracle's pruning-test statistic (Fig. 8): the
cylinder counts are the traversal's node tests, the box search finds the same
hits, hand-counted box cases, and the figure's claim that box tests grow
exponentially with the depth while cylinder tests grow by about one per level
(CPU only)."""
import numpy as np
import pytest

import oracle as O
from paper_1811_03374_gb300 import inputs as I
from tests import _geom as G


def _one(ray7, cp):
    """A case of one ray and one curve."""
    r = ray7
    rays = I.pack_rays(r[None, :3], r[None, 3:6] / np.linalg.norm(r[3:6]))
    return dict(cps=np.asarray(cp, np.float32)[None], rays=rays, row_ptr=np.array([0, 1], np.int32),
                seg_idx=np.array([0], np.int32))


@pytest.mark.parametrize("depth", [0, 3, 8, 15])
def test_cylinder_counts_are_traversal_node_tests(depth):
    case = I.sweep_case("moderate", 300, forced_hits=True)
    counts, t = O.ray_counts(case, depth, "cylinder")
    pieces = O.presplit(case["cps"])
    for i in range(300):
        if np.diff(pieces["begin"])[i] != 1:
            continue  # pre-split: several pieces, each with its own count
        h = O.intersect(O.ray7_from_packed(case["rays"][i]), pieces["cp"][pieces["begin"][i]], depth)
        assert counts[i] == h.nodes
        assert (h.hit and abs(t[i] - h.t) <= 1e-12 * h.t) or (not h.hit and np.isinf(t[i]))


@pytest.mark.parametrize("klass", list(I.SWEEP_JITTER))
def test_box_search_finds_the_same_hits(klass):
    # both searches end in the same leaf test; they agree wherever every leaf
    # cylinder the ray meets lies inside the bounding volumes of its
    # ancestors in both hierarchies.  A leaf's conservative cylinder can reach
    # out of a box (and of its parent's cylinder): at depth 2 a few rays in a
    # hundred differ, deeper at most one in a thousand
    case = I.single_fiber_case(klass, 3000)
    for depth, frac in ((2, 0.95), (4, 0.995), (7, 0.999), (12, 0.999)):
        _, tc = O.ray_counts(case, depth, "cylinder")
        _, tb = O.ray_counts(case, depth, "box")
        same = np.isclose(tb, tc, rtol=1e-12, atol=0) | (np.isinf(tb) & np.isinf(tc))
        assert same.mean() >= frac, (depth, same.mean())


def test_box_counts_by_hand():
    # a straight fiber along x from -1 to 1, radius 0.1; rays straight down
    cp = np.array([[-1.0, 0, 0, 0.1], [-1 / 3, 0, 0, 0.1], [1 / 3, 0, 0, 0.1], [1.0, 0, 0, 0.1]])
    down = np.array([0.0, 0, -1.0])
    at = lambda x: _one(G.ray7(np.array([x, 0.0, 3.0]), down), cp)
    # depth 0: the root is the leaf -- one box test
    assert O.ray_counts(at(0.5), 0, "box")[0][0] == 1
    # depth 1, ray at x = 0.5: root box, both children tested, only the right
    # one holds x = 0.5 (the left box ends at 0.1)
    assert O.ray_counts(at(0.5), 1, "box")[0][0] == 3
    # ray at x = 0: both children hit; the second is tested again when taken up
    assert O.ray_counts(at(0.0), 1, "box")[0][0] == 4
    # a ray passing beside the root box: one test
    assert O.ray_counts(at(1.5), 5, "box")[0][0] == 1


def test_fig8_boxes_grow_exponentially_cylinders_linearly():
    case = I.single_fiber_case("moderate", 2000)
    cyl, box = [], []
    depths = [10, 13, 16, 19]
    for d in depths:
        cyl.append(O.ray_counts(case, d, "cylinder")[0].mean())
        box.append(O.ray_counts(case, d, "box")[0].mean())
    for k in range(1, len(depths)):
        assert box[k] >= 2.0 * box[k - 1], box          # at least x2 per 3 levels
        assert cyl[k] - cyl[k - 1] <= 3.0 * 1.5, cyl     # about one per level
    assert box[-1] > 20 * cyl[-1]


@pytest.mark.parametrize("depth", [3, 9, 16])
def test_cylinder_counts_on_presplit_segments(depth):
    # a pre-split segment's count is the sum of its pieces' node tests, each
    # piece traversed to depth - level with the closest hit so far as t_max
    # (its leaves are the unsplit curve's)
    case = I.sweep_case("curved", 300, forced_hits=True)
    pieces = O.presplit(case["cps"])
    counts, t = O.ray_counts(case, depth, "cylinder", pieces)
    n_split = 0
    for i in range(300):
        b, e = pieces["begin"][i], pieces["begin"][i + 1]
        r7 = O.ray7_from_packed(case["rays"][i])
        best, n = r7[6], 0
        for k in range(b, e):
            r7k = r7.copy()
            r7k[6] = best
            h = O.intersect(r7k, pieces["cp"][k], max(depth - int(pieces["level"][k]), 0))
            n += h.nodes
            if h.hit and h.t < best:
                best = h.t
        assert counts[i] == n
        assert (np.isfinite(best) and abs(t[i] - best) <= 1e-12 * best) or (np.isinf(best) and np.isinf(t[i]))
        n_split += e - b > 1
    assert n_split > 30


@pytest.mark.parametrize("mode", ["cylinder", "box"])
def test_counts_with_double_rays_equal_float_rays(mode):
    # the double-precision ray entry (used to shift rays by less than an FP32
    # step) gives the float entry's counts on the same rays
    case = I.tiny_case(n_ray=512)
    pieces = O.presplit(case["cps"])
    c_f, t_f = O.ray_counts(case, 8, mode, pieces)
    r7 = np.stack([O.ray7_from_packed(r) for r in case["rays"]])
    c_d, t_d = O.ray_counts_d(r7, case["row_ptr"], case["seg_idx"], 8, mode, pieces)
    np.testing.assert_array_equal(c_d, c_f)
    np.testing.assert_array_equal(t_d, t_f)
    assert c_f.sum() > 512


def _band_delta(case):
    """Per ray: 1e-4 of the largest radius plus 22 * 2^-24 of the largest
    control-point distance over the ray's candidates (the FP32 band)."""
    rp = case["row_ptr"].astype(np.int64)
    d = np.zeros(len(rp) - 1)
    for i in range(len(d)):
        c = case["seg_idx"][rp[i]:rp[i + 1]]
        cp = case["cps"][c].astype(np.float64)
        T = np.linalg.norm(cp[:, :, :3] - case["rays"][i, :3].astype(np.float64), axis=2).max()
        d[i] = 1e-4 * cp[:, :, 3].max() + 22 * 2.0 ** -24 * T
    return d


@pytest.mark.parametrize("klass", ["straight", "curved"])
@pytest.mark.parametrize("mode", ["cylinder", "box"])
def test_band_flag_covers_every_count_a_small_shift_changes(klass, mode):
    # the flag of orc_ray_counts_amb marks rays with a decision within delta
    # of flipping; its definition fixes that any ray whose count changes when
    # the ray moves sideways by less than delta is flagged.  Checked with
    # random shifts of up to delta / 4; delta = 0 flags nothing and the
    # counts are those of the plain search
    case = I.single_fiber_case(klass, 2048)
    pieces = O.presplit(case["cps"])
    dl = _band_delta(case)
    g = np.random.default_rng(11)
    r7 = np.stack([O.ray7_from_packed(r) for r in case["rays"]])
    w = r7[:, 3:6] / np.linalg.norm(r7[:, 3:6], axis=1, keepdims=True)
    a = np.where(np.abs(w[:, :1]) < 0.9, [[1.0, 0, 0]], [[0.0, 1, 0]])
    e1 = a - np.sum(a * w, axis=1, keepdims=True) * w
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(w, e1)
    changed_total = 0
    for depth in (8, 16):
        c0, _ = O.ray_counts(case, depth, mode, pieces)
        ca, amb = O.ray_counts_amb(case, depth, mode, dl, pieces)
        np.testing.assert_array_equal(ca, c0)
        cz, amb0 = O.ray_counts_amb(case, depth, mode, np.zeros(len(dl)), pieces)
        assert not amb0.any()
        for _ in range(4):
            ang = g.uniform(0, 2 * np.pi, len(dl))
            m = g.uniform(0, 0.25, len(dl)) * dl
            rs = r7.copy()
            rs[:, :3] += (np.cos(ang)[:, None] * e1 + np.sin(ang)[:, None] * e2) * m[:, None]
            cs, _ = O.ray_counts_d(rs, case["row_ptr"], case["seg_idx"], depth, mode, pieces)
            ch = cs != c0
            assert not (ch & ~amb).any(), (depth, np.nonzero(ch & ~amb)[0][:5])
            changed_total += int(ch.sum())
        assert amb.mean() < 0.06, amb.mean()  # the flag stays selective
    assert changed_total > 0  # the check is not vacuous
