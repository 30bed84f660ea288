"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by
element on seeded inputs: the tiny workload at depth 8, the depth sweep at
every depth 2..22 on three curvature classes, the hair patch at full size
(every ray, in the bench's launch), per-pair hits pair by pair for every
kernel, the FP64 polish, counters and edge cases.  With FX_REPORT=<path>
set, every comparison appends its strict / band / silhouette counts."""
import numpy as np
import pytest

import oracle as O
from paper_1811_03374_gb300 import fiberx as F
from paper_1811_03374_gb300 import inputs as I
from tests import _parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _np(x):
    return x.cpu().numpy()


def _run_closest(case, depth, flags=0, fib=None, variant=F.FX_VARIANT_AUTO):
    own = fib is None
    if own:
        fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    tu, seg, leaf = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth, flags)
    torch.cuda.synchronize()
    st = fib.status()
    if own:
        fib.close()
    return _np(tu), _np(seg), _np(leaf), st


def _assert_parity(stats, max_band_frac=1e-3, where="", **rec):
    """Every result passes strict, band or silhouette; the band and
    silhouette passes stay within max_band_frac of the results.  The counts
    are reported (FX_REPORT) under the test's name and `rec`."""
    P.report(dict(test=where, **rec, **P.counts_of(stats)))
    assert len(stats["fail"]) == 0, "%s: %d results failing parity, e.g. %s" % (
        where, len(stats["fail"]), stats["detail"])
    exempt = stats["band"] + stats["silhouette"]
    assert exempt <= max_band_frac * max(stats["n"], 1), (where, stats["band"], stats["silhouette"], stats["n"])
    assert stats["max_rel_t"] <= P.TOL_T and stats["max_du_over_tol"] <= 1.0, where


@pytest.fixture(scope="module")
def tiny():
    case = I.tiny_case()
    pieces = O.presplit(case["cps"])
    ref = O.closest(case, 8, pieces)
    return case, pieces, ref


VARIANTS = [F.FX_VARIANT_LANE, F.FX_VARIANT_WARP]
MATH = [0, F.FX_FAST_MATH]
MATH_IDS = ["ieee", "fast"]
# (kernel flag, variant) of every forward path; the scan variant runs the
# lane kernel on handles with pre-split segments
PATHS = [(F.FX_KERNEL_PERSISTENT, F.FX_VARIANT_LANE), (F.FX_KERNEL_PERSISTENT, F.FX_VARIANT_SCAN),
         (F.FX_KERNEL_PERSISTENT, F.FX_VARIANT_RAY), (F.FX_KERNEL_PERSISTENT, F.FX_VARIANT_WARP),
         (F.FX_KERNEL_NAIVE, F.FX_VARIANT_AUTO)]
PATH_IDS = ["lane", "scan", "ray", "warp", "naive"]


@pytest.mark.parametrize("variant", VARIANTS, ids=["lane", "warp"])
@pytest.mark.parametrize("flags", MATH, ids=MATH_IDS)
def test_tiny_closest_persistent(tiny, flags, variant):
    case, pieces, ref = tiny
    tu, seg, leaf, st = _run_closest(case, 8, flags, variant=variant)
    assert st & ~F.FX_DEV_UNSUPPORTED == 0
    stats = P.compare_closest(case, 8, tu, seg, ref, pieces, leaf)
    _assert_parity(stats, where="tiny_closest", variant=int(variant), flags=int(flags))
    assert stats["hits"] > 3000
    strict = P.strict_ok(tu[:, 0], tu[:, 1], seg, ref["t"], ref["u"], ref["seg"])
    same = strict & (seg >= 0)
    assert np.mean(leaf[same] == ref["leaf"][same]) > 0.999


def test_tiny_closest_naive(tiny):
    case, pieces, ref = tiny
    tu, seg, leaf, st = _run_closest(case, 8, F.FX_KERNEL_NAIVE)
    assert st & ~F.FX_DEV_UNSUPPORTED == 0
    _assert_parity(P.compare_closest(case, 8, tu, seg, ref, pieces, leaf), where="tiny_closest_naive")


def _run_pairs(case, depth, kernel, variant, flags, fib=None):
    own = fib is None
    if own:
        fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    tu, leaf = F.intersect_pairs(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth, kernel | flags)
    torch.cuda.synchronize()
    st = fib.status()
    if own:
        fib.close()
    return _np(tu), _np(leaf), st


@pytest.mark.parametrize("kernel,variant", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("flags", MATH, ids=MATH_IDS)
def test_tiny_pairs(tiny, kernel, variant, flags):
    # every (ray, candidate) pair of the tiny workload against the oracle's
    # per-pair result, pair by pair (the paper's one-ray / one-curve routine)
    case, pieces, _ = tiny
    pr = O.pairs(case, 8, pieces)
    tu, leaf, st = _run_pairs(case, 8, kernel, variant, flags)
    assert st & ~F.FX_DEV_UNSUPPORTED == 0
    stats = P.compare_pairs(case, 8, tu, leaf, pr, pieces)
    _assert_parity(stats, max_band_frac=1e-4, where="tiny_pairs", kernel=int(kernel), variant=int(variant),
                   flags=int(flags))
    assert stats["hits"] > 10000


@pytest.mark.parametrize("kernel,variant", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("flags", MATH, ids=MATH_IDS)
@pytest.mark.parametrize("forced", [False, True], ids=["aabb", "forced"])
@pytest.mark.parametrize("klass", list(I.SWEEP_JITTER))
def test_sweep_pairs(klass, forced, flags, kernel, variant):
    # the depth-sweep classes pair by pair, with longer rows: each ray's own
    # segment among seven random others
    case = I.sweep_case(klass, 4096, forced_hits=forced)
    g = np.random.default_rng(17)
    n = len(case["rays"])
    rows = [np.concatenate([[i], g.integers(0, n, 7)]).astype(np.int32) for i in range(n)]
    case = dict(case, seg_idx=np.concatenate(rows),
                row_ptr=np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32))
    pieces = O.presplit(case["cps"])
    fib = F.Fibers(case["cps"])
    for depth in (2, 9, 15, 22):
        pr = O.pairs(case, depth, pieces)
        tu, leaf, st = _run_pairs(case, depth, kernel, variant, flags, fib)
        assert st & ~F.FX_DEV_UNSUPPORTED == 0
        stats = P.compare_pairs(case, depth, tu, leaf, pr, pieces)
        _assert_parity(stats, where="sweep_pairs", klass=klass, forced=forced, depth=depth, kernel=int(kernel),
                       variant=int(variant), flags=int(flags))
    fib.close()


def test_presplit_counts_match_oracle(tiny):
    case, pieces, _ = tiny
    fib = F.Fibers(case["cps"])
    info = fib.info()
    fib.close()
    counts = np.diff(pieces["begin"])
    assert info["n_seg"] == 16
    assert info["n_piece"] == len(pieces["seg"])
    assert info["n_presplit"] == int((counts > 1).sum())
    assert info["n_unsupported"] == int(pieces["flags"].sum())
    assert info["max_level"] == int(pieces["level"].max())


DEPTHS = list(range(2, 23))


@pytest.mark.parametrize("variant", [F.FX_VARIANT_AUTO, F.FX_VARIANT_SCAN], ids=["auto", "scan"])
@pytest.mark.parametrize("klass", list(I.SWEEP_JITTER))
@pytest.mark.parametrize("forced", [False, True], ids=["aabb", "forced"])
@pytest.mark.parametrize("flags", MATH, ids=MATH_IDS)
def test_depth_sweep(klass, forced, flags, variant):
    # every depth 2..22 on the three curvature classes (the library's own
    # choice of kernel, and the scan variant, which runs the lane kernel on
    # the pre-split curved class)
    case = I.sweep_case(klass, 4096, forced_hits=forced)
    pieces = O.presplit(case["cps"])
    fib = F.Fibers(case["cps"])
    exempt = 0
    for depth in DEPTHS:
        ref = O.closest(case, depth, pieces)
        tu, seg, leaf, _ = _run_closest(case, depth, flags, fib, variant=variant)
        stats = P.compare_closest(case, depth, tu, seg, ref, pieces, leaf)
        # per depth at most 8 of the 4096 rays pass by band or silhouette
        _assert_parity(stats, max_band_frac=2e-3, where="depth_sweep", klass=klass, forced=forced, depth=depth,
                       math="fast" if flags else "ieee", variant=int(variant))
        exempt += stats["band"] + stats["silhouette"]
        if forced:
            assert stats["hits"] > 3500
    # over all 21 depths at most 0.2 % (measured: at most 0.14 % for one class
    # and math mode, 0.018 % over all of them)
    assert exempt <= 2e-3 * len(DEPTHS) * 4096, exempt
    assert fib.status() == 0
    fib.close()


@pytest.mark.parametrize("klass", list(I.SWEEP_JITTER))
def test_single_fiber_many_rays(klass):
    # the shape of the paper's own benchmark: one fiber, many rays
    case = I.single_fiber_case(klass, 8192)
    pieces = O.presplit(case["cps"])
    fib = F.Fibers(case["cps"])
    for depth in (2, 8, 15, 22):
        ref = O.closest(case, depth, pieces)
        tu, seg, leaf, _ = _run_closest(case, depth, F.FX_FAST_MATH, fib)
        stats = P.compare_closest(case, depth, tu, seg, ref, pieces, leaf)
        _assert_parity(stats, where="single_fiber", klass=klass, depth=depth)
    assert fib.status() & ~F.FX_DEV_UNSUPPORTED == 0
    fib.close()


def _filter_vs_lane(case, depth, flags):
    fib = F.Fibers(case["cps"])
    assert fib.info()["n_piece"] == case["cps"].shape[0]  # single level-0 pieces: the filter applies
    out = {}
    for v in (F.FX_VARIANT_LANE, F.FX_VARIANT_FILTER):
        fib.set_launch(variant=v)
        fib.counters(reset=True)
        tu, seg, leaf = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth,
                                            flags | F.FX_COUNT)
        torch.cuda.synchronize()
        out[v] = (_np(tu), _np(seg), _np(leaf), fib.counters(reset=True), fib.status())
    fib.close()
    (tl, sl, ll, cl, stl), (tf, sf, lf, cf, stf) = out[F.FX_VARIANT_LANE], out[F.FX_VARIANT_FILTER]
    assert stl == 0 and stf == 0
    np.testing.assert_array_equal(sf, sl)
    np.testing.assert_array_equal(lf, ll)
    np.testing.assert_array_equal(tf, tl)
    # the same traversals; the lane kernel rejects some candidates by their
    # bound without a root node test, the filter tests every root
    for k in ("tests", "descents", "backtracks", "hits"):
        assert cf[k] == cl[k], (k, cf, cl)
    assert cl["nodes"] <= cf["nodes"]
    return sl


@pytest.mark.parametrize("klass", ["straight", "moderate"])
@pytest.mark.parametrize("forced", [False, True], ids=["aabb", "forced"])
@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
def test_filter_path_equals_lane_kernel(klass, forced, flags):
    # both paths skip only candidates whose root test cannot pass and traverse
    # the rest the same way: same hits, same traversal counters
    case = I.sweep_case(klass, 4096, forced_hits=forced)
    for depth in (0, 4, 10, 16, 22):
        _filter_vs_lane(case, depth, flags)


@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
def test_filter_path_equals_lane_kernel_on_hair(hair, flags):
    case = hair[0]
    seg = _filter_vs_lane(case, 15, flags)
    assert (seg >= 0).sum() > 100_000


def _variant_vs_lane(case, depth, flags, pairs=False, variant=F.FX_VARIANT_SCAN, presplit=False):
    """A variant against the lane kernel on one launch each: identical
    outputs, the same candidates examined and the same traversals (the scan
    variant drops candidates whose root cylinder misses before any node
    step, so it counts fewer node tests)."""
    fib = F.Fibers(case["cps"])
    # single level-0 pieces, or (presplit) a handle with pre-split segments
    assert (fib.info()["n_piece"] == case["cps"].shape[0]) != presplit
    out = {}
    for v in (F.FX_VARIANT_LANE, variant):
        fib.set_launch(variant=v)
        fib.counters(reset=True)
        if pairs:
            res = F.intersect_pairs(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth,
                                    flags | F.FX_COUNT)
        else:
            res = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth,
                                      flags | F.FX_COUNT)
        torch.cuda.synchronize()
        out[v] = ([_np(x) for x in res], fib.counters(reset=True), fib.status())
    fib.close()
    (rl, cl, stl), (rs, cs, sts) = out[F.FX_VARIANT_LANE], out[variant]
    assert stl & ~F.FX_DEV_UNSUPPORTED == 0 and sts == stl
    for a, b in zip(rl, rs):
        np.testing.assert_array_equal(b, a)
    for k in ("tests", "descents", "backtracks", "hits"):
        assert cs[k] == cl[k], (k, cs, cl)
    assert cs["nodes"] <= cl["nodes"]
    return rs


VARIANTS_EXACT = [F.FX_VARIANT_SCAN, F.FX_VARIANT_RAY]


@pytest.mark.parametrize("variant", VARIANTS_EXACT, ids=["scan", "ray"])
@pytest.mark.parametrize("klass", ["straight", "moderate"])  # the curved class is pre-split
@pytest.mark.parametrize("forced", [False, True], ids=["aabb", "forced"])
@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
@pytest.mark.parametrize("pairs", [False, True], ids=["closest", "pairs"])
def test_variant_equals_lane_kernel(klass, forced, flags, pairs, variant):
    case = I.sweep_case(klass, 4096, forced_hits=forced)
    # one ray listing many segments: rows longer than a 32-candidate window,
    # with a ragged last window
    g = np.random.default_rng(3)
    rows = [case["seg_idx"][case["row_ptr"][i]:case["row_ptr"][i + 1]] for i in range(len(case["rays"]))]
    for i in range(0, len(rows), 97):
        rows[i] = np.concatenate([rows[i], g.integers(0, case["cps"].shape[0], 1 + i % 150)]).astype(np.int32)
    case = dict(case, seg_idx=np.concatenate(rows).astype(np.int32),
                row_ptr=np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32))
    for depth in (0, 4, 10, 16, 22):
        _variant_vs_lane(case, depth, flags, pairs, variant)


@pytest.mark.parametrize("variant", VARIANTS_EXACT, ids=["scan", "ray"])
@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
@pytest.mark.parametrize("pairs", [False, True], ids=["closest", "pairs"])
def test_variant_equals_lane_kernel_on_hair(hair, flags, pairs, variant):
    case = hair[0]
    depth = 15
    if pairs:  # a seeded block of 20,000 rays with candidates
        counts = np.diff(case["row_ptr"])
        idx = np.nonzero(counts > 0)[0][::6][:20000]
        case = I.subsample_rays(case, idx)
    res = _variant_vs_lane(case, depth, flags, pairs, variant)
    if not pairs:
        assert (res[1] >= 0).sum() > 100_000


@pytest.mark.parametrize("variant", VARIANTS_EXACT, ids=["scan", "ray"])
@pytest.mark.parametrize("klass", ["straight", "moderate"])
def test_variant_equals_lane_kernel_on_single_fiber(klass, variant):
    case = I.single_fiber_case(klass, 1 << 16)
    for depth in (2, 15, 22):
        for pairs in (False, True):
            _variant_vs_lane(case, depth, F.FX_FAST_MATH, pairs, variant)


@pytest.mark.parametrize("klass", ["curved", "tiny"])
@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
@pytest.mark.parametrize("pairs", [False, True], ids=["closest", "pairs"])
def test_ray_variant_equals_lane_kernel_on_presplit_handles(klass, flags, pairs):
    # handles with pre-split segments: the per-ray variant walks each
    # candidate's pieces as the lane kernel does, with its two passes for
    # closest hits (one candidate per ray, forced hits; and 16 per ray)
    case = I.sweep_case("curved", 4096, forced_hits=True) if klass == "curved" else I.tiny_case()
    for depth in (0, 4, 8, 16, 22):
        _variant_vs_lane(case, depth, flags, pairs, F.FX_VARIANT_RAY, presplit=True)


def test_scan_variant_falls_back_on_presplit_handles(tiny):
    # the tiny fibers are pre-split: the scan variant runs the lane kernel
    variant = F.FX_VARIANT_SCAN
    case, pieces, ref = tiny
    res = {}
    for v in (F.FX_VARIANT_LANE, variant):
        res[v] = _run_closest(case, 8, 0, variant=v)
    for a, b in zip(res[F.FX_VARIANT_LANE], res[variant]):
        np.testing.assert_array_equal(np.asarray(b), np.asarray(a))


@pytest.mark.parametrize("variant", VARIANTS, ids=["lane", "warp"])
def test_counters_match_oracle(tiny, variant):
    # per-pair mode visits exactly the oracle's nodes (same decisions); the
    # closest-hit mode prunes with the running best and visits no more
    case, pieces, ref = tiny
    pr = O.pairs(case, 8, pieces)
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    fib.counters(reset=True)
    F.intersect_pairs(fib, case["rays"], case["row_ptr"], case["seg_idx"], 8, F.FX_COUNT)
    c = fib.counters(reset=True)
    F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], 8, F.FX_COUNT)
    cc = fib.counters(reset=True)
    fib.close()
    oc = pr["counters"]
    assert c["tests"] == oc["tests"]
    for k in ("nodes", "descents", "backtracks", "hits"):
        assert abs(c[k] - oc[k]) <= 1e-3 * oc[k] + 2, (k, c[k], oc[k])
    assert cc["nodes"] <= c["nodes"] and cc["tests"] <= c["tests"]


def test_polish_fp64_matches_oracle_leaf():
    case = I.sweep_case("moderate", 4096, forced_hits=True)
    pieces = O.presplit(case["cps"])
    fib = F.Fibers(case["cps"])
    for depth in (4, 12, 20):
        tu, seg, leaf, _ = _run_closest(case, depth, F.FX_POLISH_FP64, fib)
        ok = seg >= 0
        ref_t = np.full(len(seg), np.nan)
        for i in np.nonzero(ok)[0][:400]:
            r7 = O.ray7_from_packed(case["rays"][i])
            lh = O.leaf_hit(r7, case["cps"][seg[i]].astype(np.float64), depth, leaf[i] >> (23 - depth))
            if lh is not None:
                ref_t[i] = lh[0]
        m = np.isfinite(ref_t)
        assert m.sum() > 300
        rel = np.abs(tu[m, 0] - ref_t[m]) / ref_t[m]
        assert rel.max() < 2e-7  # FP64 value rounded once to FP32
    fib.close()


def test_host_entry_matches_device(tiny):
    case, _, _ = tiny
    fib = F.Fibers(case["cps"])
    tu_d, seg_d, leaf_d = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], 8)
    tu_h, seg_h, leaf_h = F.intersect_closest_host(fib, case["rays"], case["row_ptr"], case["seg_idx"], 8)
    np.testing.assert_array_equal(_np(tu_d), tu_h.numpy())
    np.testing.assert_array_equal(_np(seg_d), seg_h.numpy())
    np.testing.assert_array_equal(_np(leaf_d), leaf_h.numpy())
    fib.close()


def _chunked_case():
    """About 90 MB of host input, so the host entry cuts it into chunks:
    1M rays over 65,536 segments, each ray's own segment among 15 random
    others, every seventh row empty, rows 100,000-299,999 and 900,001-end
    empty (whole blocks of rays are then not copied), and one row of 300,000
    candidates."""
    base = I.sweep_case("moderate", 65536, forced_hits=True)
    g = np.random.default_rng(41)
    n_ray = 1 << 20
    rays = np.tile(base["rays"], (16, 1))
    own = np.tile(np.arange(65536, dtype=np.int32), 16)
    lens = np.full(n_ray, 16, np.int64)
    lens[::7] = 0
    lens[100_000:300_000] = 0
    lens[900_001:] = 0
    lens[500_001] = 300_000
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    seg_idx = g.integers(0, 65536, int(row_ptr[-1])).astype(np.int32)
    first = row_ptr[:-1][lens > 0]
    seg_idx[first + g.integers(0, 16, len(first))] = own[lens > 0]
    return dict(cps=base["cps"], rays=rays, row_ptr=row_ptr, seg_idx=seg_idx)


@pytest.mark.parametrize("variant,flags", [(F.FX_VARIANT_LANE, 0), (F.FX_VARIANT_SCAN, F.FX_FAST_MATH),
                                           (F.FX_VARIANT_LANE, F.FX_POLISH_FP64),
                                           (F.FX_VARIANT_LANE, F.FX_KERNEL_NAIVE)],
                         ids=["lane", "scan-fast", "lane-polish", "naive"])
def test_host_entry_pipeline_matches_device(variant, flags):
    # the chunked copy / compute pipeline of the host entry gives the device
    # entry's results bit for bit, with the rays copied (pageable memory) or
    # read in place by the kernels (pinned memory)
    case = _chunked_case()
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    tu_d, seg_d, leaf_d = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], 12, flags)
    torch.cuda.synchronize()
    h = tuple(torch.from_numpy(np.asarray(x)).pin_memory() for x in (case["rays"], case["row_ptr"], case["seg_idx"]))
    n = len(case["rays"])
    pinned_out = (torch.empty((n, 2)).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory(),
                  torch.empty(n, dtype=torch.int32).pin_memory())
    # pinned inputs (the kernels read the rays in place); pageable outputs,
    # then pinned ones; the second call of each reuses the staging and the
    # streams
    for out in (None, None, pinned_out, pinned_out):
        if out is not None:
            for t in out:
                t.fill_(-7)  # every element must be written by the call
        tu_h, seg_h, leaf_h = F.intersect_closest_host(fib, *h, 12, flags, out=out)
        np.testing.assert_array_equal(_np(tu_d), tu_h.numpy())
        np.testing.assert_array_equal(_np(seg_d), seg_h.numpy())
        np.testing.assert_array_equal(_np(leaf_d), leaf_h.numpy())
        h2d, d2h = F.host_bytes(fib)
        n_ray, n_pair = len(case["rays"]), len(case["seg_idx"])
        assert d2h == 16 * n_ray
        # the two empty ranges hold at least 36 whole blocks of 8192 rays at any
        # block alignment: their rays stay behind
        assert 4 * (n_ray + 1) + 4 * n_pair < h2d <= 32 * n_ray + 4 * (n_ray + 4) + 4 * n_pair - 36 * 8192 * 32
    assert (seg_h.numpy() >= 0).sum() > 400_000
    assert fib.status() & ~F.FX_DEV_UNSUPPORTED == 0
    fib.close()


@pytest.mark.parametrize("variant", [F.FX_VARIANT_LANE, F.FX_VARIANT_SCAN, F.FX_VARIANT_RAY],
                         ids=["lane", "scan", "ray"])
def test_edge_cases(variant):
    case = I.sweep_case("moderate", 64, forced_hits=True)
    fib = F.Fibers(case["cps"])
    assert fib.info()["n_piece"] == 64
    fib.set_launch(variant=variant)
    # no rays
    tu, seg, _ = F.intersect_closest(fib, np.zeros((0, 8), np.float32), np.zeros(1, np.int32),
                                     np.zeros(0, np.int32), 8)
    assert tu.shape == (0, 2)
    # rays without candidates, and a ray listing every segment
    rp = np.array([0, 0, 0, 64, 64], dtype=np.int32)
    rays = case["rays"][:4].copy()
    si = np.arange(64, dtype=np.int32)
    tu, seg, _ = F.intersect_closest(fib, rays, rp, si, 8)
    seg = _np(seg)
    assert seg[0] == -1 and seg[1] == -1 and seg[3] == -1
    sub = dict(cps=case["cps"], rays=rays, row_ptr=rp, seg_idx=si)
    ref = O.closest(sub, 8)
    assert seg[2] == ref["seg"][2]
    # finite t_max removes hits beyond it
    tu0, seg0, _ = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], 8)
    r2 = case["rays"].copy()
    r2[:, 3] = 0.5 * _np(tu0)[:, 0].clip(0, 100)
    tu1, seg1, _ = F.intersect_closest(fib, r2, case["row_ptr"], case["seg_idx"], 8)
    assert np.all(_np(seg1) == -1)
    # depth 0 (single cylinder) and 23 (finest)
    for d in (0, 23):
        ref = O.closest(case, d)
        tu, seg, _, _ = _run_closest(case, d, 0, fib, variant=variant)
        stats = P.compare_closest(case, d, tu, seg, ref, O.presplit(case["cps"]))
        _assert_parity(stats, max_band_frac=0.05, where="edge_depth", depth=d, variant=int(variant))
    # bad depth and bad sizes are refused before launch
    with pytest.raises(F.FiberxError):
        F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], 24)
    with pytest.raises(F.FiberxError):
        F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], -1)
    # out-of-range segment ids are skipped and flagged when checking is on
    bad = case["seg_idx"].copy()
    bad[5] = 10_000
    tu, seg, _ = F.intersect_closest(fib, case["rays"], case["row_ptr"], bad, 8, F.FX_CHECK_INDEX)
    assert _np(seg)[5] == -1
    assert fib.status() & F.FX_DEV_BAD_INDEX
    assert fib.status() == 0  # cleared by the read
    fib.close()


def _unsupported_at(pieces, seg, leaf):
    """Whether the piece of segment `seg` holding `leaf` (units of 2^-23)
    is flagged unsupported by the pre-split."""
    for k in range(pieces["begin"][seg], pieces["begin"][seg + 1]):
        sh = 23 - int(pieces["level"][k])
        if int(pieces["off"][k]) << sh <= leaf < (int(pieces["off"][k]) + 1) << sh:
            return bool(pieces["flags"][k] & 1)
    return False


def test_thick_fibers_presplit_and_parity():
    # bent fibers up to 0.8 of their length thick: the upload's exact
    # end-plane check (Sec. 3.4, Fig. 7) pre-splits exactly the pieces the
    # oracle's does, and their intersections agree with the oracle's.  Where
    # the radius exceeds the radius of curvature no pre-split separates the
    # end planes (the piece stays flagged unsupported) and the leaf slabs
    # overlap: dozens of adjacent leaves enter within a few 1e-7 of the same
    # t, the traversal's front-to-back order no longer finds the nearest of
    # them (the oracle's own pick is not always its smallest t), and whether
    # a leaf at the edge of the overlap is entered at all is decided by
    # rounding.  There the entry t is still determined, u is not: a ray that
    # fails the strict rule in such a piece must agree in hit, segment and t,
    # and its u must lie in the leaf it reports.
    g = np.random.default_rng(31)
    n = 2048
    A = g.uniform(-5, 5, (n, 3))
    B = A + I._unit_sphere(g, n)
    pts = np.stack([A + k / 3 * (B - A) for k in range(4)], axis=1)
    pts[:, 1:3] += 0.35 * g.uniform(-1, 1, (n, 2, 3))
    r = np.repeat(g.uniform(0.0, 0.8, (n, 1, 1)), 4, axis=1)
    cps = np.concatenate([pts, r], axis=2).astype(np.float32)
    pieces = O.presplit(cps)
    fib = F.Fibers(cps)
    info = fib.info()
    counts = np.diff(pieces["begin"])
    assert info["n_piece"] == len(pieces["seg"]) and info["n_presplit"] == int((counts > 1).sum())
    assert info["n_unsupported"] == int(pieces["flags"].sum())
    assert 0.1 * n < info["n_presplit"] < 0.9 * n  # both outcomes are exercised
    c64 = cps.astype(np.float64)
    u = g.uniform(0, 1, n)[:, None]
    v = 1 - u
    c = v ** 3 * c64[:, 0] + 3 * u * v * v * c64[:, 1] + 3 * u * u * v * c64[:, 2] + u ** 3 * c64[:, 3]
    target = c[:, :3] + 0.9 * c[:, 3:4] * I._unit_ball(g, n)
    w = I._unit_sphere(g, n)
    rp, si = I.diagonal_csr(n)
    case = dict(cps=cps, rays=I.pack_rays(target - 10.0 * w, w), row_ptr=rp, seg_idx=si)
    for depth in (6, 14):
        ref = O.closest(case, depth, pieces)
        tu, seg, leaf, st = _run_closest(case, depth, 0, fib)
        stats = P.compare_closest(case, depth, tu, seg, ref, pieces, leaf)
        overlap = []
        for i in stats["fail"]:
            s = int(seg[i])
            if s < 0 or s != ref["seg"][i] or not (_unsupported_at(pieces, s, int(leaf[i]))
                                                   or _unsupported_at(pieces, s, int(ref["leaf"][i]))):
                continue
            assert abs(tu[i, 0] - ref["t"][i]) <= P.TOL_T * ref["t"][i], (depth, i)
            k = int(leaf[i]) >> (23 - depth)
            assert k * 2.0 ** -depth <= tu[i, 1] <= (k + 1) * 2.0 ** -depth, (depth, i, k, tuple(tu[i]))
            overlap.append(i)
        stats["fail"] = np.setdiff1d(stats["fail"], overlap)
        _assert_parity(stats, max_band_frac=0.01, where="thick", depth=depth, overlap=len(overlap),
                       unsupported=info["n_unsupported"])
        assert len(overlap) <= 0.02 * n, (depth, len(overlap))
    fib.close()


def test_upload_rejects_bad_fibers():
    cps = I.tiny_case(n_ray=1)["cps"].copy()
    cps[3, 2, 3] = -0.1
    with pytest.raises(F.FiberxError):
        F.Fibers(cps)
    cps[3, 2, 3] = np.nan
    with pytest.raises(F.FiberxError):
        F.Fibers(cps)
    empty = F.Fibers(np.zeros((0, 4, 4), np.float32))
    assert empty.info()["n_piece"] == 0
    empty.close()


@pytest.fixture(scope="module")
def hair():
    """The full hair-patch frame and the oracle on every ray of it, at depth 10
    and at the benchmark's depth 15."""
    case = I.hair_patch()
    pieces = O.presplit(case["cps"])
    ref = {d: O.closest(case, d, pieces) for d in (10, 15)}
    return case, pieces, ref


# the bench's launch on the hair frame: the tuned scan variant, 5 CTAs per SM,
# chunks of 4 rays
BENCH_LAUNCH = (128, 5, 4, F.FX_VARIANT_SCAN)


@pytest.mark.parametrize("variant", [F.FX_VARIANT_AUTO, F.FX_VARIANT_LANE, F.FX_VARIANT_SCAN, F.FX_VARIANT_RAY],
                         ids=["auto", "lane", "scan", "ray"])
@pytest.mark.parametrize("depth", [10, 15])
@pytest.mark.parametrize("flags", MATH, ids=MATH_IDS)
def test_hair_patch_full_frame(hair, flags, depth, variant):
    # the benchmark's workload, every one of its 2,073,600 rays against the
    # oracle (the scan variant in the bench's launch shape)
    case, pieces, refs = hair
    ref = refs[depth]
    fib = F.Fibers(case["cps"])
    if variant == F.FX_VARIANT_SCAN:
        fib.set_launch(*BENCH_LAUNCH)
    else:
        fib.set_launch(variant=variant)
    tu, seg, leaf = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth, flags)
    torch.cuda.synchronize()
    assert fib.status() & ~F.FX_DEV_UNSUPPORTED == 0
    fib.close()
    tu, seg, leaf = _np(tu), _np(seg), _np(leaf)
    stats = P.compare_closest(case, depth, tu, seg, ref, pieces, leaf)
    # measured: at most 68 of the 2,073,600 rays pass by band, none by silhouette
    _assert_parity(stats, max_band_frac=1e-4, where="hair_full_frame", depth=depth, variant=int(variant),
                   math="fast" if flags else "ieee", rays_with_candidates=int(np.count_nonzero(np.diff(case["row_ptr"]))))
    assert stats["hits"] > 100_000
    # rays with no candidates are misses
    assert np.all(seg[np.diff(case["row_ptr"]) == 0] == -1)


@pytest.fixture(scope="module")
def hair_pairs(hair):
    """2000 seeded hair rays that have candidates (about 380,000 pairs) and the
    oracle's per-pair hits at depth 15."""
    case, pieces, _ = hair
    counts = np.diff(case["row_ptr"])
    idx = np.sort(np.random.default_rng(5).choice(np.nonzero(counts > 0)[0], 2000, replace=False))
    sub = I.subsample_rays(case, idx)
    return sub, pieces, O.pairs(sub, 15, pieces)


@pytest.mark.parametrize("kernel,variant", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("flags", MATH, ids=MATH_IDS)
def test_hair_pairs(hair_pairs, kernel, variant, flags):
    sub, pieces, pr = hair_pairs
    tu, leaf, st = _run_pairs(sub, 15, kernel, variant, flags)
    assert st & ~F.FX_DEV_UNSUPPORTED == 0
    stats = P.compare_pairs(sub, 15, tu, leaf, pr, pieces)
    _assert_parity(stats, max_band_frac=1e-4, where="hair_pairs", kernel=int(kernel), variant=int(variant),
                   flags=int(flags))
    assert stats["hits"] > 5000


def test_host_entry_edge_cases():
    # no rays; rays without any candidate (no pairs at all); a single ray;
    # per-ray depths from host memory
    case = I.sweep_case("moderate", 64, forced_hits=True)
    fib = F.Fibers(case["cps"])
    empty_rays = np.zeros((0, 8), np.float32)
    tu, seg, lf = F.intersect_closest_host(fib, empty_rays, np.zeros(1, np.int32), np.zeros(0, np.int32), 8)
    assert tu.shape[0] == 0 and seg.shape[0] == 0
    n = len(case["rays"])
    tu, seg, lf = F.intersect_closest_host(fib, case["rays"], np.zeros(n + 1, np.int32), np.zeros(0, np.int32), 8)
    assert np.all(np.isinf(tu.numpy()[:, 0])) and np.all(tu.numpy()[:, 1] == -1)
    assert np.all(seg.numpy() == -1) and np.all(lf.numpy() == -1)
    one = I.subsample_rays(case, np.array([5]))
    tu1, seg1, lf1 = F.intersect_closest_host(fib, one["rays"], one["row_ptr"], one["seg_idx"], 12)
    tu_d, seg_d, lf_d = F.intersect_closest(fib, one["rays"], one["row_ptr"], one["seg_idx"], 12)
    np.testing.assert_array_equal(tu1.numpy(), _np(tu_d))
    assert seg1.numpy()[0] == 5
    rd = np.arange(n, dtype=np.int8) % 24
    h = F.intersect_closest_host(fib, case["rays"], case["row_ptr"], case["seg_idx"], 8, ray_depth=rd)
    d = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], 8, ray_depth=rd)
    for a, b in zip(h, d):
        np.testing.assert_array_equal(a.numpy(), _np(b))
    assert fib.status() == 0
    fib.close()


@pytest.mark.parametrize("variant", [F.FX_VARIANT_LANE, F.FX_VARIANT_SCAN, F.FX_VARIANT_RAY, F.FX_VARIANT_WARP,
                                     F.FX_VARIANT_FILTER], ids=["lane", "scan", "ray", "warp", "filter"])
def test_concurrent_calls_on_one_handle(variant):
    # two calls on one handle in unordered streams, each several times over,
    # give the results of the same calls one after the other
    case = I.sweep_case("moderate", 1 << 16, forced_hits=True)
    g = np.random.default_rng(9)
    n = len(case["rays"])
    rows = [np.concatenate([[i], g.integers(0, n, 12)]).astype(np.int32) for i in range(n)]
    case2 = dict(case, seg_idx=np.concatenate(rows),
                 row_ptr=np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32))
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    dev = [tuple(torch.from_numpy(np.asarray(c[k])).cuda() for k in ("rays", "row_ptr", "seg_idx"))
           for c in (case, case2)]
    ref = [tuple(_np(x) for x in F.intersect_closest(fib, *d, 14)) for d in dev]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [[], []]
    torch.cuda.synchronize()
    for _ in range(4):
        for k in (0, 1):
            with torch.cuda.stream(streams[k]):
                outs[k].append(F.intersect_closest(fib, *dev[k], 14, stream=streams[k]))
    torch.cuda.synchronize()
    for k in (0, 1):
        for o in outs[k]:
            for a, b in zip(o, ref[k]):
                np.testing.assert_array_equal(_np(a), b)
    assert fib.status() == 0
    fib.close()


def test_host_entry_on_the_hair_frame(hair):
    # the end-to-end path the bench times (tuned launch: scan variant, fast
    # math, depth 15, pinned host buffers, chunked copies) equals the device
    # entry on the full frame, and every ray passes parity with the oracle
    case, pieces, ref = hair
    fib = F.Fibers(case["cps"])
    fib.set_launch(*BENCH_LAUNCH)
    h = [torch.from_numpy(case[k]).pin_memory() for k in ("rays", "row_ptr", "seg_idx")]
    tu_h, seg_h, leaf_h = F.intersect_closest_host(fib, *h, 15, F.FX_FAST_MATH)
    tu_d, seg_d, leaf_d = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], 15, F.FX_FAST_MATH)
    np.testing.assert_array_equal(tu_h.numpy(), _np(tu_d))
    np.testing.assert_array_equal(seg_h.numpy(), _np(seg_d))
    np.testing.assert_array_equal(leaf_h.numpy(), _np(leaf_d))
    h2d, d2h = F.host_bytes(fib)
    assert h2d < 32 * len(case["rays"]) + 4 * (len(case["rays"]) + 1) + 4 * len(case["seg_idx"])
    assert fib.status() == 0
    fib.close()
    stats = P.compare_closest(case, 15, tu_h.numpy(), seg_h.numpy(), ref[15], pieces, leaf_h.numpy())
    _assert_parity(stats, max_band_frac=1e-4, where="hair_host_entry")


def test_upload_from_device_memory_equals_host_upload(tiny):
    # fiber_upload with cps_on_device = 1 (a CUDA tensor) makes the same
    # handle as from host memory: same pieces, same results
    case, _, _ = tiny
    fh = F.Fibers(case["cps"])
    fd = F.Fibers(torch.from_numpy(case["cps"]).cuda())
    assert fh.info() == fd.info()
    args = (case["rays"], case["row_ptr"], case["seg_idx"], 12)
    for a, b in zip(F.intersect_closest(fh, *args), F.intersect_closest(fd, *args)):
        np.testing.assert_array_equal(_np(a), _np(b))
    fh.close()
    fd.close()


@pytest.mark.parametrize("variant,kernel", [(F.FX_VARIANT_LANE, 0), (F.FX_VARIANT_SCAN, 0), (F.FX_VARIANT_RAY, 0),
                                            (F.FX_VARIANT_WARP, 0), (F.FX_VARIANT_FILTER, 0),
                                            (0, F.FX_KERNEL_NAIVE)],
                         ids=["lane", "scan", "ray", "warp", "filter", "naive"])
def test_malformed_row_ptr_is_clamped_under_check_index(variant, kernel):
    # with FX_CHECK_INDEX a row_ptr with negative, too large and decreasing
    # entries reads nothing out of range: the bad rows are clamped to
    # [0, n_pair] and flagged, and every other ray's result is unchanged
    case = I.sweep_case("moderate", 4096, forced_hits=True)
    n = len(case["rays"])
    g = np.random.default_rng(13)
    rows = [np.concatenate([[i], g.integers(0, n, 3)]).astype(np.int32) for i in range(n)]
    seg_idx = np.concatenate(rows)
    good = (np.arange(n + 1) * 4).astype(np.int32)
    bad = good.copy()
    n_pair = len(seg_idx)
    bad[100] = -7
    bad[200] = n_pair + 50
    bad[300] = bad[299] - 3
    bad[n] = n_pair + 10
    touched = np.zeros(n, bool)
    touched[[99, 100, 199, 200, 299, 300, n - 1]] = True
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    flags = kernel | F.FX_CHECK_INDEX
    ref = [_np(x) for x in F.intersect_closest(fib, case["rays"], good, seg_idx, 12, flags)]
    assert fib.status() == 0
    got = [_np(x) for x in F.intersect_closest(fib, case["rays"], bad, seg_idx, 12, flags)]
    st = fib.status()
    if kernel == 0:  # the naive kernel maps pairs to rays and reads no row as such
        assert st & F.FX_DEV_BAD_INDEX
    assert st & ~F.FX_DEV_BAD_INDEX == 0
    if kernel == 0:  # the row kernels keep every other ray's result (the naive
        # kernel's pair-to-ray search assumes a sorted row_ptr)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a[~touched], b[~touched])
    assert np.all((got[1] >= -1) & (got[1] < n))
    fib.close()
