"""Per-ray subdivision depth (the ray_depth argument): each ray's result equals
that of a launch at its own depth, bit for bit, on every variant, the naive
kernel, the per-pair mode, the FP64 polish, the normals and the host-buffer
entry; against the FP64 oracle ray by ray on a pre-split workload; and
entries outside [0, 23] are clamped and reported."""
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


def _case():
    """Moderate sweep segments with forced hits, each ray's own segment among
    up to 40 random others (rows longer than a scan window)."""
    case = I.sweep_case("moderate", 4096, forced_hits=True)
    g = np.random.default_rng(17)
    n = len(case["rays"])
    rows = [np.concatenate([[i], g.integers(0, n, g.integers(0, 41))]).astype(np.int32) for i in range(n)]
    rows = [r[g.permutation(len(r))] for r in rows]
    return dict(case, seg_idx=np.concatenate(rows),
                row_ptr=np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32))


def _depths(n, seed=5):
    return np.random.default_rng(seed).integers(0, 24, n).astype(np.int8)


VARIANTS = [F.FX_VARIANT_LANE, F.FX_VARIANT_WARP, F.FX_VARIANT_FILTER, F.FX_VARIANT_SCAN, F.FX_VARIANT_RAY]


@pytest.mark.parametrize("variant", VARIANTS, ids=["lane", "warp", "filter", "scan", "ray"])
@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH, F.FX_KERNEL_NAIVE, F.FX_POLISH_FP64],
                         ids=["ieee", "fast", "naive", "polish"])
def test_closest_equals_uniform_launches(variant, flags):
    case = _case()
    rd = _depths(len(case["rays"]))
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    args = (case["rays"], case["row_ptr"], case["seg_idx"])
    got = [_np(x) for x in F.intersect_closest(fib, *args, 8, flags, ray_depth=rd)]
    for d in np.unique(rd):
        m = rd == d
        ref = [_np(x) for x in F.intersect_closest(fib, *args, int(d), flags)]
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a[m], b[m], err_msg="depth %d" % d)
    assert fib.status() == 0
    assert (got[1] >= 0).sum() > 3500
    fib.close()


@pytest.mark.parametrize("variant", [F.FX_VARIANT_LANE, F.FX_VARIANT_SCAN, F.FX_VARIANT_RAY],
                         ids=["lane", "scan", "ray"])
def test_pairs_equal_uniform_launches(variant):
    case = _case()
    rd = _depths(len(case["rays"]), seed=6)
    pair_depth = np.repeat(rd, np.diff(case["row_ptr"]))
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    args = (case["rays"], case["row_ptr"], case["seg_idx"])
    tu, lf = (_np(x) for x in F.intersect_pairs(fib, *args, 8, F.FX_FAST_MATH, ray_depth=rd))
    for d in np.unique(rd):
        m = pair_depth == d
        tu_d, lf_d = (_np(x) for x in F.intersect_pairs(fib, *args, int(d), F.FX_FAST_MATH))
        np.testing.assert_array_equal(tu[m], tu_d[m])
        np.testing.assert_array_equal(lf[m], lf_d[m])
    fib.close()


def test_normals_and_host_entry_follow_the_ray_depths():
    case = _case()
    rd = _depths(len(case["rays"]), seed=7)
    fib = F.Fibers(case["cps"])
    args = (case["rays"], case["row_ptr"], case["seg_idx"])
    tu, seg, leaf = F.intersect_closest(fib, *args, 8, ray_depth=rd)
    nrm = _np(F.intersect_normals(fib, case["rays"], tu, seg, leaf, 8, ray_depth=rd))
    for d in np.unique(rd):
        m = rd == d
        tu_d, seg_d, leaf_d = F.intersect_closest(fib, *args, int(d))
        n_d = _np(F.intersect_normals(fib, case["rays"], tu_d, seg_d, leaf_d, int(d)))
        np.testing.assert_array_equal(nrm[m], n_d[m])
    h = F.intersect_closest_host(fib, *args, 8, ray_depth=rd)
    for a, b in zip(h, (tu, seg, leaf)):
        np.testing.assert_array_equal(a.numpy(), _np(b))
    assert fib.status() == 0
    fib.close()


def test_presplit_fibers_against_the_oracle():
    # the tiny workload (pre-split pieces) with a depth per ray, compared
    # with the oracle run at each ray's depth
    case = I.tiny_case()
    n = len(case["rays"])
    rd = np.random.default_rng(8).choice(np.array([2, 5, 8, 12, 16, 22], np.int8), n)
    pieces = O.presplit(case["cps"])
    fib = F.Fibers(case["cps"])
    tu, seg, leaf = (_np(x) for x in F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], 8,
                                                          ray_depth=rd))
    assert fib.status() & ~F.FX_DEV_UNSUPPORTED == 0
    fib.close()
    for d in np.unique(rd):
        idx = np.nonzero(rd == d)[0]
        sub = I.subsample_rays(case, idx)
        ref = O.closest(sub, int(d), pieces)
        stats = P.compare_closest(sub, int(d), tu[idx], seg[idx], ref, pieces, leaf[idx])
        assert len(stats["fail"]) == 0, (int(d), stats["detail"])
        assert stats["band"] + stats["silhouette"] <= 5e-3 * stats["n"]


def test_out_of_range_depths_are_clamped_and_reported():
    case = _case()
    n = len(case["rays"])
    rd = np.where(np.arange(n) % 2 == 0, 30, -3).astype(np.int8)
    fib = F.Fibers(case["cps"])
    args = (case["rays"], case["row_ptr"], case["seg_idx"])
    got = [_np(x) for x in F.intersect_closest(fib, *args, 8, ray_depth=rd)]
    assert fib.status() & F.FX_DEV_BAD_DEPTH
    assert fib.status() == 0  # cleared by the read
    for d, m in ((23, rd == 30), (0, rd == -3)):
        ref = [_np(x) for x in F.intersect_closest(fib, *args, d)]
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a[m], b[m])
    fib.close()
