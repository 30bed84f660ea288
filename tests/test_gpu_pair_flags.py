"""Per-pair status bytes of intersect_pairs (pair_flags): zero on valid
pairs, FX_DEV_BAD_INDEX exactly on out-of-range segment ids, and
FX_DEV_UNSUPPORTED exactly on hits in pieces the pre-split left
unsupported, on every per-pair path."""
import numpy as np
import pytest

import oracle as O
from paper_1811_03374_gb300 import fiberx as F
from paper_1811_03374_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PATHS = [(F.FX_VARIANT_LANE, 0), (F.FX_VARIANT_WARP, 0), (F.FX_VARIANT_SCAN, 0), (F.FX_VARIANT_RAY, 0),
         (0, F.FX_KERNEL_NAIVE)]
IDS = ["lane", "warp", "scan", "ray", "naive"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _np(x):
    return x.cpu().numpy()


@pytest.mark.parametrize("variant,kernel", PATHS, ids=IDS)
def test_bad_ids_are_flagged_pair_by_pair(variant, kernel):
    case = I.sweep_case("moderate", 2048, forced_hits=True)
    n = len(case["rays"])
    g = np.random.default_rng(11)
    rows = [np.concatenate([[i], g.integers(0, n, 3)]).astype(np.int32) for i in range(n)]
    seg_idx = np.concatenate(rows)
    bad = g.random(len(seg_idx)) < 0.05
    seg_idx[bad] = np.where(g.random(bad.sum()) < 0.5, -1, n + 7)
    row_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    tu, leaf, pf = (_np(x) for x in F.intersect_pairs(fib, case["rays"], row_ptr, seg_idx, 12,
                                                        kernel | F.FX_CHECK_INDEX, pair_flags=True))
    assert fib.status() == F.FX_DEV_BAD_INDEX
    np.testing.assert_array_equal(pf, np.where(bad, F.FX_DEV_BAD_INDEX, 0).astype(np.uint8))
    assert np.all(np.isinf(tu[bad, 0])) and np.all(leaf[bad] == -1)
    assert np.isfinite(tu[~bad, 0]).sum() > 1500
    # the valid pairs' results equal a run without the bad ids' neighbours changed
    ok_idx = np.where(~bad, seg_idx, 0)
    tu2, _ = (_np(x) for x in F.intersect_pairs(fib, case["rays"], row_ptr, ok_idx, 12, kernel))
    np.testing.assert_array_equal(tu[~bad], tu2[~bad])
    fib.close()


@pytest.mark.parametrize("variant,kernel", [p for p in PATHS if p[0] != F.FX_VARIANT_SCAN],
                         ids=[i for i, p in zip(IDS, PATHS) if p[0] != F.FX_VARIANT_SCAN])
def test_unsupported_hits_are_flagged_pair_by_pair(variant, kernel):
    # the tiny workload has pieces the pre-split leaves unsupported; a pair
    # whose reported hit lies in one is flagged, and a flagged pair is a hit
    # of a segment with an unsupported piece (a hit there may have been
    # replaced by a closer one on a later piece of the same segment)
    case = I.subsample_rays(I.tiny_case(), np.arange(0, 16384, 4))
    pieces = O.presplit(case["cps"])
    assert pieces["flags"].any()
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    tu, leaf, pf = (_np(x) for x in F.intersect_pairs(fib, case["rays"], case["row_ptr"], case["seg_idx"], 8,
                                                        kernel, pair_flags=True))
    fib.close()
    hit = np.isfinite(tu[:, 0])
    assert set(np.unique(pf)) <= {0, F.FX_DEV_UNSUPPORTED}
    assert not np.any(pf[~hit])
    seg = case["seg_idx"]
    expect = np.zeros(len(seg), bool)
    has_unsupported = np.zeros(len(seg), bool)
    for j in np.nonzero(hit)[0]:
        b, e = pieces["begin"][seg[j]], pieces["begin"][seg[j] + 1]
        has_unsupported[j] = bool(np.any(pieces["flags"][b:e] & 1))
        for k in range(b, e):
            sh = 23 - int(pieces["level"][k])
            if int(pieces["off"][k]) << sh <= leaf[j] < (int(pieces["off"][k]) + 1) << sh:
                expect[j] = bool(pieces["flags"][k] & 1)
                break
    assert np.all(pf[expect] != 0)
    assert np.all(has_unsupported[pf != 0])
    assert expect.sum() > 0 and (pf != 0).sum() <= expect.sum() + 0.01 * hit.sum()
