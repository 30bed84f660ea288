"""Per-ray pruning-test counts on the GPU (intersect_counts, Fig. 8) against
the FP64 oracle's, ray by ray, through the C ABI: oriented cylinders and
ray-frame boxes, on single fibers of three curvature classes, the depth
sweep (the curved class pre-split), the tiny workload (pre-split, 16
candidates per ray) and the hair patch.  A count sums integer outcomes of
floating-point tests over a ray's row, so every ray's count must equal the
oracle's, or, where FP32 settled a test on a grazing bounding volume the
other way, equal the oracle's count for the same ray shifted sideways
within the FP32 resolution band (tests/_parity.py); such rays stay a small
share.  The boxes are aligned to Duff et al.'s frame on both sides (a box in
the ray's frame depends on the frame's rotation about the ray).  With
FX_REPORT=<path> set, every comparison appends its counts."""
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


def _compare(case, depth, mode, flags=0, max_band_frac=2e-3, **rec):
    pieces = O.presplit(case["cps"])
    ref, _ = O.ray_counts(case, depth, mode, pieces)
    fib = F.Fibers(case["cps"])
    got = F.intersect_counts(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth, boxes=mode == "box",
                             flags=flags).cpu().numpy().astype(np.int64)
    assert fib.status() & ~F.FX_DEV_UNSUPPORTED == 0
    fib.close()
    diff = np.nonzero(got != ref)[0]
    band = P.band_counts(case, diff, got, depth, mode, pieces)
    fail = diff[~band]
    st = dict(n=len(got), equal=int(len(got) - len(diff)), band=int(band.sum()), fail=int(len(fail)),
              mean=float(got.mean()), max=int(got.max()), p99=float(np.percentile(got, 99)))
    P.report(dict(test="counts", depth=depth, mode=mode, math="fast" if flags & F.FX_FAST_MATH else "ieee",
                  **rec, **st))
    assert len(fail) == 0, (mode, depth, fail[:8].tolist(), got[fail[:8]].tolist(), ref[fail[:8]].tolist())
    assert len(diff) <= max_band_frac * len(got), (mode, depth, len(diff))
    return st


@pytest.mark.parametrize("klass", list(I.SWEEP_JITTER))
@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
def test_counts_single_fiber(klass, flags):
    case = I.single_fiber_case(klass, 8192)
    for depth in (2, 8, 12, 16):
        for mode in ("cylinder", "box"):
            # box searches are long at depth: more tests, more grazing ones
            _compare(case, depth, mode, flags, 2e-3 if mode == "cylinder" else 1e-2, case="single_" + klass)


@pytest.mark.parametrize("klass", list(I.SWEEP_JITTER))
def test_counts_depth_sweep(klass):
    # the curved class holds pre-split segments: each piece searched to
    # depth - level
    case = I.sweep_case(klass, 4096)
    for depth in (4, 12):
        for mode in ("cylinder", "box"):
            _compare(case, depth, mode, 0, 2e-3 if mode == "cylinder" else 1e-2, case="sweep_" + klass)


@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
def test_counts_tiny_presplit(flags):
    # 16 random cubics, most of them pre-split, 16 candidates per ray
    case = I.tiny_case()
    fib = F.Fibers(case["cps"])
    assert fib.info()["n_presplit"] > 0
    fib.close()
    for depth in (4, 8):
        for mode in ("cylinder", "box"):
            _compare(case, depth, mode, flags, 5e-3 if mode == "cylinder" else 2e-2, case="tiny")


def test_counts_hair():
    case = I.hair_patch()
    counts = np.diff(case["row_ptr"])
    idx = np.sort(np.random.default_rng(9).choice(np.nonzero(counts > 0)[0], 2000, replace=False))
    sub = I.subsample_rays(case, idx)
    # a hair ray sums about 190 candidates' searches: a grazing test anywhere
    # in the row moves its count
    _compare(sub, 15, "cylinder", F.FX_FAST_MATH, 2e-2, case="hair")
