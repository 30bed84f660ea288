"""Per-ray pruning-test counts on the GPU (intersect_counts, Fig. 8) against
the FP64 oracle's, ray by ray, through the C ABI: oriented cylinders and
ray-frame boxes, on single fibers of three curvature classes, the depth
sweep (the curved class pre-split), the tiny workload (pre-split, 16
candidates per ray) and the hair patch.  A count sums integer outcomes of
floating-point tests over a ray's row.  The oracle flags the rays whose
search has a decision within the FP32 band of flipping (a move of the ray
sideways by 1e-4 r + 22 * 2^-24 T, tests/_parity.py); every other ray's
count must equal the oracle's exactly, and flagged rays with a different
count stay a small share.  The boxes are aligned to Duff et al.'s frame on
both sides (a box in the ray's frame depends on the frame's rotation about
the ray).  With FX_REPORT=<path> set, every comparison appends its counts."""
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
    ref, amb = O.ray_counts_amb(case, depth, mode, P.count_band_delta(case), pieces)
    fib = F.Fibers(case["cps"])
    got = F.intersect_counts(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth, boxes=mode == "box",
                             flags=flags).cpu().numpy().astype(np.int64)
    assert fib.status() & ~F.FX_DEV_UNSUPPORTED == 0
    fib.close()
    diff = got != ref
    fail = np.nonzero(diff & ~amb)[0]
    st = dict(n=len(got), equal=int((~diff).sum()), band=int((diff & amb).sum()), fail=int(len(fail)),
              flagged=int(amb.sum()), mean=float(got.mean()), max=int(got.max()),
              p99=float(np.percentile(got, 99)))
    P.report(dict(test="counts", depth=depth, mode=mode, math="fast" if flags & F.FX_FAST_MATH else "ieee",
                  **rec, **st))
    assert len(fail) == 0, (mode, depth, fail[:8].tolist(), got[fail[:8]].tolist(), ref[fail[:8]].tolist())
    assert diff.sum() <= max_band_frac * len(got), (mode, depth, int(diff.sum()))
    return st


@pytest.mark.parametrize("klass", list(I.SWEEP_JITTER))
@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
def test_counts_single_fiber(klass, flags):
    case = I.single_fiber_case(klass, 8192)
    for depth in (2, 8, 12, 16):
        for mode in ("cylinder", "box"):
            # box searches are long at depth: more tests, more grazing ones
            _compare(case, depth, mode, flags, 2e-3 if mode == "cylinder" else 1e-2, workload="single_" + klass)


@pytest.mark.parametrize("klass", list(I.SWEEP_JITTER))
def test_counts_depth_sweep(klass):
    # the curved class holds pre-split segments: each piece searched to
    # depth - level
    case = I.sweep_case(klass, 4096)
    for depth in (4, 12):
        for mode in ("cylinder", "box"):
            _compare(case, depth, mode, 0, 2e-3 if mode == "cylinder" else 1e-2, workload="sweep_" + klass)


@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
def test_counts_tiny_presplit(flags):
    # 16 random cubics, most of them pre-split, 16 candidates per ray
    case = I.tiny_case()
    fib = F.Fibers(case["cps"])
    assert fib.info()["n_presplit"] > 0
    fib.close()
    for depth in (4, 8):
        for mode in ("cylinder", "box"):
            _compare(case, depth, mode, flags, 5e-3 if mode == "cylinder" else 2e-2, workload="tiny")


def test_counts_hair():
    case = I.hair_patch()
    counts = np.diff(case["row_ptr"])
    idx = np.sort(np.random.default_rng(9).choice(np.nonzero(counts > 0)[0], 2000, replace=False))
    sub = I.subsample_rays(case, idx)
    # a hair ray sums about 190 candidates' searches, and at depth 15 a hit's
    # last split decisions lie within the FP32 band (leaves 6e-7 long against
    # a band of about 5e-6): the oracle flags 87 % of these rays; 5 % of them
    # were measured with a different count
    _compare(sub, 15, "cylinder", F.FX_FAST_MATH, 0.1, workload="hair")
