"""Precision stress on the GPU: rays grazing the fiber silhouette (within
1e-3 r of it) and scenes translated by 1e3 and 1e4 units against thin fibers
(r = 1e-4 of the segment length), at depths 16 and 22.  Three modes: the FP32
traversal alone (IEEE and approximate math), and FP32 followed by the FP64
re-evaluation of the hit leaf (FX_POLISH_FP64), each against the FP64
oracle.  The polish re-evaluates the FP32 traversal's leaf and its two
neighbours on either side and keeps the nearest entry.

Every ray must pass the parity rule of tests/_parity.py (strict agreement,
agreement with the oracle for a ray shifted within the FP32 resolution band,
or a silhouette within 1e-4 r of the ray).  With the polish, a hit on the
oracle's leaf must carry the oracle's t to one FP32 rounding.

Far from the origin the ray-centric frame keeps its precision: the offset of
a control point from a ray origin ten units away is exact in FP32 (both lie
within a factor of two of each other), so only the rotation rounds, at the
scale of the ten-unit distance, not of the 1e4 offset.  The hit/miss
disagreement rate is bounded accordingly.

With FX_REPORT=<path> set, every case appends one JSON line with its hit/miss
disagreement rate, its counts and its largest relative t error."""
import numpy as np
import pytest

import oracle as O
from paper_1811_03374_gb300 import fiberx as F
from paper_1811_03374_gb300 import inputs as I
from tests import _parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 50_000
MODES = {"fp32": 0, "fp32_fast": F.FX_FAST_MATH, "fp32_polish": F.FX_POLISH_FP64}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _case(name):
    if name == "grazing":
        return I.grazing_case(N)
    return I.offset_case(N, float(name.split("_")[1]))


@pytest.mark.parametrize("name", ["grazing", "offset_1e3", "offset_1e4"])
@pytest.mark.parametrize("depth", [16, 22])
def test_precision_stress(name, depth):
    case = _case(name)
    pieces = O.presplit(case["cps"])
    ref = O.closest(case, depth, pieces)
    hit_o = ref["seg"] >= 0
    fib = F.Fibers(case["cps"])
    for mode, flags in MODES.items():
        tu, seg, leaf = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth, flags)
        torch.cuda.synchronize()
        assert fib.status() & ~F.FX_DEV_UNSUPPORTED == 0
        tu, seg, leaf = tu.cpu().numpy(), seg.cpu().numpy(), leaf.cpu().numpy()
        stats = P.compare_closest(case, depth, tu, seg, ref, pieces, leaf)
        assert len(stats["fail"]) == 0, (name, depth, mode, stats["detail"])
        hit_g = seg >= 0
        disagree = float(np.mean(hit_g != hit_o))
        same = hit_g & hit_o & (seg == ref["seg"])
        rel = np.abs(tu[same, 0].astype(np.float64) - ref["t"][same]) / ref["t"][same]
        same_leaf = same & (leaf == ref["leaf"])
        rel_leaf = np.abs(tu[same_leaf, 0].astype(np.float64) - ref["t"][same_leaf]) / ref["t"][same_leaf]
        if mode == "fp32_polish" and same_leaf.any():
            # the FP64 t of the oracle's own leaf, rounded once to FP32 (at
            # depth 22 far from the origin the leaves are shorter than the
            # FP32 spacing of the hit point, and FP32 cannot single out the
            # oracle's leaf: only those hits on it are held to this)
            assert rel_leaf.max() <= 2.0 ** -23, (name, depth, rel_leaf.max())
        # FP32 can decide hit or miss only outside its resolution band (see
        # the module docstring): a bounded share of rays, all passing the
        # parity rule above
        assert disagree <= 0.05, (name, depth, mode, disagree)
        P.report(dict(case=name, depth=depth, mode=mode, n=int(len(seg)), oracle_hits=int(hit_o.sum()),
                     hit_miss_disagreement=disagree, strict=stats["strict"], band=stats["band"],
                     silhouette=stats["silhouette"], max_rel_t_same_segment=float(rel.max()) if rel.size else 0.0,
                     median_rel_t_same_segment=float(np.median(rel)) if rel.size else 0.0,
                     max_rel_t_same_leaf=float(rel_leaf.max()) if rel_leaf.size else 0.0,
                     same_leaf_fraction=float(same_leaf.sum() / max(1, hit_o.sum()))))
    fib.close()
