"""Hit normals on the GPU (intersect_normals, App. C) against the FP64
oracle's, through the C ABI, on seeded inputs: the depth-sweep classes
(single-piece handles), the tiny workload (pre-split pieces) and the hair
patch at the benchmark's depth.

Compared where both sides hit the same leaf of the same segment with the
same t (the parity rule's strict agreement).  Tolerance, from the arithmetic:
the FP32 normal is the hit point minus the axis point, a vector of length
len (the oracle's, FP64) whose ends carry the FP32 spacing of ray-frame
coordinates, 8 * 2^-24 * (|o| + t), plus the two sides' difference in t; so
the angle between the normals is at most 4 * (that spacing + |dt|) / len,
plus 1e-6.  End-cap normals are the normalised p0 - p1 (p3 - p2) on both
sides (1e-6).  The two sides may classify a hit differently (cap or lateral)
only within that spacing of the end plane."""
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


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _check_normals(case, depth, flags=0, variant=F.FX_VARIANT_AUTO, min_compared=200):
    pieces = O.presplit(case["cps"])
    ref = O.closest(case, depth, pieces)
    n_ref, kind_ref, length = O.normals(case, depth, ref, pieces)
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    tu, seg, leaf = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth, flags)
    nrm = F.intersect_normals(fib, case["rays"], tu, seg, leaf, depth, flags)
    torch.cuda.synchronize()
    assert fib.status() & ~F.FX_DEV_UNSUPPORTED == 0
    fib.close()
    tu, seg, leaf, nrm = tu.cpu().numpy(), seg.cpu().numpy(), leaf.cpu().numpy(), nrm.cpu().numpy()
    hit = seg >= 0
    assert np.all(nrm[~hit] == 0.0)
    np.testing.assert_allclose(np.linalg.norm(nrm[hit], axis=1), 1.0, atol=2e-6)
    tol_u = P.u_tolerance(case, case["rays"], ref["seg"].astype(np.int64), ref["t"], ref["u"])
    strict = P.strict_ok(tu[:, 0].astype(np.float64), tu[:, 1].astype(np.float64), seg.astype(np.int64),
                         ref["t"], ref["u"], ref["seg"].astype(np.int64), tol_u)
    same = hit & strict & (ref["seg"] >= 0) & (leaf == ref["leaf"])
    idx = np.nonzero(same)[0]
    assert len(idx) >= min_compared, len(idx)
    cp = case["cps"][seg[idx]].astype(np.float64)
    cap0, cap3 = _unit(cp[:, 0, :3] - cp[:, 1, :3]), _unit(cp[:, 3, :3] - cp[:, 2, :3])
    g = nrm[idx].astype(np.float64)
    kind_gpu = np.where(np.linalg.norm(g - cap0, axis=1) < 1e-5, 2,
                        np.where(np.linalg.norm(g - cap3, axis=1) < 1e-5, 3, 1))
    rays = case["rays"][idx].astype(np.float64)
    o = rays[:, :3]
    t = ref["t"][idx]
    dt = np.abs(tu[idx, 0] - t)
    spacing = 8 * 2.0 ** -24 * (np.linalg.norm(o, axis=1) + t) + dt
    # classification: only within the spacing of an end plane may the sides differ
    diff = kind_gpu != kind_ref[idx]
    if diff.any():
        w = _unit(rays[:, 4:7])
        x = o + t[:, None] * w
        s0 = np.abs(np.sum((x - cp[:, 0, :3]) * cap0, axis=1))
        s3 = np.abs(np.sum((x - cp[:, 3, :3]) * cap3, axis=1))
        band = np.minimum(s0, s3) <= 4 * spacing
        assert np.all(band[diff]), np.nonzero(diff & ~band)[0][:5]
        assert diff.mean() < 0.01
    agree = ~diff
    # angle from the cross and dot products of the renormalised vectors (arccos
    # of a dot product near 1 turns an FP32 length error of 1e-7 into 4e-4)
    gu = _unit(g)
    ang = np.arctan2(np.linalg.norm(np.cross(gu, n_ref[idx]), axis=1), np.sum(gu * n_ref[idx], axis=1))
    lat = agree & (kind_ref[idx] == 1)
    tol = 4 * spacing / np.maximum(length[idx], 1e-30) + 1e-6
    bad = lat & (ang > tol)
    assert not bad.any(), [(int(idx[i]), float(ang[i]), float(tol[i])) for i in np.nonzero(bad)[0][:5]]
    capm = agree & (kind_ref[idx] != 1)
    assert not capm.any() or ang[capm].max() <= 1e-6
    return dict(compared=len(idx), lateral=int(lat.sum()), caps=int(capm.sum()), kind_diff=int(diff.sum()),
                max_angle=float(ang[lat].max()) if lat.any() else 0.0,
                median_angle=float(np.median(ang[lat])) if lat.any() else 0.0)


@pytest.mark.parametrize("klass", ["straight", "moderate"])
@pytest.mark.parametrize("depth", [4, 12, 22])
@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
def test_normals_depth_sweep(klass, depth, flags):
    st = _check_normals(I.sweep_case(klass, 4096, forced_hits=True), depth, flags)
    P.report(dict(test="normals", case=klass, depth=depth, math="fast" if flags else "ieee", **st))


def test_normals_end_caps():
    # rays aimed at the end disks of straight fibers hit caps on both sides
    g = np.random.default_rng(11)
    n = 2048
    A = g.uniform(-3, 3, (n, 3))
    ax = _unit(g.standard_normal((n, 3)))
    B = A + ax
    cps = np.stack([A + k / 3.0 * (B - A) for k in range(4)], axis=1)
    r = g.uniform(0.05, 0.2, (n, 1))
    cps = np.concatenate([cps, np.repeat(r[:, None], 4, axis=1)], axis=2).astype(np.float32)
    end = g.integers(0, 2, n)
    P_ = np.where(end[:, None] == 0, A, B)
    out = np.where(end[:, None] == 0, -ax, ax)
    e = _unit(np.cross(ax, g.standard_normal((n, 3))))
    q = P_ + 0.6 * r * g.uniform(0, 1, (n, 1)) * e
    w = _unit(-out + 0.3 * np.cross(out, e))
    rays = I.pack_rays(q - 3.0 * w, w)
    rp, si = I.diagonal_csr(n)
    case = dict(cps=cps, rays=rays, row_ptr=rp, seg_idx=si)
    st = _check_normals(case, 10, 0, min_compared=1500)
    assert st["caps"] >= 1500


def test_normals_presplit_tiny():
    case = I.tiny_case()
    _check_normals(case, 8, 0, min_compared=2000)


@pytest.mark.parametrize("variant", [F.FX_VARIANT_LANE, F.FX_VARIANT_SCAN], ids=["lane", "scan"])
def test_normals_hair(variant):
    case = I.hair_patch()
    counts = np.diff(case["row_ptr"])
    idx = np.sort(np.random.default_rng(8).choice(np.nonzero(counts > 0)[0], 3000, replace=False))
    sub = I.subsample_rays(case, idx)
    st = _check_normals(sub, 15, F.FX_FAST_MATH, variant=variant, min_compared=1500)
    P.report(dict(test="normals", case="hair", depth=15, math="fast", variant=int(variant), **st))
