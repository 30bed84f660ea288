"""Quadratic fibers on the GPU (fiber_upload_quadratic: exact degree
elevation, then the cubic path) against the FP64 oracle, which raises the
same FP32 control points in FP64: the depth-sweep classes,
forced hits and box-aimed rays, IEEE and fast math, depths 2-22, and the
adjoint through the autograd Function against FP64 central finite
differences on the quadratic control points."""
import numpy as np
import pytest

import oracle as O
from paper_1811_03374_gb300 import fiberx as F
from paper_1811_03374_gb300 import inputs as I
from tests import _parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEPTHS = [2, 4, 8, 12, 16, 22]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("klass", list(I.SWEEP_JITTER))
@pytest.mark.parametrize("forced", [False, True], ids=["aabb", "forced"])
@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH], ids=["ieee", "fast"])
def test_quadratic_depth_sweep(klass, forced, flags):
    case = I.quadratic_case(klass, 4096, forced_hits=forced)
    cubic = dict(case, cps=O.elevate_quadratics(case["cps"]))  # for the parity helpers
    pieces = O.presplit(case["cps"])
    fib = F.Fibers(case["cps"])
    info = fib.info()
    # the same pre-split as the oracle's (upload in FP64 from the raised curve)
    assert fib.quadratic and info["n_piece"] == len(pieces["seg"])
    assert info["n_unsupported"] == int(pieces["flags"].sum())
    for depth in DEPTHS:
        ref = O.closest(case, depth, pieces)
        tu, seg, leaf = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth, flags)
        torch.cuda.synchronize()
        tu, seg, leaf = tu.cpu().numpy(), seg.cpu().numpy(), leaf.cpu().numpy()
        stats = P.compare_closest(cubic, depth, tu, seg, ref, pieces, leaf)
        assert len(stats["fail"]) == 0, (klass, depth, stats["detail"])
        assert stats["band"] + stats["silhouette"] <= 5e-3 * stats["n"]
        assert stats["max_rel_t"] <= P.TOL_T and stats["max_du_over_tol"] <= 1.0
        if forced:
            assert stats["hits"] > 3500
        P.report(dict(test="quadratic", klass=klass, forced=forced, math="fast" if flags else "ieee", depth=depth,
                      n=stats["n"], hits=stats["hits"], strict=stats["strict"], band=stats["band"],
                      max_rel_t=stats["max_rel_t"]))
    assert fib.status() & ~F.FX_DEV_UNSUPPORTED == 0
    fib.close()


def test_valid_quadratics_are_not_presplit():
    # a quadratic meeting App. B.1's constraint raises to a valid cubic
    case = I.quadratic_case("straight", 2048)
    valid = np.array([O.valid_quadratic(q) for q in case["cps"].astype(np.float64)])
    assert valid.all()
    fib = F.Fibers(case["cps"], thick_check=False)
    assert fib.info()["n_piece"] == 2048 and fib.info()["n_presplit"] == 0
    fib.close()


def test_quadratic_gradient_matches_finite_differences():
    # t of the limit-surface hit as a function of the quadratic control
    # points, differentiated by FP64 central differences (h = 1e-6) through
    # the elevation and the oracle's limit-surface root search, against the
    # adjoint kernel through the autograd Function (chain rule to p0..p2)
    case = I.quadratic_case("moderate", 64, seed=77, forced_hits=True)
    depth = 16
    fib = F.Fibers(case["cps"])
    cps = torch.tensor(case["cps"], device="cuda", requires_grad=True)
    t, u, s = F.fiber_intersect(cps, case["rays"], case["row_ptr"], case["seg_idx"], depth, fib)
    hit = (s >= 0).cpu().numpy()
    t.sum().backward()
    g = cps.grad.cpu().numpy().astype(np.float64)
    fib.close()
    h = 1e-6
    checked = 0
    for i in np.nonzero(hit)[0]:
        r7 = O.ray7_from_packed(case["rays"][i])
        q = case["cps"][i].astype(np.float64)
        kind, t0, u0 = O.limit_hit(r7, O.elevate_quadratics(q[None])[0], 20000)
        if kind != 1 or abs(t0 - t[i].item()) > 1e-4 * t0 or not (0.01 < u0 < 0.99):
            continue  # only well-inside lateral hits: dt/dtheta jumps at the rim
        w = r7[3:6] / np.linalg.norm(r7[3:6])
        c = O.elevate_quadratics(q[None])[0]
        x = r7[:3] + t0 * w
        cu = I.bezier(c[None], np.array([u0]))[0]
        if abs(np.dot(x - cu[:3], w)) < 0.05 * cu[3]:
            continue  # grazing: the system is near singular
        fd = np.zeros((3, 4))
        ok = True
        for k in range(3):
            for a in range(4):
                tt = []
                for sgn in (1, -1):
                    qq = q.copy()
                    qq[k, a] += sgn * h
                    kd, ti, _ = O.limit_hit(r7, O.elevate_quadratics(qq[None])[0], 20000)
                    if kd != kind:
                        ok = False
                    tt.append(ti)
                fd[k, a] = (tt[0] - tt[1]) / (2 * h)
        if not ok:
            continue
        err = np.linalg.norm(g[i] - fd) / np.linalg.norm(fd)
        assert err < 1e-3, (i, err, g[i].round(5).tolist(), fd.round(5).tolist())
        checked += 1
    assert checked > 25
