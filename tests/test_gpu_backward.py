"""The hand-written adjoint kernel (intersect_backward, through the C ABI and
the autograd Function) against the oracle's implicit-function gradient of the
limit-surface hit, on hair-patch geometry.  The oracle computes its own
forward hits; nothing from the CUDA path enters it."""
import numpy as np
import pytest

import oracle as O
from paper_1811_03374_gb300 import fiberx as F
from paper_1811_03374_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DEPTH = 16


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


GRAZING = 0.05  # incidence cosine below GRAZING: the system is near singular
RIM = 1e-3      # within RIM (in u, or relative radius on a disk) of the rim
N_GRID = 20000  # u samples of the oracle's limit-surface root search


def _oracle_grad(case, weights, depth):
    """sum_i w_i dt_i/dtheta per segment, from the oracle's own hits.  The
    adjoint differentiates the closest hit of the limit surface (lateral
    surface closed by the end disks), so each oracle hit at this depth is
    replaced by the limit-surface hit of its segment (oracle.limit_hit), which
    lies within 1e-6 of it in t (rays whose two hits are farther apart are
    left out).  Left out of the check, with zero weight on both sides, are
    grazing hits (incidence cosine below GRAZING against the surface normal;
    the system is near singular) and hits next to the rim between the
    lateral surface and an end disk (lateral u within RIM of 0 or 1, or a
    disk point beyond 1 - RIM of the disk's radius), where dt/dtheta jumps
    and FP32 and FP64 may take different sides."""
    ref = O.closest(case, depth)
    g = np.zeros((case["cps"].shape[0], 4, 4))
    used = np.zeros(len(weights), dtype=bool)
    for i in np.nonzero(ref["seg"] >= 0)[0]:
        s = ref["seg"][i]
        r7 = O.ray7_from_packed(case["rays"][i])
        w = r7[3:6] / np.linalg.norm(r7[3:6])
        cp = case["cps"][s].astype(np.float64)
        kind, tt, uu = O.limit_hit(r7, cp, N_GRID)
        if kind == 0 or abs(tt - ref["t"][i]) > 1e-6:
            continue
        x = r7[:3] + tt * w
        c = I.bezier(cp[None], np.array([uu]))[0]
        if kind == 1:
            if uu < RIM or uu > 1 - RIM:
                continue
            if abs(np.dot(x - c[:3], w)) < GRAZING * c[3]:
                continue
        else:
            n = I.bezier_tangent(cp[None], np.array([uu]))[0][:3]
            if np.linalg.norm(x - c[:3]) > (1 - RIM) * c[3]:
                continue
            if abs(np.dot(n, w)) < GRAZING * np.linalg.norm(n):
                continue
        gi = O.grad_t(r7, cp, tt, uu)
        if gi is None:
            continue
        g[s] += weights[i] * gi
        used[i] = True
    return g, used, ref


@pytest.fixture(scope="module")
def hair_hits():
    case = I.aimed_hair_case(4096)
    w = I.hit_weights(4096)
    g_ref, used, ref = _oracle_grad(case, w, DEPTH)
    return case, w, g_ref, used, ref


def test_backward_matches_oracle_ift(hair_hits):
    case, w, g_ref, used, ref = hair_hits
    fib = F.Fibers(case["cps"])
    tu, seg, _ = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], DEPTH)
    # the oracle's selection of usable hits (lateral, non-singular) decides
    # which rays carry weight, so both sides sum the same terms
    wt = torch.tensor(np.where(used, w, 0.0).astype(np.float32), device="cuda")
    g, skipped = F.intersect_backward(fib, case["rays"], tu, seg, wt)
    g = g.cpu().numpy().astype(np.float64)
    fib.close()
    assert used.sum() > 3500 and int(skipped.item()) == 0
    err = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    worst = np.argsort(-np.linalg.norm((g - g_ref).reshape(len(g), -1), axis=1))[:5]
    assert err < 1e-3, (err, [(int(s), np.round(g[s].ravel(), 4).tolist(), np.round(g_ref[s].ravel(), 4).tolist())
                              for s in worst[:2]])
    # per segment, with an absolute floor of 1e-6 of the largest entry
    floor = 1e-6 * np.abs(g_ref).max()
    per = np.linalg.norm((g - g_ref).reshape(len(g), -1), axis=1) / (
        np.linalg.norm(g_ref.reshape(len(g), -1), axis=1) + floor)
    assert np.quantile(per[np.abs(g_ref).reshape(len(g), -1).max(1) > 0], 0.999) < 1e-2
    assert per.max() < 5e-2


def test_autograd_function_matches_adjoint(hair_hits):
    case, w, g_ref, used, ref = hair_hits
    fib = F.Fibers(case["cps"])
    cps = torch.tensor(case["cps"], device="cuda", requires_grad=True)
    t, u, s = F.fiber_intersect(cps, case["rays"], case["row_ptr"], case["seg_idx"], DEPTH, fib)
    wt = torch.tensor(np.where(used, w, 0.0).astype(np.float32), device="cuda")
    loss = (torch.where(s >= 0, t, torch.zeros_like(t)) * wt).sum()
    loss.backward()
    g = cps.grad.cpu().numpy().astype(np.float64)
    fib.close()
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-3


def test_backward_accumulates_and_skips_misses():
    case = I.aimed_hair_case(512, seed=99)
    fib = F.Fibers(case["cps"])
    tu, seg, _ = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], DEPTH)
    ones = torch.ones(512, device="cuda")
    g1, _ = F.intersect_backward(fib, case["rays"], tu, seg, ones)
    g2 = g1.clone()
    F.intersect_backward(fib, case["rays"], tu, seg, ones, grad_cps=g2)
    np.testing.assert_allclose(g2.cpu().numpy(), 2 * g1.cpu().numpy(), rtol=1e-6, atol=1e-9)
    # a miss contributes nothing
    seg_m = torch.full_like(seg, -1)
    g3, sk = F.intersect_backward(fib, case["rays"], tu, seg_m, ones)
    assert float(g3.abs().max()) == 0.0 and int(sk.item()) == 0
    fib.close()


def test_backward_translation_identity():
    # moving every fiber along a ray by e moves that ray's hit by e: for a
    # single ray, sum_k dt/dp_k . w = 1
    case = I.aimed_hair_case(256, seed=7)
    fib = F.Fibers(case["cps"])
    tu, seg, _ = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], DEPTH)
    seg_np, u_np = seg.cpu().numpy(), tu[:, 1].cpu().numpy()
    rays = torch.tensor(case["rays"], device="cuda")
    checked = 0
    for i in range(256):
        if seg_np[i] < 0:
            continue
        g, sk = F.intersect_backward(fib, rays[i:i + 1], tu[i:i + 1], seg[i:i + 1],
                                     torch.ones(1, device="cuda"))
        if int(sk.item()):
            continue
        gs = g[seg_np[i]].cpu().numpy().astype(np.float64)
        w = case["rays"][i, 4:7].astype(np.float64)
        w /= np.linalg.norm(w)
        assert abs(gs[:, :3].sum(axis=0) @ w - 1.0) < 2e-3
        checked += 1
        if checked >= 40:
            break
    fib.close()
    assert checked >= 30
