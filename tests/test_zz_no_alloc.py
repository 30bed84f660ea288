"""intersect_closest_noalloc (fixed device scratch, no allocation) against
intersect_closest with the one-thread-per-pair kernel, both called through
the C ABI on the same inputs, on two calls in a row with different workloads
so that the second call runs on the keys the first one left behind.  The
file name keeps it last in collection; it passes alone or after the rest."""
import ctypes

import numpy as np
import pytest

from paper_1811_03374_gb300 import fiberx as F
from paper_1811_03374_gb300 import inputs as I
from tests import _parity as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DEPTH = 10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev(case):
    return (torch.tensor(case["rays"], device="cuda"),
            torch.tensor(case["row_ptr"].astype(np.int32), device="cuda"),
            torch.tensor(case["seg_idx"].astype(np.int32), device="cuda"))


def _call_noalloc(fib, rays, row_ptr, seg_idx, depth, flags=0, n_ray=None):
    n = rays.shape[0] if n_ray is None else n_ray
    tu = torch.full((rays.shape[0], 2), float("nan"), device="cuda")
    seg = torch.full((rays.shape[0],), -7, dtype=torch.int32, device="cuda")
    leaf = torch.full((rays.shape[0],), -7, dtype=torch.int32, device="cuda")
    vp = ctypes.c_void_p
    rc = F.lib().intersect_closest_noalloc(
        fib.handle, vp(rays.data_ptr()), n, vp(row_ptr.data_ptr()), vp(seg_idx.data_ptr()),
        seg_idx.numel(), depth, flags, vp(tu.data_ptr()), vp(seg.data_ptr()), vp(leaf.data_ptr()),
        vp(torch.cuda.current_stream().cuda_stream))
    return rc, tu, seg, leaf


def _same(case, got, want):
    tu_g, seg_g = got[1].cpu().numpy(), got[2].cpu().numpy()
    tu_w, seg_w, _ = (x.cpu().numpy() if x is not None else None for x in want)
    assert np.array_equal(seg_g, seg_w)
    hit = seg_w >= 0
    assert hit.sum() > 0
    t_g, t_w = tu_g[hit, 0].astype(np.float64), tu_w[hit, 0].astype(np.float64)
    assert np.all(np.abs(t_g - t_w) <= P.TOL_T * np.abs(t_w))
    tol_u = P.u_tolerance(case, case["rays"][hit], seg_w[hit], t_w, tu_w[hit, 1].astype(np.float64))
    assert np.all(np.abs(tu_g[hit, 1].astype(np.float64) - tu_w[hit, 1]) <= tol_u)
    assert np.all(np.isinf(tu_g[~hit, 0]))


@pytest.mark.parametrize("flags", [0, F.FX_FAST_MATH])
def test_noalloc_matches_intersect_closest_twice(flags):
    first = I.tiny_case()                          # 16384 rays, dense candidates
    second = I.sweep_case("curved", 4096, forced_hits=True)  # fewer rays: reuses stale keys
    for case in (first, second):
        fib = F.Fibers(case["cps"])
        rays, row_ptr, seg_idx = _dev(case)
        want = F.intersect_closest(fib, rays, row_ptr, seg_idx, DEPTH, flags | F.FX_KERNEL_NAIVE)
        got = _call_noalloc(fib, rays, row_ptr, seg_idx, DEPTH, flags)
        torch.cuda.synchronize()
        assert got[0] == F.FX_OK, F.lib().fx_last_error().decode()
        _same(case, got, want)
        fib.close()


def test_noalloc_rejects_more_rays_than_the_array_holds():
    case = I.tiny_case(n_ray=64)
    fib = F.Fibers(case["cps"])
    rays, row_ptr, seg_idx = _dev(case)
    rc, *_ = _call_noalloc(fib, rays, row_ptr, seg_idx, DEPTH, n_ray=F.NOALLOC_MAX_RAYS + 1)
    assert rc == -1
    assert "FX_NOALLOC_MAX_RAYS" in F.lib().fx_last_error().decode()
    # a call within the limit still works after the refusal
    rc, tu, seg, _ = _call_noalloc(fib, rays, row_ptr, seg_idx, DEPTH)
    torch.cuda.synchronize()
    assert rc == F.FX_OK
    fib.close()
