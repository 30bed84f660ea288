"""intersect_closest_noalloc (fixed device scratch, no allocation) against
intersect_closest with the one-thread-per-pair kernel, both called through
the C ABI on the same inputs, on two calls in a row with different workloads
so that the second call runs on the keys the first one left behind.  Both run
the same kernels, so their results must be identical bit for bit, with each
flag the entry accepts (approximate math, the FP64 polish, index checks with
counters).  The file name keeps it last in collection; it passes alone or
after the rest."""
import ctypes

import numpy as np
import pytest

from paper_1811_03374_gb300 import fiberx as F
from paper_1811_03374_gb300 import inputs as I

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


def _same(got, want):
    # both run the same one-thread-per-pair kernels on the same inputs: the
    # results are identical bit for bit
    for g, w in zip(got[1:], want):
        np.testing.assert_array_equal(g.cpu().numpy(), w.cpu().numpy())
    assert (want[1].cpu().numpy() >= 0).sum() > 0


FLAGS = [0, F.FX_FAST_MATH, F.FX_POLISH_FP64, F.FX_CHECK_INDEX | F.FX_COUNT]


@pytest.mark.parametrize("flags", FLAGS, ids=["ieee", "fast", "polish", "check_count"])
def test_noalloc_matches_intersect_closest_twice(flags):
    first = I.tiny_case()                          # 16384 rays, dense candidates
    second = I.sweep_case("curved", 4096, forced_hits=True)  # fewer rays: reuses stale keys
    for case in (first, second):
        fib = F.Fibers(case["cps"])
        rays, row_ptr, seg_idx = _dev(case)
        fib.counters(reset=True)
        want = F.intersect_closest(fib, rays, row_ptr, seg_idx, DEPTH, flags | F.FX_KERNEL_NAIVE)
        c_want = fib.counters(reset=True)
        got = _call_noalloc(fib, rays, row_ptr, seg_idx, DEPTH, flags)
        torch.cuda.synchronize()
        assert got[0] == F.FX_OK, F.lib().fx_last_error().decode()
        c_got = fib.counters(reset=True)
        _same(got, want)
        if flags & F.FX_COUNT:
            assert c_got == c_want and c_got["nodes"] > 0
        assert fib.status() & ~F.FX_DEV_UNSUPPORTED == 0
        fib.close()


def test_noalloc_polish_needs_the_leaf_output():
    case = I.tiny_case(n_ray=64)
    fib = F.Fibers(case["cps"])
    rays, row_ptr, seg_idx = _dev(case)
    tu = torch.zeros((64, 2), device="cuda")
    seg = torch.zeros(64, dtype=torch.int32, device="cuda")
    vp = ctypes.c_void_p
    rc = F.lib().intersect_closest_noalloc(
        fib.handle, vp(rays.data_ptr()), 64, vp(row_ptr.data_ptr()), vp(seg_idx.data_ptr()),
        seg_idx.numel(), DEPTH, F.FX_POLISH_FP64, vp(tu.data_ptr()), vp(seg.data_ptr()), None,
        vp(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert "leaf" in F.lib().fx_last_error().decode()
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
