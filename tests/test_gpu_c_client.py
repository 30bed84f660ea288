"""The C ABI from plain C: tests/c_client.c, compiled with gcc against
include/fiberx.h, the in-tree libfiberx.so and the CUDA runtime, uploads
fibers (cubic or quadratic) from host memory and runs intersect_closest,
intersect_pairs (with per-pair status bytes) and intersect_backward on device
buffers it allocates itself.  Its results equal the Python binding's, bit for
bit where each output element has one contributor, and its quadratic-fiber
gradient matches FP64 central finite differences."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1811_03374_gb300 import fiberx as F
from paper_1811_03374_gb300 import inputs as I
from tests import _grad as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = F.library_path()
    F.lib()  # built and loadable
    exe = str(tmp_path_factory.mktemp("c_client") / "c_client")
    subprocess.run([cc, "-std=c99", "-O2", os.path.join(HERE, "c_client.c"), "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(CUDA, "include"), "-L", os.path.dirname(lib), "-lfiberx",
                    "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.dirname(lib),
                    "-Wl,-rpath," + os.path.join(CUDA, "lib64"), "-o", exe], check=True)
    return exe


def _run(exe, tmp_path, case, depth, flags, variant):
    cps = np.ascontiguousarray(case["cps"], np.float32)
    rays = np.ascontiguousarray(case["rays"], np.float32)
    rp = np.ascontiguousarray(case["row_ptr"], np.int32)
    si = np.ascontiguousarray(case["seg_idx"], np.int32)
    n_seg, n_ray, n_pair, n_cp = cps.shape[0], rays.shape[0], si.size, cps.shape[1]
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(fin, "wb") as f:
        f.write(np.array([n_seg, n_ray, n_pair, n_cp], np.int64).tobytes())
        for a in (cps, rays, rp, si):
            f.write(a.tobytes())
    r = subprocess.run([exe, fin, fout, str(depth), str(flags), str(variant)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    raw = open(fout, "rb").read()
    off = 0

    def take(dtype, count):
        nonlocal off
        a = np.frombuffer(raw, dtype, count, off)
        off += a.nbytes
        return a

    tu = take(np.float32, 2 * n_ray).reshape(n_ray, 2)
    seg = take(np.int32, n_ray)
    leaf = take(np.int32, n_ray)
    tup = take(np.float32, 2 * n_pair).reshape(n_pair, 2)
    pf = take(np.uint8, n_pair)
    status = int(take(np.uint32, 1)[0])
    grad = take(np.float32, n_seg * n_cp * 4).reshape(n_seg, n_cp, 4)
    assert off == len(raw)
    return tu, seg, leaf, tup, pf, status, grad


@pytest.mark.parametrize("workload", ["tiny", "sweep"])
@pytest.mark.parametrize("variant,flags", [(F.FX_VARIANT_AUTO, 0), (F.FX_VARIANT_SCAN, F.FX_FAST_MATH),
                                           (F.FX_VARIANT_LANE, F.FX_POLISH_FP64)],
                         ids=["auto", "scan-fast", "lane-polish"])
def test_c_client_equals_python_binding(client, tmp_path, workload, variant, flags):
    case = I.tiny_case() if workload == "tiny" else I.sweep_case("moderate", 8192, forced_hits=True)
    depth = 8 if workload == "tiny" else 14
    tu, seg, leaf, tup, pf, status, grad = _run(client, tmp_path, case, depth, flags, variant)
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    ref = [x.cpu().numpy() for x in F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], depth,
                                                         flags)]
    tup_r, _, pf_r = (x.cpu().numpy() for x in F.intersect_pairs(
        fib, case["rays"], case["row_ptr"], case["seg_idx"], depth, flags & ~F.FX_POLISH_FP64, pair_flags=True))
    g_r, _ = F.intersect_backward(fib, case["rays"], torch.from_numpy(ref[0]), torch.from_numpy(ref[1]),
                                  torch.ones(len(ref[1])))
    st_r = fib.status()
    fib.close()
    # atomics add a segment's contributions in no fixed order
    np.testing.assert_allclose(grad, g_r.cpu().numpy(), rtol=1e-5, atol=1e-6 * np.abs(grad).max())
    np.testing.assert_array_equal(tu, ref[0])
    np.testing.assert_array_equal(seg, ref[1])
    np.testing.assert_array_equal(leaf, ref[2])
    np.testing.assert_array_equal(tup, tup_r)
    np.testing.assert_array_equal(pf, pf_r)
    assert status == st_r and status & ~F.FX_DEV_UNSUPPORTED == 0
    assert (seg >= 0).sum() > 1000


def test_c_client_quadratic_gradient(client, tmp_path):
    # quadratic fibers through the plain C caller: upload, closest hit and
    # the adjoint with respect to p0..p2, which equals the Python binding's
    # bit for bit (one ray per segment) and FP64 central finite differences
    case = I.quadratic_case("moderate", 64, seed=77, forced_hits=True)
    tu, seg, leaf, tup, pf, status, grad = _run(client, tmp_path, case, 16, 0, F.FX_VARIANT_AUTO)
    assert grad.shape == (64, 3, 4) and status & ~F.FX_DEV_UNSUPPORTED == 0
    fib = F.Fibers(case["cps"])
    tu_r, seg_r, _ = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], 16)
    g_r, _ = F.intersect_backward(fib, case["rays"], tu_r, seg_r, torch.ones(64))
    fib.close()
    np.testing.assert_array_equal(tu, tu_r.cpu().numpy())
    np.testing.assert_array_equal(grad, g_r.cpu().numpy())
    t = tu[:, 0].astype(np.float64)
    t[seg < 0] = np.inf
    G.check_quadratic_gradient(case, t, grad.astype(np.float64))
