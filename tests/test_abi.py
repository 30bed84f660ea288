"""The C ABI library builds, loads and exports every function include/fiberx.h
declares; host-side argument checks answer with the documented codes without
touching a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1811_03374_gb300 import fiberx as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fiberx.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_binding_exports():
    assert sorted(F.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol():
    L = F.lib()
    assert os.path.dirname(F.library_path()).startswith(ROOT)
    for name in declared_functions():
        assert hasattr(L, name), name
    assert L.fx_version() == 10000


def test_argument_errors_without_device():
    L = F.lib()
    h = ctypes.c_void_p()
    # negative segment count and null output are rejected before any CUDA call
    assert L.fiber_upload(None, -1, 0, None, None, ctypes.byref(h)) == -1
    assert L.fiber_upload(None, 1, 0, None, None, None) == -1
    assert L.fiber_upload(None, 4, 0, None, None, ctypes.byref(h)) == -1
    opts = F.UploadOpts(9, 1)
    assert L.fiber_upload(None, 0, 0, ctypes.byref(opts), None, ctypes.byref(h)) == -1
    # null handle
    assert L.intersect_closest(None, None, 0, None, None, 0, 8, None, 0, None, None, None, None) == -1
    assert L.intersect_pairs(None, None, 0, None, None, 0, 8, None, 0, None, None, None, None) == -1
    assert L.intersect_normals(None, None, 0, None, None, None, 8, None, 0, None, None) == -1
    assert L.intersect_closest_host(None, None, 0, None, None, 0, 8, None, 0, None, None, None, None) == -1
    assert L.intersect_backward(None, None, 0, None, None, None, None, None, None) == -1
    assert L.fiber_info(None, None) == -1
    assert L.fx_stream_status(None, None, None) == -1
    assert b"null" in L.fx_last_error()
    ms, tf = ctypes.c_float(), ctypes.c_double()
    assert L.fx_fma_peak(4, 16, None, None, None) == -1
    assert L.fx_fma_peak(0, 16, ctypes.byref(ms), ctypes.byref(tf), None) == -1
    assert L.fx_fma_peak(4, 0, ctypes.byref(ms), ctypes.byref(tf), None) == -1
    L.fiber_free(None)  # no-op


def test_python_binding_has_no_cpu_fallback():
    # without a CUDA device the binding must fail loudly, never compute
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1811_03374_gb300 import inputs
    case = inputs.tiny_case(n_ray=4)
    with pytest.raises(Exception):
        F.Fibers(case["cps"])


def test_product_never_loads_the_oracle():
    # the package and its C sources share nothing with oracle/: no import,
    # no include, no link (only tests, smoke() and bench.py's CPU legs use it)
    pkg = os.path.join(ROOT, "paper_1811_03374_gb300")
    for dirpath, _, files in os.walk(pkg):
        for name in files:
            if not name.endswith((".py", ".cu", ".cuh", ".cpp", ".h", ".c")):
                continue
            src = open(os.path.join(dirpath, name), encoding="utf-8").read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), name
            assert "fiber_oracle" not in src and "oracle/" not in src, name


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header compiles as strict C99 on its own
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text('#include "fiberx.h"\nint main(void) { return fx_version() > 0 ? 0 : 1; }\n')
    r = subprocess.run([cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_depends_on_no_framework():
    # the shared library stands alone: the CUDA runtime is linked in, and it
    # needs no PyTorch, Python or other framework library to load
    import shutil
    import subprocess
    if shutil.which("readelf") is None:
        pytest.skip("no readelf")
    F.lib()
    out = subprocess.run(["readelf", "-d", F.library_path()], capture_output=True, text=True).stdout
    needed = re.findall(r"\(NEEDED\)\s+Shared library: \[([^\]]+)\]", out)
    assert needed
    for lib_name in needed:
        assert not re.search(r"torch|c10|python|triton", lib_name), lib_name
