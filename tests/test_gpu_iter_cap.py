"""The runaway guard: every (ray, piece) test stops after iter_cap(depth)
node tests and reports FX_DEV_ITER_LIMIT.  A library built with a cap of 6
node tests (compile-time FX_ITER_CAP_BASE / FX_ITER_CAP_PER_LEVEL) runs in a
child process: its calls return, the status word has the bit, the per-pair
status bytes mark exactly the capped pairs, and every pair or ray the cap
did not touch equals the normal library's result -- the guard trips without
a fault, a hang or a trap."""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_1811_03374_gb300 import fiberx as F
from paper_1811_03374_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CAP = 6
DEPTH = 12

CHILD = textwrap.dedent("""
    import json, sys
    import numpy as np
    sys.path.insert(0, %(root)r)
    from paper_1811_03374_gb300 import fiberx as F
    from paper_1811_03374_gb300 import inputs as I
    case = I.sweep_case("moderate", 4096, forced_hits=True)
    out = {}
    for name, variant, kernel in %(paths)r:
        fib = F.Fibers(case["cps"])
        fib.set_launch(variant=variant)
        tup, _, pf = F.intersect_pairs(fib, case["rays"], case["row_ptr"], case["seg_idx"], %(depth)d, kernel,
                                       pair_flags=True)
        st_pairs = fib.status()
        tu, seg, leaf = F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"], %(depth)d, kernel)
        st_closest = fib.status()
        fib.close()
        np.savez(%(out)r + "_" + name + ".npz", tup=tup.cpu().numpy(), pf=pf.cpu().numpy(), tu=tu.cpu().numpy(),
                 seg=seg.cpu().numpy())
        out[name] = [st_pairs, st_closest]
    print(json.dumps(out))
""")

PATHS = [("lane", F.FX_VARIANT_LANE, 0), ("scan", F.FX_VARIANT_SCAN, 0), ("ray", F.FX_VARIANT_RAY, 0),
         ("warp", F.FX_VARIANT_WARP, 0), ("naive", 0, F.FX_KERNEL_NAIVE)]


@pytest.fixture(scope="module")
def capped(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_03374_gb300.csrc import build as B
    d = tmp_path_factory.mktemp("iter_cap")
    lib = str(d / "libfiberx_cap.so")
    B.build(extra=["-DFX_ITER_CAP_BASE=%d" % CAP, "-DFX_ITER_CAP_PER_LEVEL=0"], out=lib, obj_dir=str(d / "obj"))
    prefix = str(d / "res")
    code = CHILD % dict(root=ROOT, paths=PATHS, depth=DEPTH, out=prefix)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, FIBERX_LIB=lib))
    assert r.returncode == 0, r.stderr[-2000:]
    status = json.loads(r.stdout.strip().splitlines()[-1])
    return prefix, status


@pytest.mark.parametrize("name,variant,kernel", PATHS, ids=[p[0] for p in PATHS])
def test_capped_tests_are_reported_and_the_rest_unchanged(capped, name, variant, kernel):
    prefix, status = capped
    res = np.load(prefix + "_" + name + ".npz")
    st_pairs, st_closest = status[name]
    assert st_pairs & F.FX_DEV_ITER_LIMIT and st_closest & F.FX_DEV_ITER_LIMIT
    case = I.sweep_case("moderate", 4096, forced_hits=True)
    fib = F.Fibers(case["cps"])
    fib.set_launch(variant=variant)
    tup, _, pf = (x.cpu().numpy() for x in F.intersect_pairs(fib, case["rays"], case["row_ptr"], case["seg_idx"],
                                                           DEPTH, kernel, pair_flags=True))
    tu, seg, _ = (x.cpu().numpy() for x in F.intersect_closest(fib, case["rays"], case["row_ptr"], case["seg_idx"],
                                                             DEPTH, kernel))
    assert fib.status() == 0
    fib.close()
    assert not pf.any()
    capped_pairs = (res["pf"] & F.FX_DEV_ITER_LIMIT) != 0
    # a forced hit at depth 12 takes at least 13 node tests: most pairs trip the cap
    assert capped_pairs.mean() > 0.5
    assert np.all(res["pf"][~capped_pairs] == 0)
    np.testing.assert_array_equal(res["tup"][~capped_pairs], tup[~capped_pairs])
    # one candidate per ray: a ray whose only pair was not capped is unchanged
    np.testing.assert_array_equal(res["tu"][~capped_pairs], tu[~capped_pairs])
    np.testing.assert_array_equal(res["seg"][~capped_pairs], seg[~capped_pairs])
    # a capped test reports no hit of its own
    assert np.all(np.isinf(res["tup"][capped_pairs, 0]))
