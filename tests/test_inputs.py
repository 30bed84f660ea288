"""Seeded workload generators: determinism, layouts and the stated shapes."""
import numpy as np

from paper_1811_03374_gb300 import inputs as I


def test_tiny_case_layout_and_determinism():
    a, b = I.tiny_case(), I.tiny_case()
    assert a["cps"].shape == (16, 4, 4) and a["cps"].dtype == np.float32
    assert a["rays"].shape == (16384, 8) and a["rays"].dtype == np.float32
    assert len(a["seg_idx"]) == 262144 and a["row_ptr"][-1] == 262144
    for k in a:
        if isinstance(a[k], np.ndarray):
            np.testing.assert_array_equal(a[k], b[k])
    pts, rad = a["cps"][:, :, :3], a["cps"][:, :, 3]
    assert pts.min() >= -1 and pts.max() <= 1 and rad.min() >= 0.01 and rad.max() <= 0.05
    o = a["rays"][:, :3].astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(o, axis=1), 5.0, rtol=1e-6)
    np.testing.assert_allclose(np.linalg.norm(a["rays"][:, 4:7], axis=1), 1.0, rtol=1e-6)


def test_hair_fibers_shape_chain_and_taper():
    cps = I.hair_fibers(n_fibers=200).astype(np.float64).reshape(200, 8, 4, 4)
    # C0 and C1 continuity along each fiber
    np.testing.assert_allclose(cps[:, 1:, 0], cps[:, :-1, 3], atol=1e-6)
    np.testing.assert_allclose(cps[:, 1:, 1, :3] - cps[:, 1:, 0, :3],
                               cps[:, :-1, 3, :3] - cps[:, :-1, 2, :3], atol=1e-6)
    assert abs(cps[:, 0, 0, 3].max() - 0.002) < 1e-7 and abs(cps[:, -1, 3, 3].min() - 0.0005) < 1e-7
    steps = np.linalg.norm(cps[:, :, 3, :3] - cps[:, :, 0, :3], axis=-1)
    np.testing.assert_allclose(steps, 0.02, rtol=1e-4)
    assert np.all(cps[:, 0, 0, 2] == 0) and cps[:, 0, 0, :2].min() >= 0 and cps[:, 0, 0, :2].max() <= 1


def test_grid_cull_is_conservative_and_deduplicated():
    # every segment whose dilated AABB a ray crosses must be listed
    cps = I.hair_fibers(n_fibers=300)
    rays, _ = I.pinhole_rays(width=64, height=36)
    rp, si = I.grid_cull(cps, rays, (20, 20, 8))
    assert rp[0] == 0 and rp[-1] == len(si)
    c = cps.astype(np.float64)
    rmax = c[:, :, 3].max(1, keepdims=True)
    lo, hi = c[:, :, :3].min(1) - rmax, c[:, :, :3].max(1) + rmax
    for i in range(0, len(rays), 7):
        row = si[rp[i]:rp[i + 1]]
        assert len(np.unique(row)) == len(row)
        o, w = rays[i, :3].astype(np.float64), rays[i, 4:7].astype(np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            ta, tb = (lo - o) / w, (hi - o) / w
        t0 = np.nanmax(np.minimum(ta, tb), axis=1)
        t1 = np.nanmin(np.maximum(ta, tb), axis=1)
        crossed = np.nonzero((t0 <= t1) & (t1 >= 0))[0]
        assert set(crossed.tolist()) <= set(row.tolist())


def test_sweep_and_stress_cases():
    for k in I.SWEEP_JITTER:
        c = I.sweep_case(k, 1000)
        assert c["cps"].shape == (1000, 4, 4) and c["rays"].shape == (1000, 8)
        L = np.linalg.norm(c["cps"][:, 3, :3].astype(np.float64) - c["cps"][:, 0, :3], axis=1)
        np.testing.assert_allclose(L, 1.0, rtol=1e-5)
    g = I.grazing_case(100)
    assert np.abs(g["delta"]).max() <= 1e-3
    o = I.offset_case(100, 1e4)
    assert np.abs(o["cps"][:, :, :3]).min() > 5e3


def test_single_fiber_case():
    for k in I.SWEEP_JITTER:
        c = I.single_fiber_case(k, 1000)
        assert c["cps"].shape == (1, 4, 4) and c["rays"].shape == (1000, 8)
        assert np.all(c["seg_idx"] == 0) and c["row_ptr"][-1] == 1000
        w = c["rays"][:, 4:7].astype(np.float64)
        np.testing.assert_allclose(np.linalg.norm(w, axis=1), 1.0, rtol=1e-6)


def test_quadratic_case():
    for k in I.SWEEP_JITTER:
        c = I.quadratic_case(k, 500, forced_hits=True)
        assert c["cps"].shape == (500, 3, 4) and c["rays"].shape == (500, 8)
        L = np.linalg.norm(c["cps"][:, 2, :3].astype(np.float64) - c["cps"][:, 0, :3], axis=1)
        np.testing.assert_allclose(L, 1.0, rtol=1e-5)
