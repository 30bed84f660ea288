"""Finite-difference check of quadratic-fiber gradients: t of the
limit-surface hit (the oracle's FP64 root search on the degree-raised curve)
as a function of the quadratic control points, differentiated by FP64
central differences (h = 1e-6), against a gradient the CUDA adjoint
returned.  Shared by the tests that reach the adjoint through the autograd
Function and through the plain C caller."""
import numpy as np

import oracle as O
from paper_1811_03374_gb300 import inputs as I


def check_quadratic_gradient(case, t, g, min_checked=25, h=1e-6, tol=1e-3):
    """case: one ray per quadratic segment (ray i aims at segment i); t: the
    forward t per ray (inf on a miss); g: [n_seg, 3, 4] dL/d(cps) for
    L = sum of the hit t.  Returns the number of hits checked; only
    well-inside lateral, non-grazing hits are (dt/dtheta jumps at the rim and
    is singular for grazing rays)."""
    checked = 0
    for i in np.nonzero(np.isfinite(t))[0]:
        r7 = O.ray7_from_packed(case["rays"][i])
        q = case["cps"][i].astype(np.float64)
        c = O.elevate_quadratics(q[None])[0]
        kind, t0, u0 = O.limit_hit(r7, c, 20000)
        if kind != 1 or abs(t0 - t[i]) > 1e-4 * t0 or not (0.01 < u0 < 0.99):
            continue
        w = r7[3:6] / np.linalg.norm(r7[3:6])
        x = r7[:3] + t0 * w
        cu = I.bezier(c[None], np.array([u0]))[0]
        if abs(np.dot(x - cu[:3], w)) < 0.05 * cu[3]:
            continue
        fd = np.zeros((3, 4))
        ok = True
        for k in range(3):
            for a in range(4):
                tt = []
                for sgn in (1, -1):
                    qq = q.copy()
                    qq[k, a] += sgn * h
                    kd, ti, _ = O.limit_hit(r7, O.elevate_quadratics(qq[None])[0], 20000)
                    ok = ok and kd == kind
                    tt.append(ti)
                fd[k, a] = (tt[0] - tt[1]) / (2 * h)
        if not ok:
            continue
        err = np.linalg.norm(g[i] - fd) / np.linalg.norm(fd)
        assert err < tol, (i, err, np.round(g[i], 5).tolist(), np.round(fd, 5).tolist())
        checked += 1
    assert checked >= min_checked, checked
    return checked
