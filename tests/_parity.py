"""Element-wise comparison of the CUDA path with the FP64 oracle.

A ray passes when hit/miss agree and, for hits, the segment is the same,
|t - t_ref| <= TOL_T * t_ref and |u - u_ref| <= tol_u (the stated tolerance:
relative t error <= 1e-5, |u error| <= 1e-5).  tol_u is 1e-5 unless FP32
cannot resolve it: a hit point carries an error of a few units in the last
place of the distances involved, 8 * 2^-24 * (|o| + t) along the ray, which
in the curve's parameter is that length over the parametric speed |c'(u)|;
tol_u = max(1e-5, 8 * 2^-24 * (|o| + t) / |c'(u)|).  For short fibers seen
from afar (the hair patch: 0.02-long segments four units away) this is
about 2e-5; for the tiny and depth-sweep workloads it stays 1e-5.

Rays that fail this strict rule are re-run through the oracle with the ray
shifted sideways (8 directions orthogonal to it) by the resolution band
    delta = 1e-4 r + 8 * 2^-24 * (|o| + t):
1e-4 r is the silhouette band within which hit/miss may differ, the second
term is the spacing of FP32 coordinates along the ray, below which no FP32
computation can resolve a decision (a silhouette, a split plane, an end
plane) or place a hit (for a ray nearly parallel to a fiber a sideways
error e moves the hit along the fiber by e / tan(angle)).  A ray passes "in
band" if the oracle result of one shifted copy (shifts of delta * 2^-k,
k = 0..16, in 8 directions; the shifted rays are passed in double precision)
meets the strict rule.  The small shifts matter far from the origin: there
the difference of a control point and a ray origin is exact in FP32 and the
decisions are resolved far below the |o| term of delta, yet a ray nearly
parallel to a fiber still moves its hit along the fiber by (its sideways
error) / tan(angle).

Finally a ray is exempt ("silhouette") if it passes within 1e-4 r of the
silhouette of the leaf cylinder hit by either side: |dist(ray, leaf axis) -
r_leaf| < 1e-4 r_leaf, measured in FP64 between the ray line and the leaf's
axis line.  There the hit is ill-conditioned (grazing) and hit/miss, t and u
may all legitimately differ.  Every other ray is a failure.
"""
import json
import os

import numpy as np

import oracle as O

TOL_T = 1e-5
P_TOL_T = TOL_T
TOL_U = 1e-5
EPS32 = 2.0 ** -24


def u_tolerance(case, rays, seg, t, u):
    """Per-ray |u| tolerance (see module docstring)."""
    tol = np.full(len(seg), TOL_U)
    hit = (seg >= 0) & np.isfinite(t)
    if hit.any():
        cp = case["cps"][seg[hit]].astype(np.float64)
        uu = np.clip(u[hit], 0, 1)[:, None]
        v = 1 - uu
        d = 3 * (v * v * (cp[:, 1, :3] - cp[:, 0, :3]) + 2 * uu * v * (cp[:, 2, :3] - cp[:, 1, :3])
                 + uu * uu * (cp[:, 3, :3] - cp[:, 2, :3]))
        speed = np.linalg.norm(d, axis=1)
        o = np.linalg.norm(rays[hit, :3].astype(np.float64), axis=1)
        res = 8 * EPS32 * (o + t[hit]) / np.maximum(speed, 1e-30)
        tol[hit] = np.maximum(TOL_U, res)
    return tol


def strict_ok(t_g, u_g, s_g, t_o, u_o, s_o, tol_u=TOL_U):
    hit_g, hit_o = s_g >= 0, s_o >= 0
    ok = hit_g == hit_o
    both = hit_g & hit_o
    with np.errstate(invalid="ignore"):
        vals = (s_g == s_o) & (np.abs(t_g - t_o) <= TOL_T * np.abs(t_o)) & (np.abs(u_g - u_o) <= tol_u)
    return ok & (~both | vals)


def _radius_at(cps, seg, u):
    cp = cps[seg].astype(np.float64)
    u = np.clip(u, 0, 1)[:, None]
    v = 1 - u
    B = np.concatenate([v ** 3, 3 * u * v * v, 3 * u * u * v, u ** 3], axis=1)
    return np.sum(B * cp[:, :, 3], axis=1)


def _perp(w):
    a = np.where(np.abs(w[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0.0, 1, 0]]))
    e1 = a - np.sum(a * w, axis=1, keepdims=True) * w
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(w, e1)
    return e1, e2


SCALES = tuple(2.0 ** -k for k in range(17))


def band_check(case, idx, t_g, u_g, s_g, depth, pieces, mode="closest"):
    """Indices (subset of idx) whose GPU result the oracle reproduces for a
    sideways-shifted copy of the ray: shifts of delta * 2^-k (k = 0..16) in
    8 directions orthogonal to the ray.  Near a silhouette the result moves
    like the square root of the shift, so several magnitudes are tried."""
    if len(idx) == 0:
        return np.zeros(0, dtype=np.int64)
    rays = case["rays"][idx].astype(np.float64)
    o, w = rays[:, :3], rays[:, 4:7]
    w = w / np.linalg.norm(w, axis=1, keepdims=True)
    t_ref = np.where(np.isfinite(t_g[idx]), t_g[idx], 0.0)
    seg = np.where(s_g[idx] >= 0, s_g[idx], 0)
    r = _radius_at(case["cps"], seg, u_g[idx])
    r = np.where(s_g[idx] >= 0, r, case["cps"][:, :, 3].max())
    delta = 1e-4 * r + 8 * EPS32 * (np.linalg.norm(o, axis=1) + t_ref)
    e1, e2 = _perp(w)
    dirs = [e1, -e1, e2, -e2, (e1 + e2) / np.sqrt(2), (e1 - e2) / np.sqrt(2),
            (-e1 + e2) / np.sqrt(2), (-e1 - e2) / np.sqrt(2)]
    shifts = [sc * dv for sc in SCALES for dv in dirs]
    rp = case["row_ptr"].astype(np.int64)
    cand = [case["seg_idx"][rp[i]:rp[i + 1]] for i in idx]
    tmax = rays[:, 3]
    sub_rays, rows, segs = [], [0], []
    for sh in shifts:
        # double-precision rays: shifts far below an FP32 step of |o| stay exact
        sub_rays.append(np.concatenate([o + delta[:, None] * sh, w, tmax[:, None]], axis=1))
        for c in cand:
            segs.append(c)
            rows.append(rows[-1] + len(c))
    ref = O.closest_d(np.concatenate(sub_rays), np.array(rows, dtype=np.int32),
                      np.concatenate(segs).astype(np.int32) if segs else np.zeros(0, np.int32),
                      depth, pieces)
    m = len(idx)
    tol_u = u_tolerance(case, case["rays"][idx], s_g[idx], t_g[idx], u_g[idx])
    ok = np.zeros(m, dtype=bool)
    for k in range(len(shifts)):
        sl = slice(k * m, (k + 1) * m)
        ok |= strict_ok(t_g[idx], u_g[idx], s_g[idx], ref["t"][sl], ref["u"][sl], ref["seg"][sl], tol_u)
    return idx[ok]


def silhouette_dist(case, i, seg, leaf, depth):
    """|dist(ray line, leaf axis line) - r_leaf| / r_leaf for the leaf of
    segment `seg` starting at `leaf` (units of 2^-23), FP64."""
    if seg < 0 or leaf < 0:
        return np.inf
    cp = case["cps"][seg].astype(np.float64)
    size = O.ROOT_SIZE >> min(depth, 23)
    start = (int(leaf) // size) * size
    node = O.node_at(cp, start, size)
    r_leaf = O.cons_radius(node)
    ray = case["rays"][i].astype(np.float64)
    o, w = ray[:3], ray[4:7] / np.linalg.norm(ray[4:7])
    p, d = node[0, :3], node[1, :3]
    n = np.cross(w, d)
    if np.linalg.norm(n) == 0:
        dist = np.linalg.norm(np.cross(p - o, w))
    else:
        dist = abs(np.dot(p - o, n)) / np.linalg.norm(n)
    return abs(dist - r_leaf) / r_leaf


def compare_closest(case, depth, gpu_tu, gpu_seg, ref, pieces, gpu_leaf=None):
    """Returns a stats dict; 'fail' lists ray indices failing strict and band."""
    t_g = gpu_tu[:, 0].astype(np.float64)
    u_g = gpu_tu[:, 1].astype(np.float64)
    s_g = gpu_seg.astype(np.int64)
    tol_u = u_tolerance(case, case["rays"], ref["seg"].astype(np.int64), ref["t"], ref["u"])
    ok = strict_ok(t_g, u_g, s_g, ref["t"], ref["u"], ref["seg"].astype(np.int64), tol_u)
    bad = np.nonzero(~ok)[0]
    banded = band_check(case, bad, t_g, u_g, s_g, depth, pieces)
    rest = np.setdiff1d(bad, banded)
    sil = []
    for i in rest:
        ds = silhouette_dist(case, i, int(ref["seg"][i]), int(ref["leaf"][i]), depth) \
            if "leaf" in ref else np.inf
        if gpu_leaf is not None:
            ds = min(ds, silhouette_dist(case, i, int(s_g[i]), int(gpu_leaf[i]), depth))
        if ds < 1e-4:
            sil.append(i)
    sil = np.array(sil, dtype=np.int64)
    fail = np.setdiff1d(rest, sil)
    both = (s_g >= 0) & (ref["seg"] >= 0) & ok
    rel = np.abs(t_g[both] - ref["t"][both]) / ref["t"][both] if both.any() else np.zeros(1)
    du = np.abs(u_g[both] - ref["u"][both]) if both.any() else np.zeros(1)
    du_rel = du / tol_u[both] if both.any() else np.zeros(1)
    detail = [dict(i=int(i), gpu=(float(t_g[i]), float(u_g[i]), int(s_g[i])),
                   ref=(float(ref["t"][i]), float(ref["u"][i]), int(ref["seg"][i])), tol_u=float(tol_u[i]))
              for i in fail[:6]]
    return dict(n=len(s_g), hits=int((ref["seg"] >= 0).sum()), strict=int(ok.sum()),
                band=int(len(banded)), silhouette=int(len(sil)), fail=fail, max_rel_t=float(rel.max()), max_du=float(du.max()),
                max_du_over_tol=float(du_rel.max()), med_rel_t=float(np.median(rel)), detail=detail)


def pairs_min(pr, case):
    """Closest per ray from per-pair oracle hits (ties: earlier candidate)."""
    rp = case["row_ptr"].astype(np.int64)
    n = len(rp) - 1
    t = np.full(n, np.inf)
    u = np.full(n, -1.0)
    s = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        a, b = rp[i], rp[i + 1]
        if b > a:
            j = a + int(np.argmin(pr["t"][a:b]))
            if np.isfinite(pr["t"][j]):
                t[i], u[i], s[i] = pr["t"][j], pr["u"][j], case["seg_idx"][j]
    return dict(t=t, u=u, seg=s)


def report(rec):
    """Appends one JSON line to the file named by FX_REPORT, if set (the
    figures a run measured)."""
    path = os.environ.get("FX_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")
