"""Element-wise comparison of the CUDA path with the FP64 oracle.

A result (one ray's closest hit, or one pair's hit) passes STRICT when
hit/miss agree and, for hits, the segment is the same,
|t - t_ref| <= TOL_T * t_ref and |u - u_ref| <= tol_u (the stated tolerance:
relative t error <= 1e-5, |u error| <= 1e-5).

FP32 resolution.  Every decision the kernels take (a cylinder's silhouette,
a split plane, an end plane) is taken on ray-frame coordinates
x = R (p - o) of points p of the segment, with R the ray's orthonormal
frame.  Let T be the largest distance |p_k - o| of the segment's control
points from the ray origin (FP64), and u = 2^-24.  The FP32 kernels form
these coordinates with the following worst-case errors (IEEE operations
round to nearest, relative error <= u each; the approximate forms of
FX_FAST_MATH stay within 2.3u where they are used):
  - p - o: one rounding of each component, <= u T;
  - the direction w, normalised by 1 / sqrt(w.w): the common factor only
    scales w (|w| = 1 + eta, |eta| <= 3.5u); the rounding of each product
    turns it by at most u, i.e. <= u T sideways at distance T;
  - the frame of Duff et al. built from that w: e1 and e2 carry absolute
    errors <= 5.4u per vector (a = -1 / (s + w_z) <= 2u relative,
    b = w_x w_y a <= 4u, 1 + s w_x^2 a <= 5u), and the construction is
    orthogonal to w only up to 2 |eta| <= 7u: together <= 12.4u T sideways;
  - the rotation, three products summed by two FMAs: <= 3u T per coordinate;
  - the plane tests (split and end planes) add a dot product of the plane
    normal with a point at distance <= T, <= 3u T of offset, and the split
    point p + dp adds one rounding of p_z, <= u T.
So a decision is the exact decision for a ray displaced sideways by at most
    K_FRAME * u * T,  K_FRAME = 22 (1 + 1 + 12.4 + 3 + 3 + 1, rounded up);
subdivision adds errors relative to the node's own size, far below this.
The parameter u of a hit inherits the error of the hit position along the
leaf axis, so tol_u = max(1e-5, K_FRAME u T / |c'(u)|): about 2e-5 for the
hair patch (0.02-long segments four units away), 1e-5 for the tiny and
depth-sweep workloads.

Results that fail STRICT are re-run through the oracle with the ray shifted
sideways (8 directions orthogonal to it, passed in double precision) by
    delta * 2^-k, k = 0..16,   delta = 1e-4 r + K_FRAME * u * T:
1e-4 r is the silhouette band within which hit/miss may differ, the second
term the FP32 resolution above.  A result passes BAND if the oracle result
of one shifted copy meets the strict rule.  The small shifts matter because
near a silhouette the result moves like the square root of the shift, and
for a ray nearly parallel to a fiber a sideways error e moves the hit along
the fiber by e / tan(angle).  The smallest passing shift is recorded, in
units of u T ("band_shift_uT"): it bounds the perturbation the FP32 result
actually needed.

Finally a result is exempt (SILHOUETTE) if the ray passes within 1e-4 r of
the silhouette of the leaf cylinder hit by either side:
|dist(ray, leaf axis) - r_leaf| < 1e-4 r_leaf, in FP64 between the ray line
and the leaf's axis line.  There the hit is ill-conditioned (grazing) and
hit/miss, t and u may all legitimately differ.  Every other result is a
failure.
"""
import json
import os

import numpy as np

import oracle as O

TOL_T = 1e-5
TOL_U = 1e-5
EPS32 = 2.0 ** -24
K_FRAME = 22.0
SCALES = tuple(2.0 ** -k for k in range(17))
# the second, finer search (results the first one leaves unexplained): 32
# directions, scales delta * 2^(-k/8) down to delta * 2^-12
FINE_DIRS = 32
FINE_SCALES = tuple(2.0 ** (-k / 8.0) for k in range(97))
FINE_MAX = 200


def _bez(cp, u):
    u = np.clip(u, 0, 1)[:, None]
    v = 1 - u
    return v ** 3 * cp[:, 0] + 3 * u * v * v * cp[:, 1] + 3 * u * u * v * cp[:, 2] + u ** 3 * cp[:, 3]


def _speed(cp, u):
    u = np.clip(u, 0, 1)[:, None]
    v = 1 - u
    d = 3 * (v * v * (cp[:, 1, :3] - cp[:, 0, :3]) + 2 * u * v * (cp[:, 2, :3] - cp[:, 1, :3])
             + u * u * (cp[:, 3, :3] - cp[:, 2, :3]))
    return np.linalg.norm(d, axis=1)


def frame_extent(cps, rays8, seg):
    """T per result: the largest distance of segment seg's control points
    from the ray origin (FP64); 0 where seg < 0."""
    T = np.zeros(len(seg))
    ok = seg >= 0
    if ok.any():
        cp = cps[seg[ok]].astype(np.float64)[:, :, :3]
        o = rays8[ok, :3].astype(np.float64)[:, None, :]
        T[ok] = np.linalg.norm(cp - o, axis=2).max(axis=1)
    return T


def u_tolerance(case, rays8, seg, t, u):
    """Per-result |u| tolerance: max(1e-5, K_FRAME 2^-24 T / |c'(u)|)."""
    seg = np.asarray(seg, dtype=np.int64)
    tol = np.full(len(seg), TOL_U)
    hit = (seg >= 0) & np.isfinite(t)
    if hit.any():
        cp = case["cps"][seg[hit]].astype(np.float64)
        T = frame_extent(case["cps"], rays8[hit], seg[hit])
        tol[hit] = np.maximum(TOL_U, K_FRAME * EPS32 * T / np.maximum(_speed(cp, u[hit]), 1e-30))
    return tol


def strict_ok(t_g, u_g, s_g, t_o, u_o, s_o, tol_u=TOL_U):
    hit_g, hit_o = s_g >= 0, s_o >= 0
    ok = hit_g == hit_o
    both = hit_g & hit_o
    with np.errstate(invalid="ignore"):
        vals = (s_g == s_o) & (np.abs(t_g - t_o) <= TOL_T * np.abs(t_o)) & (np.abs(u_g - u_o) <= tol_u)
    return ok & (~both | vals)


def _perp(w):
    a = np.where(np.abs(w[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0.0, 1, 0]]))
    e1 = a - np.sum(a * w, axis=1, keepdims=True) * w
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(w, e1)
    return e1, e2


def _shift_search(case, rays8, cands, g, depth, pieces, delta, T, dirs_of, scales):
    """Oracle results of the rays shifted by delta * scale along each of
    dirs_of(e1, e2); returns (passed [m], smallest passing shift / (2^-24 T))."""
    m = len(cands)
    rays = rays8.astype(np.float64)
    o_, w = rays[:, :3], rays[:, 4:7]
    w = w / np.linalg.norm(w, axis=1, keepdims=True)
    e1, e2 = _perp(w)
    dirs = dirs_of(e1, e2)
    tmax = rays[:, 3]
    sub_rays, rows, segs = [], [0], []
    for sc in scales:
        for dv in dirs:
            # double-precision rays: shifts far below an FP32 step of |o| stay exact
            sub_rays.append(np.concatenate([o_ + (delta * sc)[:, None] * dv, w, tmax[:, None]], axis=1))
            for c in cands:
                segs.append(c)
                rows.append(rows[-1] + len(c))
    ref = O.closest_d(np.concatenate(sub_rays), np.array(rows, dtype=np.int32),
                      np.concatenate(segs).astype(np.int32) if segs else np.zeros(0, np.int32),
                      depth, pieces)
    tol_u = u_tolerance(case, rays8, g["seg"], g["t"], g["u"])
    ok = np.zeros(m, dtype=bool)
    shift = np.full(m, np.inf)
    k = 0
    for sc in scales:
        for _ in dirs:
            sl = slice(k * m, (k + 1) * m)
            hit = strict_ok(g["t"], g["u"], g["seg"], ref["t"][sl], ref["u"][sl], ref["seg"][sl], tol_u)
            shift = np.where(hit, np.minimum(shift, delta * sc / (EPS32 * np.maximum(T, 1e-30))), shift)
            ok |= hit
            k += 1
    return ok, shift


def band_check(case, rays8, cands, g, o, depth, pieces):
    """For results that failed the strict rule: rays8 [m, 8] their rays,
    cands a list of m candidate-id arrays (a ray's row, or one pair's
    segment), g / o dicts of the GPU / oracle results (t, u, seg) per
    result.  Returns (passed [m] bool, smallest passing shift in units of
    2^-24 T [m], inf where none).

    The first search takes 8 directions and factors of 2; results it leaves
    unexplained (at most FINE_MAX of them) are searched again with 32
    directions and factors of 2^(1/8).  A ray nearly parallel to its fiber
    needs the finer one: there u moves along the fiber by the shift over
    tan(angle), so only a narrow range of shifts reproduces a u to 1e-5."""
    m = len(cands)
    if m == 0:
        return np.zeros(0, bool), np.zeros(0)
    rays = rays8.astype(np.float64)
    o_, w = rays[:, :3], rays[:, 4:7]
    w = w / np.linalg.norm(w, axis=1, keepdims=True)
    # the segment and u the band is measured at: the GPU's hit, else the oracle's
    use_g = g["seg"] >= 0
    seg = np.where(use_g, g["seg"], o["seg"]).astype(np.int64)
    uu = np.where(use_g, g["u"], o["u"])
    has = seg >= 0
    r = np.full(m, case["cps"][:, :, 3].max())
    T = np.zeros(m)
    if has.any():
        r[has] = _bez(case["cps"][seg[has]].astype(np.float64), uu[has])[:, 3]
        T[has] = frame_extent(case["cps"], rays8[has], seg[has])
    T = np.where(has, T, np.linalg.norm(o_, axis=1))
    delta = 1e-4 * r + K_FRAME * EPS32 * T
    s2 = np.sqrt(0.5)
    ok, shift = _shift_search(case, rays8, cands, g, depth, pieces, delta, T,
                              lambda e1, e2: [e1, -e1, e2, -e2, s2 * (e1 + e2), s2 * (e1 - e2),
                                              s2 * (-e1 + e2), s2 * (-e1 - e2)], SCALES)
    rest = np.nonzero(~ok)[0][:FINE_MAX]
    if len(rest):
        ang = 2 * np.pi * np.arange(FINE_DIRS) / FINE_DIRS
        sub = {k: v[rest] for k, v in g.items()}
        ok2, shift2 = _shift_search(case, rays8[rest], [cands[i] for i in rest], sub, depth, pieces, delta[rest],
                                    T[rest], lambda e1, e2: [np.cos(a) * e1 + np.sin(a) * e2 for a in ang],
                                    FINE_SCALES)
        ok[rest] = ok2
        shift[rest] = shift2
    return ok, shift


def silhouette_dist(case, ray8, seg, leaf, depth):
    """|dist(ray line, leaf axis line) - r_leaf| / r_leaf for the leaf of
    segment `seg` starting at `leaf` (units of 2^-23), FP64."""
    if seg < 0 or leaf < 0:
        return np.inf
    cp = case["cps"][seg].astype(np.float64)
    size = O.ROOT_SIZE >> min(depth, 23)
    start = (int(leaf) // size) * size
    node = O.node_at(cp, start, size)
    r_leaf = O.cons_radius(node)
    ray = np.asarray(ray8, dtype=np.float64)
    o, w = ray[:3], ray[4:7] / np.linalg.norm(ray[4:7])
    p, d = node[0, :3], node[1, :3]
    n = np.cross(w, d)
    if np.linalg.norm(n) == 0:
        dist = np.linalg.norm(np.cross(p - o, w))
    else:
        dist = abs(np.dot(p - o, n)) / np.linalg.norm(n)
    return abs(dist - r_leaf) / r_leaf


def _finish(case, depth, rays8, cands, g, o, ok, g_leaf, o_leaf, pieces, n_items, hits):
    """Band and silhouette passes of the strict failures, and the stats."""
    bad = np.nonzero(~ok)[0]
    sub = lambda d: {k: v[bad] for k, v in d.items()}  # noqa: E731
    passed, shift = band_check(case, rays8[bad], [cands(i) for i in bad], sub(g), sub(o), depth, pieces)
    banded = bad[passed]
    rest = bad[~passed]
    sil = []
    for i in rest:
        ds = silhouette_dist(case, rays8[i], int(o["seg"][i]), int(o_leaf[i]), depth) \
            if o_leaf is not None else np.inf
        if g_leaf is not None:
            ds = min(ds, silhouette_dist(case, rays8[i], int(g["seg"][i]), int(g_leaf[i]), depth))
        if ds < 1e-4:
            sil.append(i)
    sil = np.array(sil, dtype=np.int64)
    fail = np.setdiff1d(rest, sil)
    tol_u = u_tolerance(case, rays8, o["seg"], o["t"], o["u"])
    both = (g["seg"] >= 0) & (o["seg"] >= 0) & ok
    rel = np.abs(g["t"][both] - o["t"][both]) / o["t"][both] if both.any() else np.zeros(1)
    du = np.abs(g["u"][both] - o["u"][both]) if both.any() else np.zeros(1)
    du_rel = du / tol_u[both] if both.any() else np.zeros(1)
    detail = [dict(i=int(i), gpu=(float(g["t"][i]), float(g["u"][i]), int(g["seg"][i])),
                   ref=(float(o["t"][i]), float(o["u"][i]), int(o["seg"][i])), tol_u=float(tol_u[i]))
              for i in fail[:6]]
    sh = shift[passed]
    return dict(n=n_items, hits=hits, strict=int(ok.sum()), band=int(len(banded)), silhouette=int(len(sil)),
                fail=fail, max_rel_t=float(rel.max()), max_du=float(du.max()),
                max_du_over_tol=float(du_rel.max()), med_rel_t=float(np.median(rel)), detail=detail,
                band_shift_uT_max=float(sh.max()) if sh.size else 0.0,
                band_shift_uT_median=float(np.median(sh)) if sh.size else 0.0)


def compare_closest(case, depth, gpu_tu, gpu_seg, ref, pieces, gpu_leaf=None):
    """Closest hits per ray against the oracle's; returns a stats dict whose
    'fail' lists the rays failing strict, band and silhouette."""
    g = dict(t=gpu_tu[:, 0].astype(np.float64), u=gpu_tu[:, 1].astype(np.float64),
             seg=np.asarray(gpu_seg).astype(np.int64))
    o = dict(t=np.asarray(ref["t"], np.float64), u=np.asarray(ref["u"], np.float64),
             seg=np.asarray(ref["seg"]).astype(np.int64))
    rays8 = case["rays"]
    tol_u = u_tolerance(case, rays8, o["seg"], o["t"], o["u"])
    ok = strict_ok(g["t"], g["u"], g["seg"], o["t"], o["u"], o["seg"], tol_u)
    rp = case["row_ptr"].astype(np.int64)
    return _finish(case, depth, rays8, lambda i: case["seg_idx"][rp[i]:rp[i + 1]], g, o, ok, gpu_leaf,
                   ref.get("leaf"), pieces, len(o["seg"]), int((o["seg"] >= 0).sum()))


def count_band_delta(case):
    """Per ray, the FP32 band of its count search: 1e-4 of the largest
    radius plus K_FRAME 2^-24 of the largest control-point distance over the
    ray's candidates.  oracle.ray_counts_amb flags the rays with a decision
    (a bounding-volume test, a child order, a hit against the closest so far)
    within that distance of flipping; a count may differ in FP32 only there."""
    rp = case["row_ptr"].astype(np.int64)
    d = np.zeros(len(rp) - 1)
    for i in range(len(d)):
        c = case["seg_idx"][rp[i]:rp[i + 1]]
        o_ = case["rays"][i, :3].astype(np.float64)
        if len(c) == 0:
            continue
        cp = case["cps"][c].astype(np.float64)
        d[i] = 1e-4 * cp[:, :, 3].max() + K_FRAME * EPS32 * np.linalg.norm(cp[:, :, :3] - o_, axis=2).max()
    return d


def pair_rays(case):
    """Ray index of every pair of the CSR."""
    rp = case["row_ptr"].astype(np.int64)
    return np.repeat(np.arange(len(rp) - 1), np.diff(rp))


def compare_pairs(case, depth, gpu_tu, gpu_leaf, ref, pieces):
    """Per-pair hits (intersect_pairs) against the oracle's (oracle.pairs),
    pair by pair, under the same strict / band / silhouette rule; a pair's
    band check shifts its ray against its one segment."""
    ray_of = pair_rays(case)
    sid = case["seg_idx"].astype(np.int64)
    t_g = gpu_tu[:, 0].astype(np.float64)
    hit_g, hit_o = np.isfinite(t_g), np.isfinite(ref["t"])
    g = dict(t=t_g, u=gpu_tu[:, 1].astype(np.float64), seg=np.where(hit_g, sid, -1))
    o = dict(t=np.asarray(ref["t"], np.float64), u=np.asarray(ref["u"], np.float64), seg=np.where(hit_o, sid, -1))
    rays8 = case["rays"][ray_of]
    tol_u = u_tolerance(case, rays8, o["seg"], o["t"], o["u"])
    ok = strict_ok(g["t"], g["u"], g["seg"], o["t"], o["u"], o["seg"], tol_u)
    return _finish(case, depth, rays8, lambda j: sid[j:j + 1], g, o, ok,
                   np.asarray(gpu_leaf) if gpu_leaf is not None else None, ref.get("leaf"), pieces,
                   len(sid), int(hit_o.sum()))


def counts_of(stats):
    """The figures of a comparison worth reporting (JSON-able)."""
    keys = ("n", "hits", "strict", "band", "silhouette", "max_rel_t", "med_rel_t", "max_du", "max_du_over_tol",
            "band_shift_uT_max", "band_shift_uT_median")
    out = {k: stats[k] for k in keys}
    out["fail"] = int(len(stats["fail"]))
    return out


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
