"""Seeded synthetic workloads for the ray/fiber intersector.

This module only draws inputs: control points, rays and candidate lists.  It
holds none of the intersection arithmetic, imports neither the CUDA library nor
the FP64 reference, and is the one module both of them are fed from.

Layouts (all float32 unless noted):

* ``cps``     -- ``[n_seg, 4, 4]``: four control points ``(x, y, z, r)`` of a
  cubic Bezier fiber segment, radius in the fourth component (Sec. 3.3 of the
  paper: four-dimensional control points, radius interpolated by the same
  Bezier basis).
* ``rays``    -- ``[n_ray, 8]``: ``(o.x, o.y, o.z, t_max, w.x, w.y, w.z, 0)``;
  ``w`` is normalised in float64 before rounding.
* ``row_ptr`` -- int32 ``[n_ray + 1]``, ``seg_idx`` -- int32 ``[n_pair]``:
  candidate segments of each ray in CSR form (grid-cull rows list segments
  front to back in the order the ray's walk meets them).

Every generator takes an explicit seed; ``SEED_BASE + k`` is the default seed
of workload ``k`` (0 tiny, 1 hair patch, 2 depth sweep, 3 precision stress,
4 differentiation).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

SEED_BASE = 1811033740

_HERE = os.path.dirname(os.path.abspath(__file__))
_CULL_SRC = os.path.join(_HERE, "grid_cull.c")
_CULL_LIB = os.path.join(_HERE, "libgridcull.so")
_lock = threading.Lock()
_lib = None


def rng(seed: int) -> np.random.Generator:
    """Counter-based Philox stream for one workload."""
    return np.random.Generator(np.random.Philox(int(seed)))


# --------------------------------------------------------------------------
# small vector helpers (sampling only)
# --------------------------------------------------------------------------

def _normalize(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _unit_sphere(g, n):
    return _normalize(g.standard_normal((n, 3)))


def _unit_ball(g, n):
    d = _unit_sphere(g, n)
    return d * np.cbrt(g.uniform(0.0, 1.0, (n, 1)))


def _perp_unit(g, d):
    """Uniform random unit vectors perpendicular to the unit rows of d."""
    v = g.standard_normal(d.shape)
    v = v - np.sum(v * d, axis=-1, keepdims=True) * d
    return _normalize(v)


def pack_rays(origin, direction, t_max=np.inf):
    origin = np.asarray(origin, dtype=np.float64)
    direction = _normalize(np.asarray(direction, dtype=np.float64))
    n = origin.shape[0]
    rays = np.zeros((n, 8), dtype=np.float32)
    rays[:, 0:3] = origin
    rays[:, 3] = t_max
    rays[:, 4:7] = direction
    return rays


def bezier(cps, u):
    """Position/radius of cubic Bezier rows at parameters u (float64)."""
    cps = np.asarray(cps, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)[..., None]
    v = 1.0 - u
    return (v ** 3 * cps[:, 0] + 3 * u * v * v * cps[:, 1]
            + 3 * u * u * v * cps[:, 2] + u ** 3 * cps[:, 3])


def bezier_tangent(cps, u):
    cps = np.asarray(cps, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)[..., None]
    v = 1.0 - u
    return 3.0 * (v * v * (cps[:, 1] - cps[:, 0]) + 2 * u * v * (cps[:, 2] - cps[:, 1])
                  + u * u * (cps[:, 3] - cps[:, 2]))


def dense_csr(n_ray, n_seg):
    row_ptr = (np.arange(n_ray + 1, dtype=np.int64) * n_seg).astype(np.int32)
    seg_idx = np.tile(np.arange(n_seg, dtype=np.int32), n_ray)
    return row_ptr, seg_idx


def diagonal_csr(n):
    return np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32)


# --------------------------------------------------------------------------
# workload 0: tiny plain case
# --------------------------------------------------------------------------

def tiny_case(seed: int = SEED_BASE + 0, n_seg: int = 16, n_ray: int = 16384):
    """16 random cubic fibers in [-1,1]^3 (radius U[0.01,0.05] per control
    point) against rays from a radius-5 sphere aimed at U[-0.5,0.5]^3; every
    ray is paired with every segment."""
    g = rng(seed)
    pts = g.uniform(-1.0, 1.0, (n_seg, 4, 3))
    rad = g.uniform(0.01, 0.05, (n_seg, 4, 1))
    cps = np.concatenate([pts, rad], axis=-1).astype(np.float32)
    origin = 5.0 * _unit_sphere(g, n_ray)
    target = g.uniform(-0.5, 0.5, (n_ray, 3))
    rays = pack_rays(origin, target - origin)
    row_ptr, seg_idx = dense_csr(n_ray, n_seg)
    return dict(cps=cps, rays=rays, row_ptr=row_ptr, seg_idx=seg_idx, name="tiny")


# --------------------------------------------------------------------------
# workload 1: hair patch
# --------------------------------------------------------------------------

def hair_fibers(seed: int = SEED_BASE + 1, n_fibers: int = 100_000, n_steps: int = 8,
                step: float = 0.02, bend_deg: float = 15.0,
                r_root: float = 0.002, r_tip: float = 0.0005):
    """C1 chains of cubic segments: roots uniform on the unit square, a random
    walk of n_steps steps whose direction turns by N(0, bend) about a random
    axis perpendicular to it, converted to Bezier form by uniform Catmull-Rom
    tangents (one-sided at the ends); radius tapers linearly root to tip."""
    g = rng(seed)
    sigma = math.radians(bend_deg)
    v = np.zeros((n_fibers, n_steps + 1, 3))
    v[:, 0, 0:2] = g.uniform(0.0, 1.0, (n_fibers, 2))
    d = np.zeros((n_fibers, 3))
    d[:, 2] = 1.0

    def turn(d):
        th = g.normal(0.0, sigma, (d.shape[0], 1))
        b = _perp_unit(g, d)
        return _normalize(d * np.cos(th) + b * np.sin(th))

    d = turn(d)
    for i in range(n_steps):
        v[:, i + 1] = v[:, i] + step * d
        d = turn(d)
    m = np.empty_like(v)
    m[:, 1:-1] = 0.5 * (v[:, 2:] - v[:, :-2])
    m[:, 0] = v[:, 1] - v[:, 0]
    m[:, -1] = v[:, -1] - v[:, -2]
    cps = np.empty((n_fibers, n_steps, 4, 4))
    cps[:, :, 0, :3] = v[:, :-1]
    cps[:, :, 1, :3] = v[:, :-1] + m[:, :-1] / 3.0
    cps[:, :, 2, :3] = v[:, 1:] - m[:, 1:] / 3.0
    cps[:, :, 3, :3] = v[:, 1:]
    s = (np.arange(n_steps)[:, None] + np.arange(4)[None, :] / 3.0) / n_steps
    cps[:, :, :, 3] = r_root - (r_root - r_tip) * s
    return cps.reshape(n_fibers * n_steps, 4, 4).astype(np.float32)


def tile_order(width, height, tile=8):
    """Pixel indices (row-major image) listed tile by tile, rows within a tile."""
    ty, tx = (height + tile - 1) // tile, (width + tile - 1) // tile
    order = []
    ys, xs = np.meshgrid(np.arange(tile), np.arange(tile), indexing="ij")
    for by in range(ty):
        for bx in range(tx):
            y = by * tile + ys.ravel()
            x = bx * tile + xs.ravel()
            ok = (y < height) & (x < width)
            order.append(y[ok] * width + x[ok])
    return np.concatenate(order).astype(np.int64)


# Camera of the hair-patch frame: 55 degrees above the patch, 3.9 units from
# its centre.  With the grid below this gives ~12 candidates per ray on average
# over the whole frame (max ~400), the mix the workload is specified with.
HAIR_EYE = (0.5, -1.73695, 3.25469)
HAIR_LOOK_AT = (0.5, 0.5, 0.06)
HAIR_GRID = (400, 400, 40)


def pinhole_rays(width=1920, height=1080, eye=HAIR_EYE, look_at=HAIR_LOOK_AT,
                 up=(0.0, 0.0, 1.0), vfov_deg=45.0, tile=8):
    """Primary rays through pixel centres, listed in tile order; returns
    (rays, pixel) where pixel[i] is the row-major pixel of ray i."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = _normalize(np.asarray(look_at, dtype=np.float64) - eye)
    right = _normalize(np.cross(fwd, np.asarray(up, dtype=np.float64)))
    upv = np.cross(right, fwd)
    th = math.tan(math.radians(vfov_deg) / 2.0)
    aspect = width / height
    pix = tile_order(width, height, tile)
    py, px = pix // width, pix % width
    sx = ((px + 0.5) / width * 2.0 - 1.0) * th * aspect
    sy = (1.0 - (py + 0.5) / height * 2.0) * th
    dirs = fwd[None, :] + sx[:, None] * right[None, :] + sy[:, None] * upv[None, :]
    origin = np.broadcast_to(eye, dirs.shape)
    return pack_rays(origin, dirs), pix


def _cull_lib():
    global _lib
    with _lock:
        if _lib is None:
            if (not os.path.exists(_CULL_LIB)
                    or os.path.getmtime(_CULL_LIB) < os.path.getmtime(_CULL_SRC)):
                build_cull()
            lib = ctypes.CDLL(_CULL_LIB)
            lib.gc_cull.restype = ctypes.c_int64
            lib.gc_cull.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            _lib = lib
    return _lib


def build_cull(cc: str = "gcc") -> str:
    """Compiles the grid cull into an in-tree shared object (host code)."""
    tmp = _CULL_LIB + ".tmp.%d" % os.getpid()
    cmd = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _CULL_SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True)
    except subprocess.CalledProcessError:
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, _CULL_LIB)
    return _CULL_LIB


def grid_cull(cps, rays, res=(128, 128, 32), nthreads=0):
    """Candidate CSR from the uniform-grid cull (see grid_cull.c)."""
    lib = _cull_lib()
    cps = np.ascontiguousarray(cps, dtype=np.float32)
    rays = np.ascontiguousarray(rays, dtype=np.float32)
    n_seg, n_ray = cps.shape[0], rays.shape[0]
    row_ptr = np.zeros(n_ray + 1, dtype=np.int32)
    args = (cps.ctypes.data, n_seg, rays.ctypes.data, n_ray, int(res[0]), int(res[1]), int(res[2]),
            int(nthreads))
    n = lib.gc_cull(*args, row_ptr.ctypes.data, None, 0)
    if n < 0:
        raise MemoryError("grid cull failed (%d)" % n)
    seg_idx = np.zeros(max(n, 1), dtype=np.int32)
    m = lib.gc_cull(*args, row_ptr.ctypes.data, seg_idx.ctypes.data, n)
    if m != n:
        raise RuntimeError("grid cull count mismatch %d vs %d" % (m, n))
    return row_ptr, seg_idx[:n]


def hair_patch(seed: int = SEED_BASE + 1, n_fibers: int = 100_000, width: int = 1920,
               height: int = 1080, grid=HAIR_GRID, nthreads: int = 0):
    """The hair-patch frame: fibers, tile-ordered pinhole rays and the grid-cull
    candidate CSR."""
    cps = hair_fibers(seed, n_fibers)
    rays, pix = pinhole_rays(width, height)
    row_ptr, seg_idx = grid_cull(cps, rays, grid, nthreads)
    return dict(cps=cps, rays=rays, pixel=pix, row_ptr=row_ptr, seg_idx=seg_idx,
                name="hair_patch", width=width, height=height)


def subsample_rays(case, idx):
    """Restricts a CSR workload to the rays idx (order kept)."""
    idx = np.asarray(idx, dtype=np.int64)
    rp = case["row_ptr"].astype(np.int64)
    counts = rp[idx + 1] - rp[idx]
    row_ptr = np.zeros(len(idx) + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    seg_idx = np.concatenate([case["seg_idx"][rp[i]:rp[i + 1]] for i in idx]) if len(idx) else \
        np.zeros(0, np.int32)
    out = dict(case)
    out.update(rays=case["rays"][idx], row_ptr=row_ptr.astype(np.int32),
               seg_idx=seg_idx.astype(np.int32))
    if "pixel" in case:
        out["pixel"] = case["pixel"][idx]
    return out


# --------------------------------------------------------------------------
# workload 2: depth sweep over three curvature classes
# --------------------------------------------------------------------------

SWEEP_JITTER = {"straight": 0.01, "moderate": 0.10, "curved": 0.50}


def sweep_segments(g, n, jitter, L=1.0):
    p0 = g.uniform(-10.0, 10.0, (n, 3))
    p3 = p0 + L * _unit_sphere(g, n)
    p1 = p0 + (p3 - p0) / 3.0 + jitter * L * _unit_ball(g, n)
    p2 = p0 + 2.0 * (p3 - p0) / 3.0 + jitter * L * _unit_ball(g, n)
    r = g.uniform(0.001, 0.01, (n, 4)) * L
    cps = np.stack([p0, p1, p2, p3], axis=1)
    return np.concatenate([cps, r[..., None]], axis=-1).astype(np.float32)


def sweep_case(klass: str, n: int, seed: int = SEED_BASE + 2, forced_hits: bool = False):
    """One ray per segment.  Default rays aim at a uniform point of the
    segment's radius-dilated control-hull AABB from 10 segment lengths away;
    forced_hits aims them at c(u) + delta with |delta| < r(u) instead."""
    g = rng(seed + 7919 * list(SWEEP_JITTER).index(klass))
    cps = sweep_segments(g, n, SWEEP_JITTER[klass])
    c64 = cps.astype(np.float64)
    if forced_hits:
        u = g.uniform(0.0, 1.0, n)
        c = bezier(c64, u)
        target = c[:, :3] + 0.9 * c[:, 3:4] * _unit_ball(g, n)
    else:
        rmax = c64[:, :, 3].max(axis=1, keepdims=True)
        lo = c64[:, :, :3].min(axis=1) - rmax
        hi = c64[:, :, :3].max(axis=1) + rmax
        target = lo + (hi - lo) * g.uniform(0.0, 1.0, (n, 3))
    w = _unit_sphere(g, n)
    rays = pack_rays(target - 10.0 * w, w)
    row_ptr, seg_idx = diagonal_csr(n)
    return dict(cps=cps, rays=rays, row_ptr=row_ptr, seg_idx=seg_idx,
                name="sweep_%s" % klass)


def single_fiber_case(klass: str, n_ray: int, seed: int = SEED_BASE + 5):
    """One segment of the curvature class against n_ray rays, each aimed at a
    uniform point of the segment's radius-dilated control-hull AABB from 10
    segment lengths away in a uniform direction: the shape of the paper's own
    benchmark (Fig. 1: about a million rays against a single fiber), whose
    three fibers are given only as images."""
    g = rng(seed + 7919 * list(SWEEP_JITTER).index(klass))
    cps = sweep_segments(g, 1, SWEEP_JITTER[klass])
    c64 = cps.astype(np.float64)[0]
    rmax = c64[:, 3].max()
    lo = c64[:, :3].min(axis=0) - rmax
    hi = c64[:, :3].max(axis=0) + rmax
    target = lo + (hi - lo) * g.uniform(0.0, 1.0, (n_ray, 3))
    w = _unit_sphere(g, n_ray)
    rays = pack_rays(target - 10.0 * w, w)
    row_ptr = np.arange(n_ray + 1, dtype=np.int32)
    seg_idx = np.zeros(n_ray, dtype=np.int32)
    return dict(cps=cps, rays=rays, row_ptr=row_ptr, seg_idx=seg_idx, name="single_%s" % klass)


def single_fiber_image_case(klass: str, res: int = 512, seed: int = SEED_BASE + 7):
    """One segment of the curvature class seen by a res x res pinhole camera
    (the setting of Fig. 8's per-pixel heat maps): radii 0.005-0.05 of the
    segment's length; the camera looks at the chord's midpoint from 2.5
    segment lengths away, perpendicular to the chord, with a 30 degree field
    of view; every ray lists the segment.
    Returns the case with `pixel` (row-major pixel of each ray) and `res`."""
    g = rng(seed + 7919 * list(SWEEP_JITTER).index(klass))
    cps = sweep_segments(g, 1, SWEEP_JITTER[klass])
    cps[..., 3] *= 5.0  # radii 0.005-0.05 of the length: a fiber some pixels wide
    c = cps[0].astype(np.float64)
    mid = 0.5 * (c[0, :3] + c[3, :3])
    chord = _normalize((c[3, :3] - c[0, :3])[None])[0]
    side = _perp_unit(g, chord[None])[0]
    eye = mid + 2.5 * side
    rays, pix = pinhole_rays(res, res, eye=eye, look_at=mid, up=tuple(np.cross(side, chord)), vfov_deg=30.0)
    n = rays.shape[0]
    return dict(cps=cps, rays=rays, row_ptr=np.arange(n + 1, dtype=np.int32), seg_idx=np.zeros(n, np.int32),
                pixel=pix, res=res, name="image_%s" % klass)


def quadratic_segments(g, n, jitter, L=1.0):
    """Quadratic segments [n, 3, 4]: p0 ~ U[-10, 10]^3, p2 = p0 + L u (u
    uniform on the sphere), p1 = the chord's midpoint + jitter * L * (a point
    of the unit ball), radius U[0.001, 0.01] L per control point."""
    p0 = g.uniform(-10.0, 10.0, (n, 3))
    p2 = p0 + L * _unit_sphere(g, n)
    p1 = 0.5 * (p0 + p2) + jitter * L * _unit_ball(g, n)
    r = g.uniform(0.001, 0.01, (n, 3)) * L
    cps = np.stack([p0, p1, p2], axis=1)
    return np.concatenate([cps, r[..., None]], axis=-1).astype(np.float32)


def quadratic_eval(cps, u):
    """Quadratic Bezier point (all four components) by de Casteljau, for
    aiming rays."""
    u = np.asarray(u)[:, None]
    a = (1 - u) * cps[:, 0] + u * cps[:, 1]
    b = (1 - u) * cps[:, 1] + u * cps[:, 2]
    return (1 - u) * a + u * b


def quadratic_case(klass: str, n: int, seed: int = SEED_BASE + 6, forced_hits: bool = False):
    """The depth-sweep workload for quadratic fibers: one ray per segment,
    aimed at its radius-dilated control-hull box, or (forced_hits) at
    c(u) + delta with |delta| < r(u)."""
    g = rng(seed + 7919 * list(SWEEP_JITTER).index(klass))
    cps = quadratic_segments(g, n, SWEEP_JITTER[klass])
    c64 = cps.astype(np.float64)
    if forced_hits:
        c = quadratic_eval(c64, g.uniform(0.0, 1.0, n))
        target = c[:, :3] + 0.9 * c[:, 3:4] * _unit_ball(g, n)
    else:
        rmax = c64[:, :, 3].max(axis=1, keepdims=True)
        lo = c64[:, :, :3].min(axis=1) - rmax
        hi = c64[:, :, :3].max(axis=1) + rmax
        target = lo + (hi - lo) * g.uniform(0.0, 1.0, (n, 3))
    w = _unit_sphere(g, n)
    rays = pack_rays(target - 10.0 * w, w)
    row_ptr, seg_idx = diagonal_csr(n)
    return dict(cps=cps, rays=rays, row_ptr=row_ptr, seg_idx=seg_idx, name="quadratic_%s" % klass)


# --------------------------------------------------------------------------
# workload 3: precision stress
# --------------------------------------------------------------------------

def grazing_case(n: int, seed: int = SEED_BASE + 3, band: float = 1e-3):
    """Rays tangent to the circle of radius r(u)(1+delta), |delta| <= band,
    around c(u) in its normal plane, on moderate-curvature segments."""
    g = rng(seed)
    cps = sweep_segments(g, n, SWEEP_JITTER["moderate"])
    c64 = cps.astype(np.float64)
    u = g.uniform(0.1, 0.9, n)
    c = bezier(c64, u)
    tg = _normalize(bezier_tangent(c64, u)[:, :3])
    e = _perp_unit(g, tg)
    delta = g.uniform(-band, band, (n, 1))
    q = c[:, :3] + c[:, 3:4] * (1.0 + delta) * e
    w = _normalize(np.cross(tg, e))
    rays = pack_rays(q - 10.0 * w, w)
    row_ptr, seg_idx = diagonal_csr(n)
    return dict(cps=cps, rays=rays, row_ptr=row_ptr, seg_idx=seg_idx, name="grazing",
                u_aim=u, delta=delta[:, 0])


def offset_case(n: int, offset: float, seed: int = SEED_BASE + 3, r_rel: float = 1e-4):
    """Thin fibers (r = r_rel * L) and rays aimed within +-2r of the curve,
    the whole scene translated by `offset` along (1,1,1)/sqrt(3)."""
    g = rng(seed + int(offset))
    cps = sweep_segments(g, n, SWEEP_JITTER["moderate"]).astype(np.float64)
    cps[:, :, 3] = r_rel
    u = g.uniform(0.0, 1.0, n)
    c = bezier(cps, u)
    tg = _normalize(bezier_tangent(cps, u)[:, :3])
    e = _perp_unit(g, tg)
    target = c[:, :3] + g.uniform(-2.0, 2.0, (n, 1)) * r_rel * e
    w = _unit_sphere(g, n)
    shift = offset / math.sqrt(3.0)
    cps[:, :, :3] += shift
    rays = pack_rays(target - 10.0 * w + shift, w)
    row_ptr, seg_idx = diagonal_csr(n)
    return dict(cps=cps.astype(np.float32), rays=rays, row_ptr=row_ptr, seg_idx=seg_idx,
                name="offset_%g" % offset)


# --------------------------------------------------------------------------
# workload 4: differentiation
# --------------------------------------------------------------------------

def hit_weights(n: int, seed: int = SEED_BASE + 4):
    """Loss weights w_i ~ N(0, 1) for L = sum_i w_i t_i."""
    return rng(seed).standard_normal(n).astype(np.float32)


def aimed_hair_case(n: int, seed: int = SEED_BASE + 4, n_fibers: int = 2000):
    """Rays aimed at points inside hair segments (one per ray), for gradient
    checks on hair-patch geometry without the full frame."""
    g = rng(seed)
    cps = hair_fibers(seed, n_fibers)
    seg = g.integers(0, cps.shape[0], n)
    c64 = cps.astype(np.float64)[seg]
    u = g.uniform(0.05, 0.95, n)
    c = bezier(c64, u)
    target = c[:, :3] + 0.8 * c[:, 3:4] * _unit_ball(g, n)
    w = _unit_sphere(g, n)
    rays = pack_rays(target - 0.5 * w, w)
    row_ptr = np.arange(n + 1, dtype=np.int32)
    return dict(cps=cps, rays=rays, row_ptr=row_ptr, seg_idx=seg.astype(np.int32),
                name="aimed_hair")
