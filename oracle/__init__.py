"""FP64 CPU oracle for the ray / cubic-fiber intersection (arXiv 1811.03374).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may use it; the library never
does.  The arithmetic lives in ``fiber_oracle.c`` (plain C, double precision,
each function citing the passage of the paper it follows); this module only
compiles it and marshals numpy arrays.

Functions with no independent pin are listed as "parity unpinned" here; at
present every exported function is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fiber_oracle.c")
_LIB = os.path.join(_HERE, "libfiber_oracle.so")
_lock = threading.Lock()
_lib = None

ROOT_SIZE = 1 << 23
MAX_PRESPLIT = 8


class OrcHit(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("u", ctypes.c_double), ("hit", ctypes.c_int32),
                ("leaf", ctypes.c_int32), ("nodes", ctypes.c_int32), ("descents", ctypes.c_int32),
                ("backtracks", ctypes.c_int32), ("pad", ctypes.c_int32)]


def build(cc: str = "gcc", src: str = _SRC, out: str = _LIB) -> str:
    """Compiles the oracle (host C, OpenMP when available) in-tree."""
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True)
    except subprocess.CalledProcessError:
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, out)
    return out


def _p(a):
    # data_as keeps a reference to the array, so temporaries outlive the call
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("FIBER_ORACLE_LIB")  # a test may load a planted-mistake copy
            if not path:
                if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
                    build()
                path = _LIB
            L = ctypes.CDLL(path)
            vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            u32 = ctypes.c_uint32
            L.orc_valid_cubic.argtypes = [vp]; L.orc_valid_cubic.restype = i32
            L.orc_thick_ok.argtypes = [vp]; L.orc_thick_ok.restype = i32
            L.orc_split_half.argtypes = [vp, vp, vp]; L.orc_split_half.restype = None
            L.orc_ray_counts.argtypes = [vp, i64, vp, vp, vp, vp, vp, i32, i32, i32, vp, vp]
            L.orc_ray_counts.restype = None
            L.orc_ray_counts_d.argtypes = [vp, i64, vp, vp, vp, vp, vp, i32, i32, i32, vp, vp]
            L.orc_ray_counts_d.restype = None
            L.orc_ray_counts_amb.argtypes = [vp, i64, vp, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp]
            L.orc_ray_counts_amb.restype = None
            L.orc_presplit_d.argtypes = [vp, i64, i32, i32, vp, vp, vp, vp, vp, i64]
            L.orc_presplit_d.restype = i64
            L.orc_valid_quadratic.argtypes = [vp]; L.orc_valid_quadratic.restype = i32
            L.orc_elevate_quadratic.argtypes = [vp, vp]; L.orc_elevate_quadratic.restype = None
            L.orc_presplit.argtypes = [vp, i64, i32, i32, vp, vp, vp, vp, vp, i64]
            L.orc_presplit.restype = i64
            L.orc_intersect.argtypes = [vp, vp, i32, ctypes.POINTER(OrcHit)]
            L.orc_intersect.restype = None
            L.orc_closest.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp]
            L.orc_closest.restype = None
            L.orc_closest_d.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp]
            L.orc_closest_d.restype = None
            L.orc_pairs.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp]
            L.orc_pairs.restype = None
            L.orc_to_ray_frame.argtypes = [vp, vp, vp]; L.orc_to_ray_frame.restype = None
            L.orc_node_at.argtypes = [vp, u32, u32, vp]; L.orc_node_at.restype = None
            L.orc_subdivide.argtypes = [vp, i32, vp]; L.orc_subdivide.restype = None
            L.orc_cons_radius.argtypes = [vp]; L.orc_cons_radius.restype = dbl
            L.orc_cylinder.argtypes = [vp, vp, dbl, vp]; L.orc_cylinder.restype = i32
            L.orc_slab.argtypes = [vp, dbl, vp]; L.orc_slab.restype = i32
            L.orc_leaf_hit.argtypes = [vp, vp, i32, u32, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
            L.orc_leaf_hit.restype = i32
            L.orc_normal.argtypes = [vp, vp, u32, u32, dbl, vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
            L.orc_normal.restype = i32
            L.orc_limit_hit.argtypes = [vp, vp, i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
            L.orc_limit_hit.restype = i32
            L.orc_grad_t.argtypes = [vp, vp, dbl, dbl, vp]; L.orc_grad_t.restype = i32
            L.orc_refine_hit.argtypes = [vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
            L.orc_refine_hit.restype = None
            L.orc_num_threads.argtypes = []; L.orc_num_threads.restype = i32
            _lib = L
    return _lib


def _d(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def ray7(o, w, tmax=np.inf):
    return np.array([o[0], o[1], o[2], w[0], w[1], w[2], tmax], dtype=np.float64)


def ray7_from_packed(r8):
    r8 = np.asarray(r8, dtype=np.float64)
    return np.array([r8[0], r8[1], r8[2], r8[4], r8[5], r8[6], r8[3]], dtype=np.float64)


# ----------------------------------------------------------------- wrappers

def valid_quadratic(cp):
    """App. B.1's constraint on a quadratic curve [3, 4]."""
    return bool(lib().orc_valid_quadratic(_p(_d(cp, (12,)))))


def elevate_quadratics(cps):
    """[n, 3, 4] quadratic control points -> [n, 4, 4] float64 cubic ones with
    the same curve and parametrisation."""
    q = np.ascontiguousarray(cps, dtype=np.float64).reshape(-1, 12)
    out = np.zeros((q.shape[0], 16))
    L = lib()
    for i in range(q.shape[0]):
        L.orc_elevate_quadratic(q[i].ctypes.data_as(ctypes.c_void_p), out[i].ctypes.data_as(ctypes.c_void_p))
    return out.reshape(-1, 4, 4)


def valid_cubic(cp):
    return bool(lib().orc_valid_cubic(_p(_d(cp, (16,)))))


def thick_ok(cp):
    return bool(lib().orc_thick_ok(_p(_d(cp, (16,)))))


def split_half(cp):
    cp = _d(cp, (16,))
    L = np.zeros(16); R = np.zeros(16)
    lib().orc_split_half(_p(cp), _p(L), _p(R))
    return L.reshape(4, 4), R.reshape(4, 4)


def presplit(cps, max_level=MAX_PRESPLIT, thick=True):
    """Pieces of every segment: dict(cp [n,4,4] f64, seg, level, off, flags,
    begin [n_seg+1]).  Cubic control points [n,4,4] (float32 as given, or
    float64 kept in double precision), or quadratic ones [n,3,4], which are
    raised to cubics in FP64 first."""
    cps = np.asarray(cps)
    if cps.ndim == 3 and cps.shape[1] == 3:
        cps = elevate_quadratics(cps)
    L = lib()
    if cps.dtype == np.float64:
        cps = np.ascontiguousarray(cps).reshape(-1, 16)
        split = L.orc_presplit_d
    else:
        cps = np.ascontiguousarray(cps, dtype=np.float32).reshape(-1, 16)
        split = L.orc_presplit
    n_seg = cps.shape[0]
    n = split(_p(cps), n_seg, max_level, int(thick), None, None, None, None, None, 0)
    cp = np.zeros((max(n, 1), 16)); seg = np.zeros(max(n, 1), np.int32)
    lv = np.zeros_like(seg); off = np.zeros_like(seg); fl = np.zeros_like(seg)
    split(_p(cps), n_seg, max_level, int(thick), _p(cp), _p(seg), _p(lv), _p(off), _p(fl), n)
    begin = np.zeros(n_seg + 1, np.int32)
    np.add.at(begin, seg[:n] + 1, 1)
    begin = np.cumsum(begin).astype(np.int32)
    return dict(cp=cp[:n].reshape(n, 4, 4), seg=seg[:n], level=lv[:n], off=off[:n], flags=fl[:n],
                begin=begin)


def intersect(ray, cp, depth):
    """One ray (7-vector o, w, t_max) against one curve; returns OrcHit."""
    h = OrcHit()
    lib().orc_intersect(_p(_d(ray, (7,))), _p(_d(cp, (16,))), int(depth), ctypes.byref(h))
    return h


def _ws(case, pieces):
    rays = np.ascontiguousarray(case["rays"], dtype=np.float32)
    rp = np.ascontiguousarray(case["row_ptr"], dtype=np.int32)
    si = np.ascontiguousarray(case["seg_idx"], dtype=np.int32)
    pc = np.ascontiguousarray(pieces["cp"], dtype=np.float64).reshape(-1, 16)
    return rays, rp, si, pc


def closest(case, depth, pieces=None, nthreads=0):
    """Closest hit per ray; dict(t, u, seg, leaf, counters)."""
    if pieces is None:
        pieces = presplit(case["cps"])
    rays, rp, si, pc = _ws(case, pieces)
    n = rays.shape[0]
    t = np.zeros(n); u = np.zeros(n); seg = np.zeros(n, np.int32); leaf = np.zeros(n, np.int32)
    cnt = np.zeros(5, np.int64)
    lib().orc_closest(_p(rays), n, _p(rp), _p(si), _p(pc), _p(pieces["begin"]), _p(pieces["level"]),
                      _p(pieces["off"]), int(depth), int(nthreads), _p(t), _p(u), _p(seg), _p(leaf),
                      _p(cnt))
    return dict(t=t, u=u, seg=seg, leaf=leaf,
                counters=dict(zip(["nodes", "descents", "backtracks", "hits", "tests"], cnt.tolist())))


def ray_counts(case, depth, mode, pieces=None, nthreads=0):
    """Per-ray pruning tests (Fig. 8): mode "cylinder" (the
    traversal's node tests) or "box" (ray-frame axis-aligned boxes); each ray's
    candidates in row order with the closest hit so far as t_max.  Returns
    (counts int64 [n_ray], closest t [n_ray])."""
    if pieces is None:
        pieces = presplit(case["cps"])
    rays, rp, si, pc = _ws(case, pieces)
    n = rays.shape[0]
    counts = np.zeros(n, np.int64)
    t = np.zeros(n)
    lib().orc_ray_counts(_p(rays), n, _p(rp), _p(si), _p(pc), _p(pieces["begin"]), _p(pieces["level"]),
                         int(depth), {"cylinder": 0, "box": 1}[mode], int(nthreads), _p(counts), _p(t))
    return counts, t


def ray_counts_amb(case, depth, mode, delta, pieces=None, nthreads=0):
    """ray_counts() and, per ray, whether any decision of its search lies
    within delta[i] (a length; per ray) of flipping under a sideways move of
    the ray: (counts int64 [n_ray], ambiguous bool [n_ray])."""
    if pieces is None:
        pieces = presplit(case["cps"])
    rays, rp, si, pc = _ws(case, pieces)
    n = rays.shape[0]
    counts = np.zeros(n, np.int64)
    amb = np.zeros(n, np.int32)
    dl = np.ascontiguousarray(np.broadcast_to(np.asarray(delta, np.float64), (n,)))
    lib().orc_ray_counts_amb(_p(rays), n, _p(rp), _p(si), _p(pc), _p(pieces["begin"]), _p(pieces["level"]),
                             int(depth), {"cylinder": 0, "box": 1}[mode], int(nthreads), _p(dl), _p(counts),
                             _p(amb))
    return counts, amb.astype(bool)


def ray_counts_d(rays7, row_ptr, seg_idx, depth, mode, pieces, nthreads=0):
    """ray_counts() with double-precision rays [n, 7] (o, w, t_max)."""
    rays7 = np.ascontiguousarray(rays7, dtype=np.float64)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    si = np.ascontiguousarray(seg_idx, dtype=np.int32)
    pc = np.ascontiguousarray(pieces["cp"], dtype=np.float64).reshape(-1, 16)
    n = rays7.shape[0]
    counts = np.zeros(n, np.int64)
    t = np.zeros(n)
    lib().orc_ray_counts_d(_p(rays7), n, _p(rp), _p(si), _p(pc), _p(pieces["begin"]), _p(pieces["level"]),
                           int(depth), {"cylinder": 0, "box": 1}[mode], int(nthreads), _p(counts), _p(t))
    return counts, t


def closest_d(rays7, row_ptr, seg_idx, depth, pieces, nthreads=0):
    """closest() with double-precision rays [n, 7] (o, w, t_max)."""
    rays7 = np.ascontiguousarray(rays7, dtype=np.float64)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    si = np.ascontiguousarray(seg_idx, dtype=np.int32)
    pc = np.ascontiguousarray(pieces["cp"], dtype=np.float64).reshape(-1, 16)
    n = rays7.shape[0]
    t = np.zeros(n); u = np.zeros(n); seg = np.zeros(n, np.int32); leaf = np.zeros(n, np.int32)
    lib().orc_closest_d(_p(rays7), n, _p(rp), _p(si), _p(pc), _p(pieces["begin"]), _p(pieces["level"]),
                        _p(pieces["off"]), int(depth), int(nthreads), _p(t), _p(u), _p(seg), _p(leaf), None)
    return dict(t=t, u=u, seg=seg, leaf=leaf)


def pairs(case, depth, pieces=None, nthreads=0):
    """Per-pair hits; dict(t, u, leaf, counters)."""
    if pieces is None:
        pieces = presplit(case["cps"])
    rays, rp, si, pc = _ws(case, pieces)
    n = rays.shape[0]
    m = si.shape[0]
    t = np.zeros(m); u = np.zeros(m); leaf = np.zeros(m, np.int32)
    cnt = np.zeros(5, np.int64)
    lib().orc_pairs(_p(rays), n, _p(rp), _p(si), _p(pc), _p(pieces["begin"]), _p(pieces["level"]),
                    _p(pieces["off"]), int(depth), int(nthreads), _p(t), _p(u), _p(leaf), _p(cnt))
    return dict(t=t, u=u, leaf=leaf,
                counters=dict(zip(["nodes", "descents", "backtracks", "hits", "tests"], cnt.tolist())))


def to_ray_frame(ray, cp):
    out = np.zeros(16)
    lib().orc_to_ray_frame(_p(_d(ray, (7,))), _p(_d(cp, (16,))), _p(out))
    return out.reshape(4, 4)


def node_at(cp, start, size):
    out = np.zeros(16)
    lib().orc_node_at(_p(_d(cp, (16,))), int(start), int(size), _p(out))
    return out.reshape(4, 4)


def subdivide(node, go_right):
    out = np.zeros(16)
    lib().orc_subdivide(_p(_d(node, (16,))), int(go_right), _p(out))
    return out.reshape(4, 4)


def cons_radius(node):
    return float(lib().orc_cons_radius(_p(_d(node, (16,)))))


def cylinder(p, a, r):
    out = np.zeros(2)
    ok = lib().orc_cylinder(_p(_d(p, (3,))), _p(_d(a, (3,))), float(r), _p(out))
    return (float(out[0]), float(out[1])) if ok else None


def slab(node, ray_tmax=np.inf):
    out = np.zeros(2)
    ok = lib().orc_slab(_p(_d(node, (16,))), float(ray_tmax), _p(out))
    return bool(ok), float(out[0]), float(out[1])


def leaf_hit(ray, cp, depth, leaf):
    t = ctypes.c_double(); u = ctypes.c_double()
    ok = lib().orc_leaf_hit(_p(_d(ray, (7,))), _p(_d(cp, (16,))), int(depth), int(leaf),
                            ctypes.byref(t), ctypes.byref(u))
    return (t.value, u.value) if ok else None


def normal(ray, cp, start, size, t, with_len=False):
    """Normal at a hit t on the leaf [start, start + size) (units of 2^-23)
    of curve cp (App. C): (n (3,), kind, u) with kind 1 lateral, 2 / 3 the
    end cap at u = 0 / 1; with_len adds the vector's length before it was
    normalised."""
    n = np.zeros(3)
    u = ctypes.c_double()
    ln = ctypes.c_double()
    k = lib().orc_normal(_p(_d(ray, 7)), _p(_d(cp, (4, 4))), int(start), int(size), float(t), _p(n),
                         ctypes.byref(u), ctypes.byref(ln))
    return (n, int(k), u.value, ln.value) if with_len else (n, int(k), u.value)


def normals(case, depth, ref, pieces=None):
    """Normals of the closest hits `ref` (from closest()) of a case: (n_ray, 3)
    array (zero for misses), the kind per ray (0 miss, 1 lateral, 2 / 3 end
    caps) and the length of each normal before it was normalised.  The leaf of
    a hit in a piece pre-split to level k has the size 2^-max(depth, k) of
    the segment."""
    pieces = presplit(case["cps"]) if pieces is None else pieces
    n_ray = len(ref["seg"])
    out = np.zeros((n_ray, 3))
    kind = np.zeros(n_ray, dtype=np.int32)
    length = np.zeros(n_ray)
    for i in np.nonzero(ref["seg"] >= 0)[0]:
        s, leaf = int(ref["seg"][i]), int(ref["leaf"][i])
        b, e = pieces["begin"][s], pieces["begin"][s + 1]
        lvl = 0
        for k in range(b, e):
            lo = int(pieces["off"][k]) << (23 - int(pieces["level"][k]))
            hi = (int(pieces["off"][k]) + 1) << (23 - int(pieces["level"][k]))
            if lo <= leaf < hi:
                lvl = int(pieces["level"][k])
        size = ROOT_SIZE >> max(depth, lvl)
        out[i], kind[i], _, length[i] = normal(ray7_from_packed(case["rays"][i]),
                                               case["cps"][s].astype(np.float64), leaf, size, ref["t"][i],
                                               with_len=True)
    return out, kind, length


def limit_hit(ray, cp, n_grid=100000):
    t = ctypes.c_double(); u = ctypes.c_double()
    kind = lib().orc_limit_hit(_p(_d(ray, (7,))), _p(_d(cp, (16,))), int(n_grid), ctypes.byref(t),
                               ctypes.byref(u))
    return kind, t.value, u.value


def grad_t(ray, cp, t, u):
    g = np.zeros(16)
    ok = lib().orc_grad_t(_p(_d(ray, (7,))), _p(_d(cp, (16,))), float(t), float(u), _p(g))
    return g.reshape(4, 4) if ok else None


def refine_hit(ray, cp, t, u):
    tt = ctypes.c_double(t); uu = ctypes.c_double(u)
    lib().orc_refine_hit(_p(_d(ray, (7,))), _p(_d(cp, (16,))), ctypes.byref(tt), ctypes.byref(uu))
    return tt.value, uu.value


def num_threads():
    return int(lib().orc_num_threads())
