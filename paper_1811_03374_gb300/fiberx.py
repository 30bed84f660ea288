"""Python binding of the fiberx C ABI (include/fiberx.h).

Argument marshalling only: every step of the intersection runs in the CUDA
kernels of ``libfiberx.so``.  PyTorch supplies device memory and streams.
The library is built in-tree on first use if it is missing; if it cannot be
loaded the calls raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .csrc import build as _build

FX_OK = 0
FX_ERRORS = {-1: "FX_EINVAL", -2: "FX_ECUDA", -3: "FX_ENOMEM", -4: "FX_EUNSUPPORTED",
             -5: "FX_ETIMEOUT", -6: "FX_EDEPTH", -7: "FX_EDEVICE"}

FX_DEV_ITER_LIMIT = 0x1
FX_DEV_UNSUPPORTED = 0x2
FX_DEV_BAD_INDEX = 0x4
FX_DEV_BAD_DEPTH = 0x8

FX_KERNEL_PERSISTENT = 0x0
FX_KERNEL_NAIVE = 0x1
FX_FAST_MATH = 0x2
FX_POLISH_FP64 = 0x4
FX_COUNT = 0x8
FX_CHECK_INDEX = 0x10
FX_COUNT_BOXES = 0x20

FX_VARIANT_AUTO = 0
FX_VARIANT_LANE = 1
FX_VARIANT_WARP = 2
FX_VARIANT_FILTER = 3
FX_VARIANT_SCAN = 4
FX_VARIANT_RAY = 5

MAX_DEPTH = 23
EXPORTS = ["fiber_upload", "fiber_upload_quadratic", "fiber_free", "fiber_info", "intersect_closest", "intersect_pairs",
           "intersect_backward", "intersect_normals", "intersect_counts", "intersect_closest_host", "fx_host_bytes",
           "intersect_closest_noalloc",
           "fx_set_launch",
           "fx_get_launch", "fx_counters", "fx_stream_status", "fx_fma_peak", "fx_last_error", "fx_version"]
NOALLOC_MAX_RAYS = 1 << 20


class FiberxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (FX_ERRORS.get(code, code), msg))
        self.code = code


class UploadOpts(ctypes.Structure):
    _fields_ = [("max_presplit", ctypes.c_int32), ("thick_check", ctypes.c_int32)]


class FibersInfo(ctypes.Structure):
    _fields_ = [("n_seg", ctypes.c_int64), ("n_piece", ctypes.c_int64), ("n_presplit", ctypes.c_int64),
                ("n_unsupported", ctypes.c_int64), ("max_level", ctypes.c_int32),
                ("sm_count", ctypes.c_int32)]


class Launch(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("variant", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    """The in-tree library, or the build named by FIBERX_LIB (a library built
    with other compile-time settings, for comparing them)."""
    return os.environ.get("FIBERX_LIB") or _build.LIB


def lib():
    """Loads libfiberx.so (building it in-tree if missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if path == _build.LIB and _build.stale():
                _build.build()
            L = ctypes.CDLL(path)
            vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
            L.fiber_upload.argtypes = [vp, i64, i32, ctypes.POINTER(UploadOpts), vp, ctypes.POINTER(vp)]
            L.fiber_upload.restype = i32
            L.fiber_upload_quadratic.argtypes = [vp, i64, i32, ctypes.POINTER(UploadOpts), vp, ctypes.POINTER(vp)]
            L.fiber_upload_quadratic.restype = i32
            L.fiber_free.argtypes = [vp]
            L.fiber_free.restype = None
            L.fiber_info.argtypes = [vp, ctypes.POINTER(FibersInfo)]
            L.fiber_info.restype = i32
            L.intersect_closest.argtypes = [vp, vp, i64, vp, vp, i64, i32, vp, u32, vp, vp, vp, vp]
            L.intersect_closest.restype = i32
            L.intersect_pairs.argtypes = [vp, vp, i64, vp, vp, i64, i32, vp, u32, vp, vp, vp, vp]
            L.intersect_pairs.restype = i32
            L.intersect_backward.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp]
            L.intersect_backward.restype = i32
            L.intersect_counts.argtypes = [vp, vp, i64, vp, vp, i64, i32, u32, vp, vp]
            L.intersect_counts.restype = i32
            L.intersect_normals.argtypes = [vp, vp, i64, vp, vp, vp, i32, vp, u32, vp, vp]
            L.intersect_normals.restype = i32
            L.intersect_closest_host.argtypes = [vp, vp, i64, vp, vp, i64, i32, vp, u32, vp, vp, vp, vp]
            L.intersect_closest_host.restype = i32
            L.fx_host_bytes.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
            L.fx_host_bytes.restype = i32
            L.intersect_closest_noalloc.argtypes = [vp, vp, i64, vp, vp, i64, i32, u32, vp, vp, vp, vp]
            L.intersect_closest_noalloc.restype = i32
            L.fx_set_launch.argtypes = [vp, ctypes.POINTER(Launch)]
            L.fx_set_launch.restype = i32
            L.fx_get_launch.argtypes = [vp, ctypes.POINTER(Launch)]
            L.fx_get_launch.restype = i32
            L.fx_counters.argtypes = [vp, vp, vp, i32]
            L.fx_counters.restype = i32
            L.fx_stream_status.argtypes = [vp, vp, ctypes.POINTER(u32)]
            L.fx_stream_status.restype = i32
            L.fx_fma_peak.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double), vp]
            L.fx_fma_peak.restype = i32
            L.fx_last_error.argtypes = []
            L.fx_last_error.restype = ctypes.c_char_p
            L.fx_version.argtypes = []
            L.fx_version.restype = i32
            _lib = L
    return _lib


def _check(code):
    if code != FX_OK:
        raise FiberxError(code, lib().fx_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _dev(x, dtype, device):
    import torch
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    return x.to(device=device, dtype=dtype).contiguous()


class Fibers:
    """Device copy of fiber segments (fiber_upload).  ``cps``: [n_seg, 4, 4]
    float32 (x, y, z, r per control point) for cubic segments, or
    [n_seg, 3, 4] for quadratic ones (fiber_upload_quadratic), host or
    device."""

    def __init__(self, cps, max_presplit=8, thick_check=True, stream=None, device=None):
        import torch
        L = lib()
        if isinstance(cps, np.ndarray):
            cps = torch.from_numpy(np.ascontiguousarray(cps, dtype=np.float32))
        cps = cps.detach().to(torch.float32).contiguous()
        if cps.dim() != 3 or cps.shape[1:] not in ((4, 4), (3, 4)):
            raise ValueError("cps must be [n_seg, 4, 4] (cubic) or [n_seg, 3, 4] (quadratic)")
        self.quadratic = cps.shape[1] == 3
        upload = L.fiber_upload_quadratic if self.quadratic else L.fiber_upload
        self.device = torch.device(device) if device is not None else (
            cps.device if cps.is_cuda else torch.device("cuda", torch.cuda.current_device()))
        self.n_seg = int(cps.shape[0])
        opts = UploadOpts(int(max_presplit), int(bool(thick_check)))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(upload(_ptr(cps) if cps.numel() else None, self.n_seg, int(cps.is_cuda),
                          ctypes.byref(opts), _stream(stream), ctypes.byref(h)))
        self._h = h
        self._lib = L

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("fibers already freed")
        return self._h

    def info(self):
        inf = FibersInfo()
        _check(self._lib.fiber_info(self.handle, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in FibersInfo._fields_}

    def get_launch(self):
        c = Launch()
        _check(self._lib.fx_get_launch(self.handle, ctypes.byref(c)))
        return dict(block=c.block, blocks_per_sm=c.blocks_per_sm, chunk=c.chunk, variant=c.variant)

    def set_launch(self, block=128, blocks_per_sm=0, chunk=32, variant=0):
        _check(self._lib.fx_set_launch(self.handle, ctypes.byref(Launch(block, blocks_per_sm, chunk, variant))))

    def counters(self, reset=True, stream=None):
        out = np.zeros(5, dtype=np.uint64)
        _check(self._lib.fx_counters(self.handle, _stream(stream), out.ctypes.data_as(ctypes.c_void_p),
                                     int(reset)))
        return dict(zip(["nodes", "descents", "backtracks", "tests", "hits"], out.tolist()))

    def status(self, stream=None):
        v = ctypes.c_uint32(0)
        _check(self._lib.fx_stream_status(self.handle, _stream(stream), ctypes.byref(v)))
        return int(v.value)

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.fiber_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _inputs(fibers, rays, row_ptr, seg_idx):
    import torch
    dev = fibers.device
    rays = _dev(rays, torch.float32, dev)
    row_ptr = _dev(row_ptr, torch.int32, dev)
    seg_idx = _dev(seg_idx, torch.int32, dev)
    if rays.dim() != 2 or rays.shape[1] != 8:
        raise ValueError("rays must be [n_ray, 8]")
    if row_ptr.numel() != rays.shape[0] + 1:
        raise ValueError("row_ptr must have n_ray + 1 entries")
    return rays, row_ptr, seg_idx


def fma_peak(blocks_per_sm=4, iters=4096, stream=None):
    """Measured FP32 FMA throughput of the current device: (TFLOP/s, ms of
    the timed launch)."""
    ms, tf = ctypes.c_float(), ctypes.c_double()
    _check(lib().fx_fma_peak(blocks_per_sm, iters, ctypes.byref(ms), ctypes.byref(tf), _stream(stream)))
    return tf.value, ms.value


def _ray_depth(fibers, ray_depth, n_ray):
    """Per-ray depths as a device int8 tensor of n_ray entries, or None."""
    import torch
    if ray_depth is None:
        return None
    d = _dev(ray_depth, torch.int8, fibers.device)
    if d.numel() != n_ray:
        raise ValueError("ray_depth must have n_ray entries")
    return d


def intersect_closest(fibers, rays, row_ptr, seg_idx, depth, flags=0, leaf=True, stream=None,
                      out=None, ray_depth=None):
    """Closest hit per ray: returns (tu [n_ray, 2] f32, seg [n_ray] i32,
    leaf [n_ray] i32 or None).  ray_depth: optional per-ray depths (int8,
    n_ray) replacing ``depth`` ray by ray."""
    import torch
    rays, row_ptr, seg_idx = _inputs(fibers, rays, row_ptr, seg_idx)
    rd = _ray_depth(fibers, ray_depth, rays.shape[0])
    n_ray, n_pair = rays.shape[0], seg_idx.numel()
    if out is None:
        tu = torch.empty((n_ray, 2), dtype=torch.float32, device=fibers.device)
        seg = torch.empty(n_ray, dtype=torch.int32, device=fibers.device)
        lf = torch.empty(n_ray, dtype=torch.int32, device=fibers.device) if leaf else None
    else:
        tu, seg, lf = out
    _check(lib().intersect_closest(fibers.handle, _ptr(rays), n_ray, _ptr(row_ptr), _ptr(seg_idx), n_pair,
                                   int(depth), _ptr(rd), int(flags), _ptr(tu), _ptr(seg), _ptr(lf),
                                   _stream(stream)))
    return tu, seg, lf


def intersect_closest_noalloc(fibers, rays, row_ptr, seg_idx, depth, flags=0, out=None, stream=None):
    """intersect_closest on the one-thread-per-pair kernel without any device
    allocation inside the library: its per-ray scratch is a fixed 8 MiB device
    array shared by all calls (at most NOALLOC_MAX_RAYS rays; calls that
    overlap on the GPU race on it).  For callers that cannot allocate device
    memory while they run; pass preallocated ``out = (tu, seg, leaf)`` and
    device inputs so that this wrapper allocates nothing either."""
    import torch
    rays, row_ptr, seg_idx = _inputs(fibers, rays, row_ptr, seg_idx)
    n_ray, n_pair = rays.shape[0], seg_idx.numel()
    if out is None:
        tu = torch.empty((n_ray, 2), dtype=torch.float32, device=fibers.device)
        seg = torch.empty(n_ray, dtype=torch.int32, device=fibers.device)
        lf = torch.empty(n_ray, dtype=torch.int32, device=fibers.device)
    else:
        tu, seg, lf = out
    _check(lib().intersect_closest_noalloc(fibers.handle, _ptr(rays), n_ray, _ptr(row_ptr), _ptr(seg_idx),
                                           n_pair, int(depth), int(flags), _ptr(tu), _ptr(seg), _ptr(lf),
                                           _stream(stream)))
    return tu, seg, lf


def intersect_pairs(fibers, rays, row_ptr, seg_idx, depth, flags=0, leaf=True, stream=None, ray_depth=None,
                    pair_flags=False):
    """Per-pair hits: returns (tu [n_pair, 2], leaf [n_pair] or None), and
    with pair_flags=True also the FX_DEV_* bits of each pair [n_pair] uint8."""
    import torch
    rays, row_ptr, seg_idx = _inputs(fibers, rays, row_ptr, seg_idx)
    rd = _ray_depth(fibers, ray_depth, rays.shape[0])
    n_ray, n_pair = rays.shape[0], seg_idx.numel()
    tu = torch.empty((n_pair, 2), dtype=torch.float32, device=fibers.device)
    lf = torch.empty(n_pair, dtype=torch.int32, device=fibers.device) if leaf else None
    pf = torch.empty(n_pair, dtype=torch.uint8, device=fibers.device) if pair_flags else None
    _check(lib().intersect_pairs(fibers.handle, _ptr(rays), n_ray, _ptr(row_ptr), _ptr(seg_idx), n_pair,
                                 int(depth), _ptr(rd), int(flags), _ptr(tu), _ptr(lf), _ptr(pf), _stream(stream)))
    return (tu, lf, pf) if pair_flags else (tu, lf)


def intersect_counts(fibers, rays, row_ptr, seg_idx, depth, boxes=False, flags=0, stream=None):
    """Per-ray pruning-test counts [n_ray] uint32 as int64 (Fig. 8): oriented
    cylinders, or ray-frame axis-aligned boxes with boxes=True."""
    import torch
    rays, row_ptr, seg_idx = _inputs(fibers, rays, row_ptr, seg_idx)
    n = torch.zeros(rays.shape[0], dtype=torch.int32, device=fibers.device)
    _check(lib().intersect_counts(fibers.handle, _ptr(rays), rays.shape[0], _ptr(row_ptr), _ptr(seg_idx),
                                  seg_idx.numel(), int(depth), int(flags) | (FX_COUNT_BOXES if boxes else 0),
                                  _ptr(n), _stream(stream)))
    return n.to(torch.int64) & 0xffffffff


def intersect_normals(fibers, rays, tu, seg, leaf, depth, flags=0, stream=None, out=None, ray_depth=None):
    """Unit surface normals [n_ray, 3] at the closest hits (tu, seg, leaf from
    intersect_closest at `depth` and `ray_depth`); zero for misses."""
    import torch
    dev = fibers.device
    rays = _dev(rays, torch.float32, dev)
    tu = _dev(tu, torch.float32, dev)
    seg = _dev(seg, torch.int32, dev)
    leaf = _dev(leaf, torch.int32, dev)
    rd = _ray_depth(fibers, ray_depth, rays.shape[0])
    n = out if out is not None else torch.empty((rays.shape[0], 3), dtype=torch.float32, device=dev)
    _check(lib().intersect_normals(fibers.handle, _ptr(rays), rays.shape[0], _ptr(tu), _ptr(seg), _ptr(leaf),
                                   int(depth), _ptr(rd), int(flags), _ptr(n), _stream(stream)))
    return n


def intersect_backward(fibers, rays, tu, seg, grad_t, grad_cps=None, stream=None):
    """dL/d(cps) for L with dL/dt = grad_t; returns (grad_cps [n_seg, 4, 4],
    or [n_seg, 3, 4] for quadratic fibers, number of skipped singular hits as
    a device tensor)."""
    import torch
    dev = fibers.device
    rays = _dev(rays, torch.float32, dev)
    tu = _dev(tu, torch.float32, dev)
    seg = _dev(seg, torch.int32, dev)
    grad_t = _dev(grad_t, torch.float32, dev)
    if grad_cps is None:
        grad_cps = torch.zeros((fibers.n_seg, 3 if fibers.quadratic else 4, 4), dtype=torch.float32, device=dev)
    skipped = torch.zeros(1, dtype=torch.int64, device=dev)
    _check(lib().intersect_backward(fibers.handle, _ptr(rays), rays.shape[0], _ptr(tu), _ptr(seg),
                                    _ptr(grad_t), _ptr(grad_cps), _ptr(skipped), _stream(stream)))
    return grad_cps, skipped


def intersect_closest_host(fibers, rays, row_ptr, seg_idx, depth, flags=0, out=None, stream=None,
                           ray_depth=None):
    """intersect_closest on host (numpy or CPU torch, ideally pinned) buffers;
    returns host (tu, seg, leaf) and synchronises."""
    import torch

    def host(x, dt):
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x))
        return x.to(dtype=dt).contiguous()

    rays, row_ptr, seg_idx = host(rays, torch.float32), host(row_ptr, torch.int32), host(seg_idx, torch.int32)
    n_ray, n_pair = rays.shape[0], seg_idx.numel()
    rd = host(ray_depth, torch.int8) if ray_depth is not None else None
    if rd is not None and rd.numel() != n_ray:
        raise ValueError("ray_depth must have n_ray entries")
    if out is None:
        out = (torch.empty((n_ray, 2), dtype=torch.float32), torch.empty(n_ray, dtype=torch.int32),
               torch.empty(n_ray, dtype=torch.int32))
    tu, seg, lf = out
    _check(lib().intersect_closest_host(fibers.handle, _ptr(rays), n_ray, _ptr(row_ptr), _ptr(seg_idx),
                                        n_pair, int(depth), _ptr(rd), int(flags), _ptr(tu), _ptr(seg), _ptr(lf),
                                        _stream(stream)))
    return tu, seg, lf


def host_bytes(fibers):
    """(h2d, d2h): bytes the last intersect_closest_host call on ``fibers``
    copied each way."""
    h2d, d2h = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().fx_host_bytes(fibers.handle, ctypes.byref(h2d), ctypes.byref(d2h)))
    return int(h2d.value), int(d2h.value)


def _autograd():
    import torch

    class FiberIntersect(torch.autograd.Function):
        """Closest hit t (differentiable in the control points) with u and the
        hit segment: ``t, u, seg = FiberIntersect.apply(cps, rays, row_ptr,
        seg_idx, depth, fibers)``.  ``fibers`` must hold an upload of the same
        ``cps`` values; the backward pass is the hand-written adjoint kernel."""

        @staticmethod
        def forward(ctx, cps, rays, row_ptr, seg_idx, depth, fibers, flags=0):
            rays, row_ptr, seg_idx = _inputs(fibers, rays, row_ptr, seg_idx)
            tu, seg, _ = intersect_closest(fibers, rays, row_ptr, seg_idx, depth, flags=flags, leaf=False)
            ctx.fibers = fibers
            ctx.save_for_backward(rays, tu, seg)
            ctx.cps_shape = cps.shape
            t, u = tu[:, 0].clone(), tu[:, 1].clone()
            ctx.mark_non_differentiable(u, seg)
            return t, u, seg

        @staticmethod
        def backward(ctx, grad_t, grad_u, grad_seg):
            rays, tu, seg = ctx.saved_tensors
            if grad_t is None:
                return (None,) * 7
            g, _ = intersect_backward(ctx.fibers, rays, tu, seg, grad_t.float().contiguous())
            return g.reshape(ctx.cps_shape), None, None, None, None, None, None

    return FiberIntersect


_FI = None


def FiberIntersect():
    global _FI
    if _FI is None:
        _FI = _autograd()
    return _FI


def fiber_intersect(cps, rays, row_ptr, seg_idx, depth, fibers, flags=0):
    """Differentiable closest hit: returns (t, u, seg)."""
    return FiberIntersect().apply(cps, rays, row_ptr, seg_idx, depth, fibers, flags)
