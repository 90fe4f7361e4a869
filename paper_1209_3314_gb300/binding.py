"""Thin ctypes binding over libiwpp (``include/iwpp.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch supplies device memory and streams; tensors are passed as
raw device pointers with their row pitch.  There is no CPU fallback: if the
library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

IWPP_OK = 0
IWPP_EINVAL = -1
IWPP_ENOMEM = -2
IWPP_ECUDA = -3
IWPP_ETIMEOUT = -4
IWPP_EOVERFLOW = -5
IWPP_U8 = 0
IWPP_I32 = 1
IWPP_EDT_FEATURE_ZERO = 0
IWPP_EDT_FEATURE_NONZERO = 1
IWPP_EDT_EXACT_PROPAGATION = 2
IWPP_OP_RECON = 0
IWPP_OP_EDT = 1

# every function the header declares, with (restype, argtypes)
_vp = ctypes.c_void_p
_i32 = ctypes.c_int


class Image(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("pitch", ctypes.c_int64), ("dtype", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_uint64) for n in (
        "calls", "tiles_processed", "tiles_initial", "seeds", "pushes", "spills",
        "rescans", "relaunches", "rounds", "wait_ns", "visit_ns")] +
        [("phase_ns", ctypes.c_uint64 * 4)] +
        [(n, ctypes.c_uint64) for n in ("kernel_launches", "kernel_ns", "sweep_sets", "revisits")])


class Options(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("sweeps", ctypes.c_int32), ("queue_factor", ctypes.c_int32),
                ("spill_cap", ctypes.c_int32), ("max_relaunch", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("revisit_sweep_min", ctypes.c_int32), ("edt_sweeps", ctypes.c_int32),
                ("edt_revisit_sweep_min", ctypes.c_int32), ("revisit_sweeps", ctypes.c_int32),
                ("queue_mode", ctypes.c_int32), ("test_empty_slot", ctypes.c_int32),
                ("gdt_sweeps", ctypes.c_int32), ("batch_split", ctypes.c_int32),
                ("ws_sweeps", ctypes.c_int32), ("ws_revisit_sweep_min", ctypes.c_int32),
                ("gdt_revisit_sweep_min", ctypes.c_int32), ("edt_wide_step", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("conn", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("marker", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("sqdist", ctypes.c_void_p), ("nearest", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "batches", "pending",
                                                 "bytes_in_use", "peak_bytes_in_use", "workspace_bytes",
                                                 "pool_used_high", "records")]


class Job(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("conn", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("a", Image), ("b", Image), ("out", Image),
                ("sqdist", ctypes.c_void_p), ("nearest", ctypes.c_void_p)]


SIGNATURES = {
    "iwpp_version": (_i32, []),
    "iwpp_ctx_create": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.c_size_t]),
    "iwpp_ctx_destroy": (_i32, [_vp]),
    "iwpp_last_error": (ctypes.c_char_p, [_vp]),
    "iwpp_get_options": (_i32, [_vp, ctypes.POINTER(Options)]),
    "iwpp_set_options": (_i32, [_vp, ctypes.POINTER(Options)]),
    "iwpp_recon": (_i32, [_vp, ctypes.POINTER(Image), ctypes.POINTER(Image), _i32,
                          ctypes.POINTER(Image), _vp]),
    "iwpp_recon_async": (_i32, [_vp, ctypes.POINTER(Image), ctypes.POINTER(Image), _i32,
                                ctypes.POINTER(Image), _vp]),
    "iwpp_edt": (_i32, [_vp, ctypes.POINTER(Image), _vp, _vp, _i32, _vp]),
    "iwpp_edt_async": (_i32, [_vp, ctypes.POINTER(Image), _vp, _vp, _i32, _vp]),
    "iwpp_edt_exact": (_i32, [_vp, ctypes.POINTER(Image), _vp, _vp, _i32, _vp]),
    "iwpp_geodesic": (_i32, [_vp, ctypes.POINTER(Image), ctypes.POINTER(Image), _vp, _vp]),
    "iwpp_geodesic_async": (_i32, [_vp, ctypes.POINTER(Image), ctypes.POINTER(Image), _vp, _vp]),
    "iwpp_watershed": (_i32, [_vp, ctypes.POINTER(Image), ctypes.POINTER(Image), _vp, _vp, _vp]),
    "iwpp_skiz": (_i32, [_vp, ctypes.POINTER(Image), ctypes.POINTER(Image), _vp, _vp, _vp, _vp]),
    "iwpp_recon_batched": (_i32, [_vp, _i32, ctypes.POINTER(Image), ctypes.POINTER(Image), _i32,
                                  ctypes.POINTER(Image), _vp]),
    "iwpp_edt_batched": (_i32, [_vp, _i32, ctypes.POINTER(Image), ctypes.POINTER(_vp),
                                ctypes.POINTER(_vp), _i32, _vp]),
    "iwpp_run_jobs": (_i32, [_vp, _i32, ctypes.POINTER(Job), _vp]),
    "iwpp_run_jobs_async": (_i32, [_vp, _i32, ctypes.POINTER(Job), _vp]),
    "iwpp_submit": (_i32, [_vp, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)]),
    "iwpp_poll": (_i32, [_vp, ctypes.c_uint64, ctypes.POINTER(_i32)]),
    "iwpp_wait": (_i32, [_vp, ctypes.c_uint64, ctypes.POINTER(_i32)]),
    "iwpp_sync": (_i32, [_vp, _vp]),
    "iwpp_stats": (_i32, [_vp, ctypes.POINTER(Stats)]),
    "iwpp_stats_reset": (_i32, [_vp]),
    "iwpp_plan_create": (_i32, [_vp, _i32, ctypes.POINTER(Job), ctypes.POINTER(_vp)]),
    "iwpp_plan_launch": (_i32, [_vp, _vp]),
    "iwpp_plan_launch_graph": (_i32, [_vp, _vp]),
    "iwpp_plan_autotune": (_i32, [_vp, _vp, _i32, ctypes.POINTER(Options)]),
    "iwpp_plan_destroy": (_i32, [_vp]),
    "iwpp_server_create": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.c_size_t, _i32, _i32]),
    "iwpp_server_submit": (_i32, [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "iwpp_server_poll": (_i32, [_vp, ctypes.c_uint64, ctypes.POINTER(_i32)]),
    "iwpp_server_wait": (_i32, [_vp, ctypes.c_uint64, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double)]),
    "iwpp_server_stats": (_i32, [_vp, ctypes.POINTER(ServerStats)]),
    "iwpp_server_destroy": (_i32, [_vp]),
    "iwpp_recon_u8_noalloc": (_i32, [_vp, ctypes.c_int64, _vp, ctypes.c_int64, _vp, ctypes.c_int64,
                                     _i32, _i32, _i32, _vp]),
}

_lib = None


def load_library(path: str | None = None):
    """Loads libiwpp.so (built by ``paper_1209_3314_gb300.build``).  Raises if
    it is missing: there is no fallback implementation."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise ImportError(f"libiwpp not built ({p} missing); run paper_1209_3314_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class IWPPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"iwpp error {code}: {msg}")
        self.code = code


def _torch():
    import torch
    return torch


def image_of(t) -> Image:
    """Describes a 2-D CUDA tensor (uint8 or int32, unit column stride)."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2-D tensor with unit column stride")
    if t.dtype == torch.uint8:
        dt = IWPP_U8
    elif t.dtype == torch.int32:
        dt = IWPP_I32
    else:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return Image(t.data_ptr(), t.shape[0], t.shape[1], max(t.stride(0), t.shape[1]), dt)


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def recon_u8_noalloc(marker, mask, conn: int = 8, out=None, stream=None):
    """uint8 reconstruction through the allocation-free entry point (no
    context; library-internal static scratch).  ``out`` must be supplied by
    callers that cannot allocate; when omitted a tensor is created here."""
    torch = _torch()
    lib = load_library()
    if out is None:
        out = torch.empty_like(mask)
    m, k, o = image_of(marker), image_of(mask), image_of(out)
    if not (m.dtype == k.dtype == o.dtype == IWPP_U8):
        raise TypeError("uint8 images required")
    if (m.h, m.w) != (k.h, k.w) or (o.h, o.w) != (k.h, k.w):
        raise ValueError("marker, mask and out must have the same shape")
    rc = lib.iwpp_recon_u8_noalloc(m.data, m.pitch, k.data, k.pitch, o.data, o.pitch, k.h, k.w, conn,
                                   _stream_ptr(stream))
    if rc != IWPP_OK:
        raise IWPPError(rc, "iwpp_recon_u8_noalloc failed")
    return out


class Context:
    """An iwpp context on one device: owns the library workspace."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self.lib = load_library()
        h = ctypes.c_void_p()
        rc = self.lib.iwpp_ctx_create(ctypes.byref(h), device, hbm_budget)
        if rc != IWPP_OK:
            raise IWPPError(rc, "iwpp_ctx_create failed")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.iwpp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != IWPP_OK:
            raise IWPPError(rc, self.lib.iwpp_last_error(self.h).decode())

    # ---- options / stats
    def options(self) -> dict:
        o = Options()
        self._check(self.lib.iwpp_get_options(self.h, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in Options._fields_ if k != "reserved"}

    def set_options(self, **kw):
        o = Options()
        self._check(self.lib.iwpp_get_options(self.h, ctypes.byref(o)))
        for k, v in kw.items():
            if k == "reserved" or not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, int(v))
        self._check(self.lib.iwpp_set_options(self.h, ctypes.byref(o)))

    def stats(self) -> dict:
        s = Stats()
        self._check(self.lib.iwpp_stats(self.h, ctypes.byref(s)))
        d = {k: getattr(s, k) for k, _ in Stats._fields_}
        d["phase_ns"] = [int(v) for v in s.phase_ns]
        return {k: (v if isinstance(v, list) else int(v)) for k, v in d.items()}

    def stats_reset(self):
        self._check(self.lib.iwpp_stats_reset(self.h))

    def sync(self, stream=None):
        self._check(self.lib.iwpp_sync(self.h, _stream_ptr(stream)))

    # ---- operations
    def recon(self, marker, mask, conn: int = 8, out=None, stream=None, sync: bool = True):
        """Reconstruction by dilation of ``mask`` from ``marker`` (CUDA
        tensors, uint8 or int32).  Returns ``out`` (new tensor unless given;
        ``out=marker`` reconstructs in place)."""
        torch = _torch()
        if out is None:
            out = torch.empty_like(mask)
        m, k, o = image_of(marker), image_of(mask), image_of(out)
        fn = self.lib.iwpp_recon if sync else self.lib.iwpp_recon_async
        self._check(fn(self.h, ctypes.byref(m), ctypes.byref(k), conn, ctypes.byref(o),
                       _stream_ptr(stream)))
        return out

    def edt(self, binary, feature_nonzero: bool = False, sqdist=None, nearest=None,
            stream=None, sync: bool = True, exact: bool = False, exact_propagation: bool = False):
        """Distance transform of a uint8 CUDA tensor.  Returns
        (sqdist int32, nearest int32 linear index).  exact=True runs the
        exact separable transform (iwpp_edt_exact, synchronous) instead of
        the propagation method; exact_propagation=True adds the wide-window
        second wavefront (IWPP_EDT_EXACT_PROPAGATION)."""
        torch = _torch()
        h, w = binary.shape
        if sqdist is None:
            sqdist = torch.empty((h, w), dtype=torch.int32, device=binary.device)
        if nearest is None:
            nearest = torch.empty((h, w), dtype=torch.int32, device=binary.device)
        for t in (sqdist, nearest):
            if t.dtype != torch.int32 or tuple(t.shape) != (h, w) or not t.is_contiguous() or not t.is_cuda:
                raise ValueError("sqdist/nearest must be contiguous int32 CUDA tensors of the image shape")
        b = image_of(binary)
        fn = self.lib.iwpp_edt_exact if exact else (self.lib.iwpp_edt if sync else self.lib.iwpp_edt_async)
        flags = IWPP_EDT_FEATURE_NONZERO if feature_nonzero else IWPP_EDT_FEATURE_ZERO
        if exact_propagation:
            flags |= IWPP_EDT_EXACT_PROPAGATION
        self._check(fn(self.h, ctypes.byref(b), ctypes.c_void_p(sqdist.data_ptr()),
                       ctypes.c_void_p(nearest.data_ptr()), flags, _stream_ptr(stream)))
        return sqdist, nearest

    def geodesic(self, mask, seeds, dist=None, stream=None, sync: bool = True):
        """Shortest-path distance through free pixels (mask != 0) from the
        sources (free pixels with seeds != 0): uint8 CUDA tensors of one
        shape.  8 moves, cost 5 straight / 7 diagonal.  Returns dist (int32;
        INT32_MAX at obstacles and unreachable pixels)."""
        torch = _torch()
        h, w = mask.shape
        if dist is None:
            dist = torch.empty((h, w), dtype=torch.int32, device=mask.device)
        if dist.dtype != torch.int32 or tuple(dist.shape) != (h, w) or not dist.is_contiguous() or not dist.is_cuda:
            raise ValueError("dist must be a contiguous int32 CUDA tensor of the image shape")
        m, s = image_of(mask), image_of(seeds)
        fn = self.lib.iwpp_geodesic if sync else self.lib.iwpp_geodesic_async
        self._check(fn(self.h, ctypes.byref(m), ctypes.byref(s), ctypes.c_void_p(dist.data_ptr()),
                       _stream_ptr(stream)))
        return dist

    def watershed(self, relief, markers, labels=None, levels=None, with_levels: bool = False,
                  stream=None):
        """Watershed from markers: relief (uint8 or int32 CUDA tensor),
        markers (int32 CUDA tensor of the same shape, 0 = no marker).
        Returns labels (int32), or (labels, levels) with with_levels (levels
        in the relief's dtype: the flooding level of each pixel)."""
        torch = _torch()
        h, w = relief.shape
        if labels is None:
            labels = torch.empty((h, w), dtype=torch.int32, device=relief.device)
        if with_levels and levels is None:
            levels = torch.empty((h, w), dtype=relief.dtype, device=relief.device)
        if labels.dtype != torch.int32 or tuple(labels.shape) != (h, w) or not labels.is_contiguous() \
                or not labels.is_cuda:
            raise ValueError("labels must be a contiguous int32 CUDA tensor of the image shape")
        if levels is not None and (levels.dtype != relief.dtype or tuple(levels.shape) != (h, w)
                                   or not levels.is_contiguous() or not levels.is_cuda):
            raise ValueError("levels must be a contiguous CUDA tensor of the relief's dtype and shape")
        f, m = image_of(relief), image_of(markers)
        lv = ctypes.c_void_p(levels.data_ptr()) if levels is not None else None
        self._check(self.lib.iwpp_watershed(self.h, ctypes.byref(f), ctypes.byref(m),
                                            ctypes.c_void_p(labels.data_ptr()), lv, _stream_ptr(stream)))
        return (labels, levels) if levels is not None else labels

    def skiz(self, mask, labels, with_dist: bool = False, stream=None):
        """Influence zones of labelled sources (free pixels with labels != 0;
        mask uint8, labels int32 CUDA tensors of one shape) and their
        skeleton.  Returns (zones int32, skiz uint8) or, with with_dist,
        (zones, skiz, dist int32)."""
        torch = _torch()
        h, w = mask.shape
        zones = torch.empty((h, w), dtype=torch.int32, device=mask.device)
        sk = torch.empty((h, w), dtype=torch.uint8, device=mask.device)
        dist = torch.empty((h, w), dtype=torch.int32, device=mask.device) if with_dist else None
        m, lab = image_of(mask), image_of(labels)
        self._check(self.lib.iwpp_skiz(self.h, ctypes.byref(m), ctypes.byref(lab),
                                       ctypes.c_void_p(zones.data_ptr()), ctypes.c_void_p(sk.data_ptr()),
                                       ctypes.c_void_p(dist.data_ptr()) if dist is not None else None,
                                       _stream_ptr(stream)))
        return (zones, sk, dist) if with_dist else (zones, sk)

    def recon_batched(self, markers, masks, conn: int = 8, outs=None, stream=None):
        torch = _torch()
        n = len(markers)
        if outs is None:
            outs = [torch.empty_like(m) for m in masks]
        M = (Image * n)(*[image_of(t) for t in markers])
        K = (Image * n)(*[image_of(t) for t in masks])
        O = (Image * n)(*[image_of(t) for t in outs])
        self._check(self.lib.iwpp_recon_batched(self.h, n, M, K, conn, O, _stream_ptr(stream)))
        return outs

    def edt_batched(self, bins, feature_nonzero: bool = False, stream=None):
        torch = _torch()
        n = len(bins)
        sq = [torch.empty(b.shape, dtype=torch.int32, device=b.device) for b in bins]
        nn = [torch.empty(b.shape, dtype=torch.int32, device=b.device) for b in bins]
        B = (Image * n)(*[image_of(t) for t in bins])
        S = (ctypes.c_void_p * n)(*[t.data_ptr() for t in sq])
        N = (ctypes.c_void_p * n)(*[t.data_ptr() for t in nn])
        flags = IWPP_EDT_FEATURE_NONZERO if feature_nonzero else IWPP_EDT_FEATURE_ZERO
        self._check(self.lib.iwpp_edt_batched(self.h, n, B, S, N, flags, _stream_ptr(stream)))
        return list(zip(sq, nn))

    def plan(self, jobs):
        """Prepares a fixed batch (see ``run_jobs`` for the job dicts) for
        repeated, graph-capturable launches."""
        return Plan(self, jobs)

    def run_jobs(self, jobs, stream=None, sync: bool = True):
        """Mixed batch in one launch.  ``jobs``: list of dicts, either
        {'op': 'recon', 'marker', 'mask', 'out', 'conn'} or
        {'op': 'edt', 'binary', 'sqdist', 'nearest', 'feature_nonzero'}."""
        n = len(jobs)
        arr = _job_array(jobs)
        fn = self.lib.iwpp_run_jobs if sync else self.lib.iwpp_run_jobs_async
        self._check(fn(self.h, n, arr, _stream_ptr(stream)))


    # ---- asynchronous jobs with tickets (the context's own stream)
    def submit(self, job) -> int:
        """Enqueues one job (a dict as for ``run_jobs``) on the context's own
        stream and returns its ticket at once.  The job's tensors are kept
        alive until the ticket is retired by ``poll`` or ``wait``."""
        arr = _job_array([job])
        t = ctypes.c_uint64(0)
        self._check(self.lib.iwpp_submit(self.h, arr, ctypes.byref(t)))
        self.__dict__.setdefault("_submitted", {})[t.value] = job
        return t.value

    def poll(self, ticket: int):
        """None while the job runs; its outcome code (0 = IWPP_OK) once it
        has finished (the ticket is then retired)."""
        st = ctypes.c_int(0)
        rc = self.lib.iwpp_poll(self.h, ticket, ctypes.byref(st))
        if rc < 0:
            self._check(rc)
        if rc == 0:
            return None
        self.__dict__.get("_submitted", {}).pop(ticket, None)
        return st.value

    def wait(self, ticket: int) -> int:
        """Blocks until the job has finished; returns its outcome code."""
        st = ctypes.c_int(0)
        self._check(self.lib.iwpp_wait(self.h, ticket, ctypes.byref(st)))
        self.__dict__.get("_submitted", {}).pop(ticket, None)
        return st.value


def _job_array(jobs):
    n = len(jobs)
    arr = (Job * n)()
    for i, j in enumerate(jobs):
        if j["op"] == "recon":
            arr[i].op = IWPP_OP_RECON
            arr[i].conn = int(j.get("conn", 8))
            arr[i].a = image_of(j["marker"])
            arr[i].b = image_of(j["mask"])
            arr[i].out = image_of(j["out"])
        else:
            arr[i].op = IWPP_OP_EDT
            arr[i].flags = ((IWPP_EDT_FEATURE_NONZERO if j.get("feature_nonzero") else 0) |
                            (IWPP_EDT_EXACT_PROPAGATION if j.get("exact_propagation") else 0))
            arr[i].a = image_of(j["binary"])
            arr[i].sqdist = j["sqdist"].data_ptr()
            arr[i].nearest = j["nearest"].data_ptr()
    return arr


class Plan:
    """A batch prepared once (C ``iwpp_plan``): launches enqueue kernels only
    and can be replayed as a CUDA graph."""

    def __init__(self, ctx: "Context", jobs):
        self.ctx = ctx
        self.jobs = list(jobs)  # keeps the tensors alive
        arr = _job_array(self.jobs)
        h = ctypes.c_void_p()
        ctx._check(ctx.lib.iwpp_plan_create(ctx.h, len(self.jobs), arr, ctypes.byref(h)))
        self.h = h

    def launch(self, stream=None, graph: bool = False):
        fn = self.ctx.lib.iwpp_plan_launch_graph if graph else self.ctx.lib.iwpp_plan_launch
        self.ctx._check(fn(self.h, _stream_ptr(stream)))

    def autotune(self, reps: int = 3, stream=None) -> dict:
        o = Options()
        self.ctx._check(self.ctx.lib.iwpp_plan_autotune(self.h, _stream_ptr(stream), reps, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in Options._fields_ if k != "reserved"}

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.iwpp_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (C ``iwpp_server``).  Requests
    carry host (CPU) tensors, ideally pinned; results land in the request's
    output tensors.  The tensors must stay alive until the request is done."""

    def __init__(self, device: int = 0, hbm_budget: int = 120 << 30, streams: int = 3, max_batch: int = 64):
        self.lib = load_library()
        h = ctypes.c_void_p()
        rc = self.lib.iwpp_server_create(ctypes.byref(h), device, hbm_budget, streams, max_batch)
        if rc != IWPP_OK:
            raise IWPPError(rc, "iwpp_server_create failed")
        self.h = h
        self._keep = {}

    def submit_recon(self, marker, mask, out, conn: int = 8) -> int:
        import numpy as np  # noqa: F401

        r = Request()
        r.op, r.conn = IWPP_OP_RECON, conn
        r.dtype = IWPP_U8 if marker.dtype.itemsize == 1 else IWPP_I32
        r.h, r.w = marker.shape
        r.marker, r.mask, r.out = marker.data_ptr(), mask.data_ptr(), out.data_ptr()
        return self._submit(r, (marker, mask, out))

    def submit_edt(self, binary, sqdist, nearest, feature_nonzero: bool = False) -> int:
        r = Request()
        r.op = IWPP_OP_EDT
        r.flags = IWPP_EDT_FEATURE_NONZERO if feature_nonzero else 0
        r.h, r.w = binary.shape
        r.marker, r.sqdist, r.nearest = binary.data_ptr(), sqdist.data_ptr(), nearest.data_ptr()
        return self._submit(r, (binary, sqdist, nearest))

    def _submit(self, r, keep):
        for t in keep:
            if t.device.type != "cpu" or not t.is_contiguous():
                raise ValueError("server requests take contiguous host tensors")
        t = ctypes.c_uint64()
        rc = self.lib.iwpp_server_submit(self.h, ctypes.byref(r), ctypes.byref(t))
        if rc != IWPP_OK:
            raise IWPPError(rc, "iwpp_server_submit failed")
        self._keep[t.value] = keep
        return t.value

    def wait(self, ticket: int):
        """Returns (status, latency_ms)."""
        st = ctypes.c_int()
        lat = ctypes.c_double()
        rc = self.lib.iwpp_server_wait(self.h, ticket, ctypes.byref(st), ctypes.byref(lat))
        if rc != IWPP_OK:
            raise IWPPError(rc, "iwpp_server_wait failed")
        self._keep.pop(ticket, None)
        return st.value, lat.value

    def stats(self) -> dict:
        s = ServerStats()
        self.lib.iwpp_server_stats(self.h, ctypes.byref(s))
        return {k: int(getattr(s, k)) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.iwpp_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
