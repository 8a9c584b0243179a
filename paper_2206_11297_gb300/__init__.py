"""Python binding of libroibin, the GB300 ROIBIN-SZ compression library.

This module only marshals arguments: every step of the method runs in the CUDA
kernels behind the C ABI of include/roibin.h.  PyTorch supplies device memory
and streams.  There is no fallback: if the CUDA library is missing or cannot be
loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

__all__ = ["Geometry", "Params", "Context", "library", "default_params", "validate",
           "compress_bound", "status_string", "GEOMETRIES", "PATH_AUTO", "PATH_PLAIN",
           "PATH_FUSED", "DEC_AUTO", "DEC_PANEL", "DEC_MULTIPASS", "EXPORTED_SYMBOLS",
           "compress_frame_static", "STATIC_SCRATCH_BYTES", "Job", "Graph"]

OK = 0
ERR_INVALID_ARG = -1
ERR_CAPACITY = -2
ERR_CORRUPT_STREAM = -3
ERR_OUT_OF_BUDGET = -4
ERR_CUDA = -5
ERR_TIMEOUT = -6
ERR_CODE_LENGTH = -7
ERR_CHECK = -8
REJECTED = 1  # per-frame status: non-hit rejection, nothing written

PATH_AUTO, PATH_PLAIN, PATH_FUSED = 0, 1, 2
DEC_AUTO, DEC_PANEL, DEC_MULTIPASS = 0, 1, 2
GRAPH_SERIAL, GRAPH_CONCURRENT, GRAPH_FUSED = 0, 1, 2

GEOMETRIES = {"cspad": (32, 185, 388), "epix10k": (16, 352, 384), "jungfrau": (8, 512, 1024)}


class Geometry(ctypes.Structure):
    _fields_ = [("n_panels", ctypes.c_uint32), ("rows", ctypes.c_uint32), ("cols", ctypes.c_uint32)]


class Params(ctypes.Structure):
    _fields_ = [
        ("amax_thr", ctypes.c_float), ("atot_thr", ctypes.c_float),
        ("son_min", ctypes.c_float), ("pix_nsigma", ctypes.c_float),
        ("rank", ctypes.c_int32), ("ring_r0", ctypes.c_int32), ("ring_dr", ctypes.c_int32),
        ("npix_min", ctypes.c_int32), ("npix_max", ctypes.c_int32),
        ("roi_h", ctypes.c_int32), ("roi_w", ctypes.c_int32),
        ("bin_h", ctypes.c_int32), ("bin_w", ctypes.c_int32),
        ("abs_eb", ctypes.c_float), ("quant_radius", ctypes.c_int32), ("max_peaks", ctypes.c_int32),
        ("lorenzo_dims", ctypes.c_int32), ("nhr_min_peaks", ctypes.c_int32), ("roi_coder", ctypes.c_int32),
        ("chunk_frames", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_u32, _i32, _u64 = ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64
_G, _Pr = ctypes.POINTER(Geometry), ctypes.POINTER(Params)


class Job(ctypes.Structure):
    """One job of a graph (roibin_job): a context and the arguments of its compress call."""
    _fields_ = [("ctx", ctypes.c_void_p), ("d_frames", ctypes.c_void_p), ("n_frames", ctypes.c_uint32),
                ("d_peaks", ctypes.c_void_p), ("d_npeaks", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
                ("out_stride", ctypes.c_uint64), ("d_frame_bytes", ctypes.c_void_p),
                ("d_frame_status", ctypes.c_void_p)]


# name -> (restype, argtypes); every symbol include/roibin.h declares
_SIGNATURES = {
    "roibin_default_params": (ctypes.c_int, [_Pr]),
    "roibin_validate": (ctypes.c_int, [_G, _Pr]),
    "roibin_compress_bound": (_u64, [_G, _Pr]),
    "roibin_ctx_create": (ctypes.c_int, [ctypes.POINTER(_P), _G, _Pr, _u32, _u64, ctypes.c_int]),
    "roibin_ctx_destroy": (ctypes.c_int, [_P]),
    "roibin_ctx_scratch_bytes": (_u64, [_P]),
    "roibin_ctx_set_path": (ctypes.c_int, [_P, ctypes.c_int]),
    "roibin_ctx_resolved_path": (ctypes.c_int, [_P]),
    "roibin_ctx_set_decompress_path": (ctypes.c_int, [_P, ctypes.c_int]),
    "roibin_ctx_set_plain_shape": (ctypes.c_int, [_P, _u32, _u32]),
    "roibin_ctx_set_fused_dense_peaks": (ctypes.c_int, [_P, ctypes.c_int]),
    "roibin_ctx_fused_dense_peaks": (ctypes.c_int, [_P]),
    "roibin_ctx_plain_shape": (ctypes.c_int, [_P, ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    "roibin_graph_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Job), _u32, ctypes.c_int]),
    "roibin_graph_launch": (ctypes.c_int, [_P, _P]),
    "roibin_graph_launch_count": (ctypes.c_int, [_P]),
    "roibin_graph_destroy": (ctypes.c_int, [_P]),
    "roibin_ctx_resolved_decompress_path": (ctypes.c_int, [_P]),
    "roibin_ctx_set_fused_shape": (ctypes.c_int, [_P, _u32, _u32, _u32]),
    "roibin_ctx_fused_shape": (ctypes.c_int, [_P] + [ctypes.POINTER(_u32)] * 5),
    "roibin_ctx_set_trace": (ctypes.c_int, [_P, _P, _u32]),
    "roibin_ctx_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_int64]),
    "roibin_ctx_debug_status": (ctypes.c_int, [_P, ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                                               ctypes.POINTER(_u32), ctypes.POINTER(_u64)]),
    "roibin_ctx_debug_poke_guard": (ctypes.c_int, [_P, _u32]),
    "roibin_compress": (ctypes.c_int, [_P, _P, _u32, _P, _P, _P, _u64, _P, _P, _P]),
    "roibin_decompress": (ctypes.c_int, [_P, _P, _u64, _P, _u32, _P, _P, _P]),
    "roibin_ctx_reserve_host_path": (ctypes.c_int, [_P]),
    "roibin_compress_host": (ctypes.c_int, [_P, _P, _u32, _P, _u64, _P, _P, _P]),
    "roibin_roi_mask": (ctypes.c_int, [_P, _P, _P, _u32, _P, _P]),
    "roibin_last_peaks": (ctypes.c_int, [_P, _P, _P, _u32, _P]),
    "roibin_ctx_enable_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "roibin_ctx_kernel_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_char_p),
                                               ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_uint32), ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)]),
    "roibin_ctx_last_launch_count": (_u32, [_P]),
    "roibin_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "roibin_compress_frame_static": (ctypes.c_int, [_G, _Pr, _P, _P, _P, _P, _u64, _P, _P, _P]),
    "roibin_ctx_autotune": (ctypes.c_int, [_P, _P, _u32, _P, _u64, _P, _P, _P, ctypes.POINTER(ctypes.c_float)]),
}
EXPORTED_SYMBOLS = sorted(_SIGNATURES)

_lib = None


def checks_requested() -> bool:
    """ROIBIN_CHECKS=1 in the environment selects the checks build of the library."""
    return os.environ.get("ROIBIN_CHECKS", "") not in ("", "0")


def library(build_if_needed: bool = True):
    """Loads libroibin.so (libroibin_checks.so when ROIBIN_CHECKS=1), building
    it first if asked; raises if unavailable."""
    global _lib
    if _lib is None:
        checks = checks_requested()
        path = _build.LIB_CHECKS if checks else _build.LIB
        if build_if_needed and not _build.up_to_date(checks):
            _build.build(checks=checks)
        if not os.path.exists(path):
            raise RuntimeError(f"libroibin.so is not built ({path}); run __graft_entry__.build()")
        try:
            import torch  # noqa: F401  (load PyTorch's CUDA runtime first; the library shares it)
        except ImportError:
            pass
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def status_string(code: int) -> str:
    return library().roibin_status_string(code).decode()


class RoibinError(RuntimeError):
    def __init__(self, where: str, code: int):
        super().__init__(f"{where}: {status_string(code)} ({code})")
        self.code = code


def _check(where, code):
    if code != OK:
        raise RoibinError(where, code)


def default_params(**overrides) -> Params:
    p = Params()
    _check("roibin_default_params", library().roibin_default_params(ctypes.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def validate(geometry, params: Params) -> int:
    g = Geometry(*geometry)
    return library().roibin_validate(ctypes.byref(g), ctypes.byref(params))


def compress_bound(geometry, params: Params) -> int:
    g = Geometry(*geometry)
    return int(library().roibin_compress_bound(ctypes.byref(g), ctypes.byref(params)))


STATIC_SCRATCH_BYTES = 16 << 20


def compress_frame_static(geometry, params: Params, frame, out, frame_bytes, status, peaks=None,
                          npeaks=None, stream=None):
    """roibin_compress_frame_static: one CUDA float32 [P, H, W] frame into the caller's
    buffers (out u8 [capacity], frame_bytes int64 [1], status int32 [1]) with the
    library's static scratch; allocates nothing.  Asynchronous on `stream`.
    peaks (int16/uint16 [max_peaks, 3]) and npeaks (int32/uint32 [1]) optionally
    replace the peak finder, as in Context.compress."""
    import torch
    geometry = tuple(int(x) for x in geometry)
    # the kernels index these buffers by the geometry and dtypes below: a
    # mismatch would make them read or write out of bounds, so it is refused here
    assert frame.dtype == torch.float32 and frame.is_cuda and frame.is_contiguous(), "frame: contiguous CUDA float32"
    assert tuple(frame.shape) == geometry, f"frame shape {tuple(frame.shape)} is not the geometry {geometry}"
    dev = frame.device
    assert out.dtype == torch.uint8 and out.is_contiguous() and out.device == dev, "out: contiguous uint8 on the frame's device"
    assert frame_bytes.dtype == torch.int64 and frame_bytes.numel() >= 1 and frame_bytes.device == dev
    assert status.dtype == torch.int32 and status.numel() >= 1 and status.device == dev
    assert (peaks is None) == (npeaks is None), "peaks and npeaks go together"
    if peaks is not None:
        mp = max(int(params.max_peaks), 1)
        assert peaks.dtype in (torch.int16, torch.uint16) and peaks.is_contiguous() and peaks.device == dev
        assert peaks.numel() >= 3 * mp, "peaks must hold max_peaks (panel, row, col) triples"
        assert npeaks.dtype in (torch.int32, torch.uint32) and npeaks.numel() >= 1 and npeaks.device == dev
    g = Geometry(*geometry)
    with torch.cuda.device(dev):
        _check("roibin_compress_frame_static", library().roibin_compress_frame_static(
            ctypes.byref(g), ctypes.byref(params), _ptr(frame), _ptr(peaks), _ptr(npeaks), _ptr(out),
            out.numel() // 16 * 16, _ptr(frame_bytes), _ptr(status), _stream_handle(stream)))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """One compression context: geometry, parameters and preallocated scratch."""

    def __init__(self, geometry, params: Params | None = None, max_frames: int = 1,
                 hbm_budget: int = 0, device: int = 0):
        self.lib = library()
        self.geometry = tuple(int(x) for x in geometry)
        self.params = params if params is not None else default_params()
        self.max_frames = int(max_frames)
        self.device = int(device)
        g = Geometry(*self.geometry)
        h = ctypes.c_void_p()
        _check("roibin_ctx_create", self.lib.roibin_ctx_create(
            ctypes.byref(h), ctypes.byref(g), ctypes.byref(self.params), self.max_frames,
            int(hbm_budget), self.device))
        self._h = h

    @property
    def n_bins(self) -> int:
        """Bins per frame: P * ceil(rows / bin_h) * ceil(cols / bin_w)."""
        P, H, W = self.geometry
        bh, bw = int(self.params.bin_h), int(self.params.bin_w)
        return P * (-(-H // bh)) * (-(-W // bw))

    # -- lifetime
    def close(self):
        """Frees the context.  In the checks build a failed device check or an
        overwritten guard band raises RoibinError(ERR_CHECK) here."""
        if getattr(self, "_h", None):
            h, self._h = self._h, None
            _check("roibin_ctx_destroy", self.lib.roibin_ctx_destroy(h))

    def debug_status(self):
        """roibin_ctx_debug_status: (status, checks_build, first_check, failed, bad_guard)."""
        cb, first, failed, bad = _u32(), _u32(), _u32(), _u64()
        st = self.lib.roibin_ctx_debug_status(self._h, ctypes.byref(cb), ctypes.byref(first), ctypes.byref(failed),
                                              ctypes.byref(bad))
        return st, bool(cb.value), int(first.value), int(failed.value), int(bad.value)

    def debug_poke_guard(self, index: int):
        _check("roibin_ctx_debug_poke_guard", self.lib.roibin_ctx_debug_poke_guard(self._h, int(index)))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- properties
    @property
    def bound(self) -> int:
        return compress_bound(self.geometry, self.params)

    @property
    def scratch_bytes(self) -> int:
        return int(self.lib.roibin_ctx_scratch_bytes(self._h))

    def set_path(self, path: int):
        _check("roibin_ctx_set_path", self.lib.roibin_ctx_set_path(self._h, int(path)))

    def set_fused_dense_peaks(self, on: bool):
        _check("roibin_ctx_set_fused_dense_peaks", self.lib.roibin_ctx_set_fused_dense_peaks(self._h, 1 if on else 0))

    @property
    def fused_dense_peaks(self) -> bool:
        return self.lib.roibin_ctx_fused_dense_peaks(self._h) == 1

    def set_plain_shape(self, rows_per_step: int = 0, bands_per_panel: int = 0):
        _check("roibin_ctx_set_plain_shape", self.lib.roibin_ctx_set_plain_shape(
            self._h, int(rows_per_step), int(bands_per_panel)))

    @property
    def plain_shape(self):
        """(rows per step, bands per panel) set on the context; 0 = chosen per call."""
        r, b = _u32(), _u32()
        _check("roibin_ctx_plain_shape", self.lib.roibin_ctx_plain_shape(self._h, ctypes.byref(r), ctypes.byref(b)))
        return r.value, b.value

    def set_decompress_path(self, path: int):
        _check("roibin_ctx_set_decompress_path", self.lib.roibin_ctx_set_decompress_path(self._h, int(path)))

    @property
    def resolved_decompress_path(self) -> int:
        return int(self.lib.roibin_ctx_resolved_decompress_path(self._h))

    def set_fused_shape(self, ctas_per_sm: int, rows_per_step: int = 0, stages: int = 2):
        _check("roibin_ctx_set_fused_shape", self.lib.roibin_ctx_set_fused_shape(
            self._h, int(ctas_per_sm), int(rows_per_step), int(stages)))

    @property
    def fused_shape(self):
        """(CTAs per SM, rows per step, ring stages, grid CTAs, shared memory bytes) or None."""
        v = [_u32() for _ in range(5)]
        if self.lib.roibin_ctx_fused_shape(self._h, *[ctypes.byref(x) for x in v]) != OK:
            return None
        return tuple(x.value for x in v)

    def autotune(self, frames, out=None, out_stride=None, frame_bytes=None, status=None, stream=None):
        """roibin_ctx_autotune on a CUDA float32 [n, P, H, W] batch: times every shape of the
        path the context resolves to and keeps the fastest.  Returns (the kept shape: fused_shape
        or plain_shape, best ms per call)."""
        import torch
        n = frames.shape[0]
        stride = int(out_stride or self.bound)
        dev = frames.device
        if out is None:
            out = torch.empty((n, stride), dtype=torch.uint8, device=dev)
        if frame_bytes is None:
            frame_bytes = torch.empty(n, dtype=torch.int64, device=dev)
        if status is None:
            status = torch.empty(n, dtype=torch.int32, device=dev)
        ms = ctypes.c_float(-1.0)
        _check("roibin_ctx_autotune", self.lib.roibin_ctx_autotune(
            self._h, _ptr(frames), n, _ptr(out), stride, _ptr(frame_bytes), _ptr(status),
            _stream_handle(stream), ctypes.byref(ms)))
        return (self.fused_shape if self.resolved_path == PATH_FUSED else self.plain_shape), ms.value

    def set_wait_limit(self, polls: int = -1):
        """roibin_ctx_set_wait_limit: polls of the fused path's flag waits (-1: the default)."""
        _check("roibin_ctx_set_wait_limit", self.lib.roibin_ctx_set_wait_limit(self._h, int(polls)))

    def set_trace(self, trace=None, n_frames: int = 0):
        """trace: CUDA int64 tensor of n_frames * (16 + 4 P) entries (None switches tracing off)."""
        _check("roibin_ctx_set_trace", self.lib.roibin_ctx_set_trace(self._h, _ptr(trace), int(n_frames)))

    @property
    def resolved_path(self) -> int:
        return int(self.lib.roibin_ctx_resolved_path(self._h))

    @property
    def last_launch_count(self) -> int:
        return int(self.lib.roibin_ctx_last_launch_count(self._h))

    # -- compression
    def compress(self, frames, out=None, out_stride=None, peaks=None, npeaks=None,
                 frame_bytes=None, status=None, stream=None):
        """frames: CUDA float32 [n, P, H, W].  Returns (out u8 [n, stride], frame_bytes int64 [n],
        status int32 [n]); all asynchronous on `stream` (default: torch's current stream)."""
        import torch
        n = frames.shape[0]
        assert frames.dtype == torch.float32 and frames.is_cuda and frames.is_contiguous()
        assert tuple(frames.shape[1:]) == self.geometry
        stride = int(out_stride or self.bound)
        dev = frames.device
        if out is None:
            out = torch.empty((n, stride), dtype=torch.uint8, device=dev)
        if frame_bytes is None:
            frame_bytes = torch.empty(n, dtype=torch.int64, device=dev)
        if status is None:
            status = torch.empty(n, dtype=torch.int32, device=dev)
        _check("roibin_compress", self.lib.roibin_compress(
            self._h, _ptr(frames), n, _ptr(peaks), _ptr(npeaks), _ptr(out), stride,
            _ptr(frame_bytes), _ptr(status), _stream_handle(stream)))
        return out, frame_bytes, status

    def decompress(self, data, offsets, n_frames, out=None, status=None, stream=None):
        """data: CUDA u8 buffer; offsets: CUDA int64 [n] byte offsets.  Returns (frames, status)."""
        import torch
        dev = data.device
        if out is None:
            out = torch.empty((n_frames, *self.geometry), dtype=torch.float32, device=dev)
        if status is None:
            status = torch.empty(n_frames, dtype=torch.int32, device=dev)
        _check("roibin_decompress", self.lib.roibin_decompress(
            self._h, _ptr(data), data.numel(), _ptr(offsets), n_frames, _ptr(out), _ptr(status),
            _stream_handle(stream)))
        return out, status

    def reserve_host_path(self):
        _check("roibin_ctx_reserve_host_path", self.lib.roibin_ctx_reserve_host_path(self._h))

    def compress_host(self, frames, out, frame_bytes, status, stream=None):
        """Host (ideally pinned) CPU tensors in and out; synchronous."""
        n = frames.shape[0]
        _check("roibin_compress_host", self.lib.roibin_compress_host(
            self._h, _ptr(frames), n, _ptr(out), out.numel(), _ptr(frame_bytes), _ptr(status),
            _stream_handle(stream)))

    def roi_mask(self, peaks, npeaks, n_frames, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((n_frames, *self.geometry), dtype=torch.uint8, device=peaks.device)
        _check("roibin_roi_mask", self.lib.roibin_roi_mask(
            self._h, _ptr(peaks), _ptr(npeaks), n_frames, _ptr(out), _stream_handle(stream)))
        return out

    def last_peaks(self, n_frames, stream=None):
        import torch
        mp = max(int(self.params.max_peaks), 1)
        peaks = torch.zeros((n_frames, mp, 3), dtype=torch.int16, device=f"cuda:{self.device}")
        npeaks = torch.zeros(n_frames, dtype=torch.int32, device=f"cuda:{self.device}")
        _check("roibin_last_peaks", self.lib.roibin_last_peaks(
            self._h, _ptr(peaks), _ptr(npeaks), n_frames, _stream_handle(stream)))
        return peaks, npeaks

    # -- timing
    def enable_timing(self, on: bool = True):
        _check("roibin_ctx_enable_timing", self.lib.roibin_ctx_enable_timing(self._h, int(on)))

    def kernel_times(self):
        """{kernel name: (total ms, launches)} since the last read; synchronises."""
        maxk = 32
        names = (ctypes.c_char_p * maxk)()
        ms = (ctypes.c_double * maxk)()
        cnt = (ctypes.c_uint32 * maxk)()
        nk = ctypes.c_int(0)
        _check("roibin_ctx_kernel_times", self.lib.roibin_ctx_kernel_times(
            self._h, names, ms, cnt, maxk, ctypes.byref(nk)))
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(nk.value, maxk))}


class Graph:
    """Several contexts' compress calls captured into one CUDA graph
    (roibin_graph_create): one after another, with `concurrent` on branches
    the GPU may overlap, or with `fused` the fused-path jobs in one persistent
    launch.  `jobs` is a list of dicts with the keys ctx, frames, out,
    frame_bytes, status and optionally out_stride, peaks, npeaks (CUDA
    tensors, as Context.compress takes them).  The graph keeps the tensors'
    addresses: refill `frames` in place between launches."""

    def __init__(self, jobs, concurrent: bool = False, fused: bool = False):
        if concurrent and fused:
            raise ValueError("a graph is concurrent or fused, not both")
        self.lib = library()
        self._keep = []
        arr = (Job * len(jobs))()
        for i, j in enumerate(jobs):
            ctx, frames, out = j["ctx"], j["frames"], j["out"]
            assert tuple(frames.shape[1:]) == ctx.geometry and frames.is_contiguous()
            stride = int(j.get("out_stride") or out.shape[-1])
            arr[i] = Job(ctx._h, _ptr(frames), frames.shape[0], _ptr(j.get("peaks")), _ptr(j.get("npeaks")),
                         _ptr(out), stride, _ptr(j["frame_bytes"]), _ptr(j["status"]))
            self._keep.append(j)
        h = ctypes.c_void_p()
        _check("roibin_graph_create", self.lib.roibin_graph_create(
            ctypes.byref(h), arr, len(jobs),
            GRAPH_FUSED if fused else GRAPH_CONCURRENT if concurrent else GRAPH_SERIAL))
        self._h = h

    def launch(self, stream=None):
        _check("roibin_graph_launch", self.lib.roibin_graph_launch(self._h, _stream_handle(stream)))

    @property
    def launch_count(self) -> int:
        return int(self.lib.roibin_graph_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self.lib.roibin_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
