"""ctypes binding of the ROIBIN-SZ CPU oracle.

TEST INFRASTRUCTURE ONLY: the oracle checks the CUDA library and is never
called by it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.

Each wrapper follows one step of the method; the C source cites the passage of
the paper (arXiv 2206.11297) that each step restates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "roibin_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID_ARG = -1
ERR_CAPACITY = -2
ERR_CORRUPT_STREAM = -3
ERR_CODE_LENGTH = -7
REJECTED = 1  # non-hit rejection: the frame has fewer than nhr_min_peaks peaks
ROI_CLASSES = 33

CHUNK_SYMBOLS = 4096
HEADER_BYTES = 96


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


DEFAULTS = dict(amax_thr=300.0, atot_thr=600.0, son_min=10.0, pix_nsigma=3.0, rank=3,
                ring_r0=5, ring_dr=2, npix_min=2, npix_max=30, roi_h=17, roi_w=17,
                bin_h=2, bin_w=2, abs_eb=10.0, quant_radius=512, max_peaks=2048, lorenzo_dims=2,
                nhr_min_peaks=0, roi_coder=0, chunk_frames=1)


def make_params(**kw) -> Params:
    d = dict(DEFAULTS)
    d.update(kw)
    return Params(**d)


def _compile(src: str, out: str, cc: str = "gcc") -> None:
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call([cc, "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                           "-I", _HERE, "-shared", "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)


def build(force: bool = False, cc: str = "gcc") -> str:
    """Compile liboracle.so in-tree: -O2, no FMA contraction, one translation unit."""
    with _lock:
        hdr = os.path.join(_HERE, "roibin_oracle.h")
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
                os.path.getmtime(_SRC), os.path.getmtime(hdr)):
            _compile(_SRC, _LIB_PATH, cc)
    return _LIB_PATH


_SIGNATURES = None


def _bind(path: str):
    global _SIGNATURES
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    u32, i32, u64, i64 = ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64
    G, Pr = ctypes.POINTER(Geometry), ctypes.POINTER(Params)
    sig = {
        "orc_is_peak_candidate": (ctypes.c_int, [P, u32, u32, u32, u32, i32, ctypes.c_float]),
        "orc_evaluate_peak": (ctypes.c_int, [P, u32, u32, u32, u32, Pr]),
        "orc_find_peaks": (ctypes.c_int, [P, G, Pr, P, u32, P]),
        "orc_roi_extract": (None, [P, G, Pr, P, u32, P]),
        "orc_roi_mask": (None, [G, Pr, P, u32, P]),
        "orc_bin": (None, [P, G, i32, i32, P]),
        "orc_prequantize": (None, [P, u64, ctypes.c_float, P, P]),
        "orc_lorenzo": (None, [P, u32, u32, u32, P]),
        "orc_lorenzo_nd": (None, [P, u32, u32, u32, ctypes.c_int32, P]),
        "orc_quant_codes": (None, [P, u64, i32, P]),
        "orc_histogram": (None, [P, u64, u32, P]),
        "orc_huffman_lengths": (ctypes.c_int, [P, u32, P]),
        "orc_canonical_codes": (None, [P, u32, P]),
        "orc_pack_chunks": (u32, [P, u64, P, P, P, P]),
        "orc_roi_order_bits": (u32, [ctypes.c_float]),
        "orc_roi_residuals": (None, [P, i32, i32, P]),
        "orc_roi_class": (u32, [u32]),
        "orc_roi_encode": (u64, [P, u32, i32, i32, P, P, P]),
        "orc_roi_decode": (ctypes.c_int, [P, u64, u32, u32, u32, i32, i32, P]),
        "orc_compress_bound": (u64, [G, Pr]),
        "orc_compress_frame": (ctypes.c_int, [P, G, Pr, P, i64, P, u64, P]),
        "orc_decompress_frame": (ctypes.c_int, [P, u64, G, P]),
        "orc_compress_frames": (ctypes.c_int, [P, u32, G, Pr, P, P, P, u64, P, P]),
        "orc_decompress_frames": (ctypes.c_int, [P, u64, P, u32, G, P, P]),
    }
    _SIGNATURES = sorted(sig)
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


class use_library:
    """Context manager: route every wrapper of this module through another build
    of the oracle (used by the tests that plant mistakes in a copy of it)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = _lib
        _lib = _bind(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def compile_variant(source_text: str, out_dir: str, name: str) -> str:
    """Compile a modified copy of the oracle source into out_dir; returns the .so path."""
    src = os.path.join(out_dir, name + ".c")
    with open(src, "w") as f:
        f.write(source_text)
    out = os.path.join(out_dir, name + ".so")
    _compile(src, out)
    return out


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "arrays passed to the oracle must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def binned_shape(geom, bin_h, bin_w):
    P, H, W = geom
    return P, -(-H // bin_h), -(-W // bin_w)


# ---------------------------------------------------------------- step wrappers
def is_peak_candidate(panel: np.ndarray, r: int, c: int, rank: int, amax_thr: float) -> bool:
    panel = np.ascontiguousarray(panel, dtype=np.float32)
    return bool(lib().orc_is_peak_candidate(_ptr(panel), panel.shape[0], panel.shape[1], r, c, rank, amax_thr))


def evaluate_peak(panel: np.ndarray, r: int, c: int, params: Params) -> bool:
    panel = np.ascontiguousarray(panel, dtype=np.float32)
    return bool(lib().orc_evaluate_peak(_ptr(panel), panel.shape[0], panel.shape[1], r, c, ctypes.byref(params)))


def find_peaks(frame: np.ndarray, params: Params):
    """Returns (status, peaks u16[n,3]).  On CAPACITY the array holds the first max_peaks."""
    frame = np.ascontiguousarray(frame, dtype=np.float32)
    g = Geometry(*frame.shape)
    cap = max(int(params.max_peaks), 0)
    out = np.zeros((cap + 1, 3), np.uint16)
    n = ctypes.c_uint32(0)
    st = lib().orc_find_peaks(_ptr(frame), ctypes.byref(g), ctypes.byref(params), _ptr(out), cap, ctypes.byref(n))
    return st, out[: min(n.value, cap)].copy(), n.value


def roi_extract(frame: np.ndarray, params: Params, peaks: np.ndarray) -> np.ndarray:
    frame = np.ascontiguousarray(frame, dtype=np.float32)
    peaks = np.ascontiguousarray(peaks, dtype=np.uint16).reshape(-1, 3)
    out = np.zeros((len(peaks), params.roi_h, params.roi_w), np.float32)
    g = Geometry(*frame.shape)
    lib().orc_roi_extract(_ptr(frame), ctypes.byref(g), ctypes.byref(params), _ptr(peaks), len(peaks), _ptr(out))
    return out


def roi_mask(shape, params: Params, peaks: np.ndarray) -> np.ndarray:
    peaks = np.ascontiguousarray(peaks, dtype=np.uint16).reshape(-1, 3)
    out = np.zeros(shape, np.uint8)
    g = Geometry(*shape)
    lib().orc_roi_mask(ctypes.byref(g), ctypes.byref(params), _ptr(peaks), len(peaks), _ptr(out))
    return out


def bin_frame(frame: np.ndarray, bin_h: int, bin_w: int) -> np.ndarray:
    frame = np.ascontiguousarray(frame, dtype=np.float32)
    out = np.zeros(binned_shape(frame.shape, bin_h, bin_w), np.float32)
    g = Geometry(*frame.shape)
    lib().orc_bin(_ptr(frame), ctypes.byref(g), bin_h, bin_w, _ptr(out))
    return out


def prequantize(binned: np.ndarray, abs_eb: float):
    b = np.ascontiguousarray(binned, dtype=np.float32)
    q = np.zeros(b.shape, np.int32)
    pq = np.zeros(b.shape, np.uint8)
    lib().orc_prequantize(_ptr(b), b.size, abs_eb, _ptr(q), _ptr(pq))
    return q, pq


def lorenzo(q: np.ndarray, dims: int = 2) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.int32)
    P, hb, wb = q.shape
    d = np.zeros_like(q)
    if dims == 2:
        lib().orc_lorenzo(_ptr(q), P, hb, wb, _ptr(d))
    else:
        lib().orc_lorenzo_nd(_ptr(q), P, hb, wb, dims, _ptr(d))
    return d


def quant_codes(delta: np.ndarray, radius: int) -> np.ndarray:
    d = np.ascontiguousarray(delta, dtype=np.int32)
    c = np.zeros(d.shape, np.uint16)
    lib().orc_quant_codes(_ptr(d), d.size, radius, _ptr(c))
    return c


def histogram(codes: np.ndarray, n_symbols: int) -> np.ndarray:
    c = np.ascontiguousarray(codes, dtype=np.uint16)
    h = np.zeros(n_symbols, np.uint64)
    lib().orc_histogram(_ptr(c), c.size, n_symbols, _ptr(h))
    return h


def huffman_lengths(hist) -> tuple[int, np.ndarray]:
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    out = np.zeros(len(h), np.uint8)
    st = lib().orc_huffman_lengths(_ptr(h), len(h), _ptr(out))
    return st, out


def canonical_codes(lengths) -> np.ndarray:
    L = np.ascontiguousarray(lengths, dtype=np.uint8)
    out = np.zeros(len(L), np.uint32)
    lib().orc_canonical_codes(_ptr(L), len(L), _ptr(out))
    return out


def pack_chunks(codes: np.ndarray, lengths: np.ndarray, codewords: np.ndarray):
    c = np.ascontiguousarray(codes, dtype=np.uint16).ravel()
    L = np.ascontiguousarray(lengths, dtype=np.uint8)
    cw = np.ascontiguousarray(codewords, dtype=np.uint32)
    n_chunks = -(-c.size // CHUNK_SYMBOLS)
    idx = np.zeros(n_chunks, np.uint32)
    words = np.zeros(c.size + 1, np.uint32)
    n = lib().orc_pack_chunks(_ptr(c), c.size, _ptr(L), _ptr(cw), _ptr(idx), _ptr(words))
    return idx, words[:n].copy()


# ---------------------------------------------------------------- ROI coding
def roi_order_bits(x: float) -> int:
    return int(lib().orc_roi_order_bits(ctypes.c_float(x)))


def roi_residuals(window: np.ndarray) -> np.ndarray:
    """Folded prediction residuals z of one roi_h x roi_w float32 window."""
    w = np.ascontiguousarray(window, dtype=np.float32)
    z = np.zeros(w.shape, np.uint32)
    lib().orc_roi_residuals(_ptr(w), w.shape[0], w.shape[1], _ptr(z))
    return z


def roi_class(z: int) -> int:
    return int(lib().orc_roi_class(int(z) & 0xFFFFFFFF))


def roi_encode(windows: np.ndarray):
    """Section of n float32 windows [n, h, w]: (coding 1 or 2, n_words, section bytes)."""
    w = np.ascontiguousarray(windows, dtype=np.float32)
    n, h, ww = w.shape
    out = np.zeros(w.size * 4 + 64, np.uint8)
    coding, words = ctypes.c_uint32(0), ctypes.c_uint32(0)
    nb = lib().orc_roi_encode(_ptr(w), n, h, ww, _ptr(out), ctypes.byref(coding), ctypes.byref(words))
    return coding.value, words.value, out[:nb].copy()


def roi_decode(section: np.ndarray, coding: int, n_words: int, n: int, h: int, w: int):
    """(status, windows float32 [n, h, w]) from a section written by roi_encode."""
    sec = np.ascontiguousarray(section, dtype=np.uint8)
    if sec.size == 0:
        sec = np.zeros(16, np.uint8)[:0]
    out = np.zeros((n, h, w), np.float32)
    buf = np.zeros(max(sec.size, 16), np.uint8)
    buf[:sec.size] = sec
    st = lib().orc_roi_decode(_ptr(buf), sec.size, coding, n_words, n, h, w, _ptr(out))
    return st, out


# ---------------------------------------------------------------- whole frame
def compress_bound(shape, params: Params) -> int:
    g = Geometry(*shape)
    return int(lib().orc_compress_bound(ctypes.byref(g), ctypes.byref(params)))


def compress_frame(frame: np.ndarray, params: Params, user_peaks=None, capacity=None):
    """Returns (status, bytes).  bytes is the whole frame stream on success."""
    frame = np.ascontiguousarray(frame, dtype=np.float32)
    g = Geometry(*frame.shape)
    cap = compress_bound(frame.shape, params) if capacity is None else int(capacity)
    out = np.zeros(max(cap, 16), np.uint8)
    nbytes = ctypes.c_uint64(0)
    if user_peaks is None:
        up, n_up = None, -1
    else:
        arr = np.ascontiguousarray(user_peaks, dtype=np.uint16).reshape(-1, 3)
        up, n_up = _ptr(arr), len(arr)
    st = lib().orc_compress_frame(_ptr(frame), ctypes.byref(g), ctypes.byref(params), up, n_up,
                                  _ptr(out), cap, ctypes.byref(nbytes))
    if st != OK:
        return st, None if st != ERR_CAPACITY else int(nbytes.value)
    return st, out[: nbytes.value].copy()


def compress_frames(frames: np.ndarray, params: Params, user_peaks=None, n_user=None, stride=None):
    """A call of frames (chunks of params.chunk_frames share a codebook).
    user_peaks: u16 [n, max_peaks, 3] with n_user[f] entries each (or None).
    Returns (status int32 [n], streams: list of uint8 arrays or None, sizes int64 [n])."""
    frames = np.ascontiguousarray(frames, dtype=np.float32)
    n = frames.shape[0]
    g = Geometry(*frames.shape[1:])
    st_ = stride or compress_bound(frames.shape[1:], params)
    outs = np.zeros((n, max(int(st_), 16)), np.uint8)
    sizes = np.zeros(n, np.uint64)
    status = np.zeros(n, np.int32)
    up = nu = None
    if user_peaks is not None:
        upa = np.ascontiguousarray(user_peaks, dtype=np.uint16)
        nua = np.ascontiguousarray(n_user, dtype=np.int64)
        up, nu = _ptr(upa), _ptr(nua)
    lib().orc_compress_frames(_ptr(frames), n, ctypes.byref(g), ctypes.byref(params), up, nu, _ptr(outs),
                              outs.shape[1], _ptr(sizes), _ptr(status))
    streams = [outs[k, :sizes[k]].copy() if status[k] == OK else None for k in range(n)]
    return status, streams, sizes.astype(np.int64)


def pack_streams(streams):
    """Streams back to back, each padded to 16 bytes: (buffer, offsets)."""
    offs, pos = [], 0
    for s in streams:
        offs.append(pos)
        pos += (len(s) + 15) // 16 * 16
    buf = np.zeros(max(pos, 16), np.uint8)
    for o, s in zip(offs, streams):
        buf[o:o + len(s)] = s
    return buf, np.array(offs, np.uint64)


def decompress_frames(streams, shape):
    """A call of streams (a stream may take its code lengths from its chunk's
    head earlier in the call).  Returns (status int32 [n], frames float32)."""
    buf, offs = pack_streams(streams)
    n = len(streams)
    out = np.zeros((n, *shape), np.float32)
    status = np.zeros(n, np.int32)
    g = Geometry(*shape)
    lib().orc_decompress_frames(_ptr(buf), buf.size, _ptr(offs), n, ctypes.byref(g), _ptr(out), _ptr(status))
    return status, out


def decompress_frame(stream: np.ndarray, shape):
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    out = np.zeros(shape, np.float32)
    g = Geometry(*shape)
    st = lib().orc_decompress_frame(_ptr(s), s.size, ctypes.byref(g), _ptr(out))
    return st, out


def parse_header(stream: np.ndarray) -> dict:
    """Field view of the 96-byte frame header (format version 1)."""
    b = np.ascontiguousarray(stream[:HEADER_BYTES], dtype=np.uint8)
    u32 = b[:64].view(np.uint32)
    tail = b[76:92].view(np.uint32)
    u16 = b[20:28].view(np.uint16)
    return dict(magic=int(u32[0]), version=int(u32[1]), n_panels=int(u32[2]), rows=int(u32[3]),
                cols=int(u32[4]), roi_h=int(u16[0]), roi_w=int(u16[1]), bin_h=int(u16[2]),
                bin_w=int(u16[3]), abs_eb=float(b[28:32].view(np.float32)[0]),
                quant_radius=int(u32[8]), n_peaks=int(u32[9]), n_lorenzo=int(u32[10]),
                n_prequant=int(u32[11]), n_symbols=int(u32[12]), chunk_symbols=int(u32[13]),
                n_chunks=int(u32[14]), n_words=int(u32[15]),
                total_bytes=int(b[64:72].view(np.uint64)[0]),
                lorenzo_dims={0: 2}.get(int(b[72:76].view(np.uint32)[0]), int(b[72:76].view(np.uint32)[0])),
                roi_coding=int(tail[0]), roi_bytes=int(tail[1]), roi_words=int(tail[2]), back_ref=int(tail[3]))


def section_offsets(h: dict) -> dict:
    """Byte offsets of each section, from the header counts (format version 1)."""
    a16 = lambda x: (x + 15) & ~15
    o = {"peaks": HEADER_BYTES}
    o["roi"] = o["peaks"] + a16(h["n_peaks"] * 6)
    in_place = h.get("roi_coding", 0) == 0
    o["lengths"] = o["roi"] + (a16(h["n_peaks"] * h["roi_h"] * h["roi_w"] * 4) if in_place else 0)
    o["chunk_index"] = o["lengths"] + (a16(2 * h["quant_radius"]) if h.get("back_ref", 0) == 0 else 0)
    o["lorenzo"] = o["chunk_index"] + a16(h["n_chunks"] * 4)
    o["prequant"] = o["lorenzo"] + a16(h["n_lorenzo"] * 8)
    o["bitstream"] = o["prequant"] + a16(h["n_prequant"] * 8)
    o["roi_section"] = o["bitstream"] + a16(h["n_words"] * 4)
    o["end"] = o["roi_section"] + h.get("roi_bytes", 0)
    return o
