"""Helpers for the GPU parity tests: run the CUDA library through its C ABI
and the CPU oracle on the same seeded frames."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2206_11297_gb300 as rb


# a path token for the tests: the fused path in its dense-peaks variant
FUSED_DENSE = 1002


def oparams(params: rb.Params):
    return oracle.make_params(**params.as_dict())


def gpu_compress(frames: np.ndarray, params: rb.Params, path: int = rb.PATH_AUTO, peaks=None,
                 npeaks=None, out_stride=None, ctx=None):
    """Returns (status int32[n], sizes int64[n], streams list of np.uint8 arrays or None)."""
    import torch
    frames = np.ascontiguousarray(frames, dtype=np.float32)
    n = frames.shape[0]
    own = ctx is None
    if own:
        ctx = rb.Context(frames.shape[1:], params, max_frames=n)
    dense = path == FUSED_DENSE
    if dense:
        path = rb.PATH_FUSED
    try:
        try:
            ctx.set_path(path)
        except rb.RoibinError as e:
            if path == rb.PATH_FUSED and e.code == rb.ERR_INVALID_ARG:
                pytest.skip("the fused path does not cover this shape (bin 2x2, cols % 4 == 0 only)")
            raise
        if dense:
            ctx.set_fused_dense_peaks(True)
        d = torch.from_numpy(frames).cuda()
        dp = dn = None
        if peaks is not None:
            dp = torch.from_numpy(np.ascontiguousarray(peaks).view(np.int16)).cuda()
            dn = torch.from_numpy(np.ascontiguousarray(npeaks, dtype=np.uint32).view(np.int32)).cuda()
        out, nb, st = ctx.compress(d, out_stride=out_stride, peaks=dp, npeaks=dn)
        torch.cuda.synchronize()
        out, nb, st = out.cpu().numpy(), nb.cpu().numpy(), st.cpu().numpy()
    finally:
        if own:
            ctx.close()
    streams = [out[k, :nb[k]].copy() if st[k] == 0 else None for k in range(n)]
    return st, nb, streams


def gpu_decompress(streams, geometry, params: rb.Params, ctx=None, dec_path=rb.DEC_AUTO):
    """Packs the streams (16-byte aligned) and decompresses them on the GPU."""
    import torch
    n = len(streams)
    offs, pos = [], 0
    for s in streams:
        offs.append(pos)
        pos += (len(s) + 15) // 16 * 16
    buf = np.zeros(max(pos, 16), np.uint8)
    for o, s in zip(offs, streams):
        buf[o:o + len(s)] = s
    own = ctx is None
    if own:
        ctx = rb.Context(geometry, params, max_frames=n)
    try:
        data = torch.from_numpy(buf).cuda()
        off = torch.tensor(offs, dtype=torch.int64, device="cuda")
        ctx.set_decompress_path(dec_path)
        rec, st = ctx.decompress(data, off, n)
        torch.cuda.synchronize()
        return rec.cpu().numpy(), st.cpu().numpy()
    finally:
        if own:
            ctx.close()


def dec_paths(geometry, params):
    """Every decompression path the geometry has: the panel path when it fits, and multi-pass."""
    ctx = rb.Context(geometry, params, max_frames=1)
    try:
        panel = ctx.resolved_decompress_path == rb.DEC_PANEL
    finally:
        ctx.close()
    return ([rb.DEC_PANEL] if panel else []) + [rb.DEC_MULTIPASS]


def assert_parity(frames, params, path=rb.PATH_AUTO, peaks=None, npeaks=None, check_decompress=True):
    """GPU bytes == oracle bytes for every frame, and (optionally) the GPU
    reconstruction == the oracle reconstruction bit for bit."""
    op = oparams(params)
    st, nb, streams = gpu_compress(frames, params, path=path, peaks=peaks, npeaks=npeaks)
    refs = []
    for k in range(frames.shape[0]):
        up = None
        if peaks is not None:
            up = np.asarray(peaks[k][:npeaks[k]], np.uint16)
        ost, ref = oracle.compress_frame(frames[k], op, user_peaks=up)
        assert st[k] == ost, f"frame {k}: GPU status {st[k]} vs oracle {ost}"
        if ost != 0:
            refs.append(None)
            continue
        assert nb[k] == len(ref), f"frame {k}: GPU {nb[k]} bytes vs oracle {len(ref)}"
        if not np.array_equal(streams[k], ref):
            diff = np.flatnonzero(streams[k] != ref)
            h = oracle.parse_header(ref)
            raise AssertionError(f"frame {k}: {len(diff)} bytes differ, first at {diff[0]}; "
                                 f"sections {oracle.section_offsets(h)}")
        refs.append(ref)
    if check_decompress:
        ok = [k for k in range(len(refs)) if refs[k] is not None]
        if ok:
            orecs = []
            for k in ok:
                ost, orec = oracle.decompress_frame(refs[k], frames.shape[1:])
                assert ost == 0
                orecs.append(orec)
            for dp in dec_paths(frames.shape[1:], params):
                rec, dst = gpu_decompress([refs[k] for k in ok], frames.shape[1:], params, dec_path=dp)
                for i, k in enumerate(ok):
                    assert dst[i] == 0, f"frame {k}: decompress path {dp} status {dst[i]}"
                    assert np.array_equal(rec[i].view(np.uint32), orecs[i].view(np.uint32)), \
                        f"frame {k}: decompress path {dp}: reconstruction differs"
    return st, nb, streams
