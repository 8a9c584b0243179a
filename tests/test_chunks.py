"""Chunks of frames sharing one Huffman code (§5.3.4: a compressor call takes
1-64 events): the GPU writes the oracle's bytes for every frame of a call on
every compression path, the chunk's head alone keeps the code lengths, and
both decompression paths rebuild the oracle's frames, following each
stream's back reference to its head in the same call."""
import numpy as np
import pytest

import oracle
import paper_2206_11297_gb300 as rb
from synthetic import FrameRecipe, make_frame

from gpu_util import FUSED_DENSE, dec_paths, gpu_compress, gpu_decompress, oparams

PATHS = [rb.PATH_PLAIN, rb.PATH_FUSED, FUSED_DENSE]


def frames_of(geom, n, seed, **kw):
    r = FrameRecipe(geom, peaks=("uniform", 1, 8), seed=seed, **kw)
    return np.stack([make_frame(r, k) for k in range(n)])


def test_params_validate():
    g = (4, 40, 48)
    assert rb.validate(g, rb.default_params(chunk_frames=64)) == rb.OK
    assert rb.validate(g, rb.default_params(chunk_frames=0)) == rb.ERR_INVALID_ARG
    assert rb.validate(g, rb.default_params(chunk_frames=65)) == rb.ERR_INVALID_ARG
    assert rb.default_params().chunk_frames == 1


def check_call(frames, params, path, peaks=None, npeaks=None):
    op = oparams(params)
    up = nu = None
    if peaks is not None:
        up = np.zeros((len(frames), max(params.max_peaks, 1), 3), np.uint16)
        up[:, :peaks.shape[1]] = peaks[:, :max(params.max_peaks, 1)]
        nu = np.asarray(npeaks, np.int64)
    ost, orefs, osz = oracle.compress_frames(frames, op, user_peaks=up, n_user=nu)
    st, nb, streams = gpu_compress(frames, params, path=path, peaks=peaks, npeaks=npeaks)
    assert st.tolist() == ost.tolist()
    for k in range(len(frames)):
        if ost[k] != 0:
            continue
        assert nb[k] == len(orefs[k]) and np.array_equal(streams[k], orefs[k]), f"frame {k}: bytes differ"
    ok = [k for k in range(len(frames)) if ost[k] == 0]
    if not ok:
        return ost, orefs
    # decompress the call's coded frames in their order: back references stay within it
    call = [orefs[k] for k in ok]
    dst_o, rec_o = oracle.decompress_frames(call, frames.shape[1:])
    assert (dst_o == 0).all()
    for dp in dec_paths(frames.shape[1:], params):
        rec, dst = gpu_decompress(call, frames.shape[1:], params, dec_path=dp)
        assert dst.tolist() == dst_o.tolist(), dp
        assert np.array_equal(rec.view(np.uint32), rec_o.view(np.uint32)), dp
    return ost, orefs


@pytest.mark.gpu
@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("chunk", [2, 3, 64])
def test_chunks_parity(path, chunk):
    f = frames_of((4, 37, 52), 7, seed=70 + chunk)
    p = rb.default_params(atot_thr=300.0, chunk_frames=chunk)
    ost, refs = check_call(f, p, path)
    refs_h = [oracle.parse_header(r) for r in refs]
    assert [h["back_ref"] for h in refs_h] == [k % chunk for k in range(7)]


@pytest.mark.gpu
@pytest.mark.parametrize("path", [rb.PATH_PLAIN, rb.PATH_FUSED])
def test_chunk_head_skips_rejected_and_bad_frames(path):
    """A rejected first frame, a frame with a bad coordinate and one with too
    many peaks: the chunk's head is its first coded frame."""
    geom = (3, 30, 44)
    f = frames_of(geom, 6, seed=81)
    peaks = np.zeros((6, 8, 3), np.uint16)
    peaks[:, 0] = [0, 5, 5]
    peaks[:, 1] = [1, 20, 30]
    peaks[2, 1] = [3, 0, 0]          # panel 3 of 3: INVALID_ARG
    npeaks = np.array([1, 2, 2, 9, 2, 2], np.uint32)  # 1 < nhr: REJECTED; 9 > max_peaks: CAPACITY
    p = rb.default_params(chunk_frames=3, nhr_min_peaks=2, max_peaks=8)
    ost, refs = check_call(f, p, path, peaks=peaks, npeaks=npeaks)
    assert ost.tolist() == [rb.REJECTED, 0, rb.ERR_INVALID_ARG, rb.ERR_CAPACITY, 0, 0]
    assert oracle.parse_header(refs[1])["back_ref"] == 0 and oracle.parse_header(refs[5])["back_ref"] == 1


@pytest.mark.gpu
def test_follower_needs_its_head():
    """A stream with a back reference decodes only with its head in the call."""
    geom = (4, 37, 52)
    f = frames_of(geom, 3, seed=90)
    p = rb.default_params(atot_thr=300.0, chunk_frames=3)
    ost, refs, _ = oracle.compress_frames(f, oparams(p))
    assert oracle.parse_header(refs[1])["back_ref"] == 1
    for dp in dec_paths(geom, p):
        rec, dst = gpu_decompress([refs[1], refs[2]], geom, p, dec_path=dp)
        assert dst.tolist() == [rb.ERR_CORRUPT_STREAM, rb.ERR_CORRUPT_STREAM], dp
        rec, dst = gpu_decompress([refs[0], refs[1]], geom, p, dec_path=dp)
        assert dst.tolist() == [0, 0], dp


@pytest.mark.gpu
def test_chunks_with_roi_coder_and_hot_pixels():
    f = frames_of((4, 88, 96), 4, seed=95, bg_mean=30.0, bg_sd=8.0, hot_fraction=0.01)
    p = rb.default_params(chunk_frames=4, roi_coder=1, max_peaks=2048, abs_eb=1.0)
    for path in PATHS:
        check_call(f, p, path)
