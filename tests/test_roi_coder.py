"""GPU parity of the two additions at the edges of the path: the lossless ROI
coder (paper §4 keeps each ROI losslessly with fpzip; ours is a coder of that
kind) and non-hit rejection (§1, §4).  Compressed bytes must equal the
oracle's on every compression path, and both decompression paths must give
the oracle's frames and statuses, also for corrupt ROI sections."""
import numpy as np
import pytest

import oracle
import paper_2206_11297_gb300 as rb
from synthetic import RECIPES, FrameRecipe, make_batch, make_frame

from gpu_util import FUSED_DENSE, assert_parity, dec_paths, gpu_compress, gpu_decompress, oparams

PATHS = [rb.PATH_PLAIN, rb.PATH_FUSED, FUSED_DENSE]


def small_batch(geom, n, seed, peaks=("uniform", 2, 12), **kw):
    r = FrameRecipe(geom, peaks=peaks, seed=seed, **kw)
    return np.stack([make_frame(r, k) for k in range(n)])


def test_params_validate():
    g = (4, 40, 48)
    assert rb.validate(g, rb.default_params(roi_coder=1)) == rb.OK
    assert rb.validate(g, rb.default_params(roi_coder=2)) == rb.ERR_INVALID_ARG
    assert rb.validate(g, rb.default_params(nhr_min_peaks=10)) == rb.OK
    assert rb.validate(g, rb.default_params(nhr_min_peaks=-1)) == rb.ERR_INVALID_ARG
    assert rb.validate(g, rb.default_params(nhr_min_peaks=8193)) == rb.ERR_INVALID_ARG
    p = rb.default_params()
    assert p.roi_coder == 0 and p.nhr_min_peaks == 0
    # the coder never needs more room than the raw windows
    assert rb.compress_bound(g, rb.default_params(roi_coder=1)) == rb.compress_bound(g, p)


@pytest.mark.gpu
@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("geom", [(2, 12, 13), (3, 21, 28), (4, 37, 52), (2, 64, 100)])
def test_roi_coder_small_geometries(geom, path):
    f = small_batch(geom, 3, seed=sum(geom) + 7)
    assert_parity(f, rb.default_params(atot_thr=300.0, roi_coder=1), path)


@pytest.mark.gpu
@pytest.mark.parametrize("path", PATHS)
def test_roi_coder_hot_pixels(path):
    """Hundreds of windows per frame around hot-pixel pairs."""
    f = small_batch((4, 88, 96), 3, seed=31, bg_mean=30.0, bg_sd=8.0, hot_fraction=0.01)
    st, _, streams = assert_parity(f, rb.default_params(roi_coder=1, max_peaks=2048, abs_eb=1.0), path)
    h = [oracle.parse_header(s) for s in streams]
    assert all(x["roi_coding"] == 1 and x["n_peaks"] > 20 for x in h)


@pytest.mark.gpu
@pytest.mark.parametrize("roi", [(1, 1), (5, 3), (2, 9), (63, 63)])
def test_roi_coder_window_shapes(roi):
    f = small_batch((2, 70, 72), 2, seed=41)
    assert_parity(f, rb.default_params(atot_thr=300.0, roi_coder=1, roi_h=roi[0], roi_w=roi[1]), rb.PATH_PLAIN)


@pytest.mark.gpu
def test_roi_coder_raw_fallback_and_empty():
    """Incompressible windows (random bit patterns) store the raw floats
    (coding 2); a frame without peaks has an empty section."""
    rng = np.random.default_rng(5)
    geom = (2, 40, 48)
    noise = rng.integers(0, 1 << 32, (1, *geom), dtype=np.uint64).astype(np.uint32).view(np.float32)
    quiet = np.full((1, *geom), 20.0, np.float32)
    frames = np.concatenate([noise, quiet])
    peaks = np.zeros((2, 64, 3), np.uint16)
    peaks[0, :4] = [[0, 15, 15], [1, 20, 30], [0, 25, 25], [1, 10, 20]]  # whole windows in the panel
    npeaks = np.array([4, 0], np.uint32)
    p = rb.default_params(roi_coder=1, max_peaks=64)
    for path in (rb.PATH_PLAIN, rb.PATH_FUSED):
        st, nb, streams = assert_parity(frames, p, path, peaks=peaks, npeaks=npeaks)
        h0, h1 = oracle.parse_header(streams[0]), oracle.parse_header(streams[1])
        assert h0["roi_coding"] == 2 and h0["roi_bytes"] == 4 * 17 * 17 * 4
        assert h1["roi_coding"] == 2 and h1["roi_bytes"] == 0


@pytest.mark.gpu
@pytest.mark.parametrize("path", PATHS)
def test_roi_coder_capacity(path):
    """An output slot that holds the frame but not its ROI section: CAPACITY,
    with the size the whole stream needs, as the oracle reports."""
    f = small_batch((4, 48, 64), 2, seed=43, peaks=("uniform", 6, 10))
    p = rb.default_params(atot_thr=300.0, roi_coder=1)
    op = oparams(p)
    sizes = [len(oracle.compress_frame(x, op)[1]) for x in f]
    hdrs = [oracle.parse_header(oracle.compress_frame(x, op)[1]) for x in f]
    stride = (max(sz - h["roi_bytes"] for sz, h in zip(sizes, hdrs)) + 15) // 16 * 16
    assert stride < min(sizes), "the slot must hold the main part but not the ROI section"
    st, nb, _ = gpu_compress(f, p, path=path, out_stride=stride)
    for k in range(len(f)):
        ost, need = oracle.compress_frame(f[k], op, capacity=stride)
        assert ost == oracle.ERR_CAPACITY and st[k] == rb.ERR_CAPACITY
        assert nb[k] == need == sizes[k]


@pytest.mark.gpu
@pytest.mark.parametrize("path", PATHS)
def test_non_hit_rejection(path):
    geom = (4, 37, 52)
    f = small_batch(geom, 6, seed=51, peaks=("uniform", 0, 8))
    p0 = rb.default_params(atot_thr=300.0)
    counts = [oracle.find_peaks(x, oparams(p0))[2] for x in f]
    thr = int(np.median(counts))
    p = rb.default_params(atot_thr=300.0, nhr_min_peaks=thr)
    st, nb, _ = assert_parity(f, p, path)
    for k, c in enumerate(counts):
        if c < thr:
            assert st[k] == rb.REJECTED and nb[k] == 0
        else:
            assert st[k] == rb.OK
    assert (st == rb.REJECTED).any() and (st == rb.OK).any()


@pytest.mark.gpu
@pytest.mark.parametrize("path", [rb.PATH_PLAIN, rb.PATH_FUSED])
def test_non_hit_rejection_user_peaks_and_capacity(path):
    geom = (3, 30, 44)
    f = small_batch(geom, 3, seed=52)
    peaks = np.zeros((3, 16, 3), np.uint16)
    peaks[0, :1] = [[0, 3, 3]]
    peaks[1, :3] = [[0, 3, 3], [1, 10, 10], [2, 29, 43]]
    npeaks = np.array([1, 3, 17], np.uint32)  # 17 > max_peaks: CAPACITY wins over rejection
    p = rb.default_params(nhr_min_peaks=2, max_peaks=16, roi_coder=1)
    st, nb, streams = gpu_compress(f, p, path=path, peaks=peaks, npeaks=npeaks)
    assert st.tolist() == [rb.REJECTED, rb.OK, rb.ERR_CAPACITY]
    op = oparams(p)
    assert oracle.compress_frame(f[0], op, user_peaks=peaks[0, :1])[0] == oracle.REJECTED
    ost, ref = oracle.compress_frame(f[1], op, user_peaks=peaks[1, :3])
    assert ost == oracle.OK and np.array_equal(streams[1], ref)
    seventeen = np.zeros((17, 3), np.uint16)  # a list longer than max_peaks, as the oracle takes it
    assert oracle.compress_frame(f[2], op, user_peaks=seventeen)[0] == oracle.ERR_CAPACITY
    assert nb[0] == 0


@pytest.mark.gpu
def test_coded_streams_decode_in_any_context_and_corrupt_sections():
    """The decompressor reads the ROI coding from each header (a context
    without the coder decodes coded streams), and rejects a corrupt section
    exactly where the oracle does."""
    geom = (3, 40, 52)
    f = small_batch(geom, 2, seed=61, peaks=("uniform", 4, 8))
    p = rb.default_params(atot_thr=300.0, roi_coder=1)
    op = oparams(p)
    refs = [oracle.compress_frame(x, op)[1] for x in f]
    orecs = [oracle.decompress_frame(r, geom)[1] for r in refs]
    plain_params = rb.default_params(atot_thr=300.0)
    for dp in dec_paths(geom, plain_params):
        rec, dst = gpu_decompress(refs, geom, plain_params, dec_path=dp)
        assert (dst == 0).all()
        for k in range(2):
            assert np.array_equal(rec[k].view(np.uint32), orecs[k].view(np.uint32))
    h = oracle.parse_header(refs[0])
    sec = oracle.section_offsets(h)["roi_section"]
    bad = []
    b = refs[0].copy(); b[sec] = 40; bad.append(b)                                    # a length above 32
    b = refs[0].copy(); b[sec + int(np.flatnonzero(b[sec:sec + 33])[0])] += 1; bad.append(b)  # incomplete code
    b = refs[0].copy(); b[sec + 48:sec + 52] = np.array([3], "<u4").view(np.uint8); bad.append(b)  # first offset
    b = refs[0].copy(); b[84:88] = np.array([h["roi_words"] + 1], "<u4").view(np.uint8); bad.append(b)  # word count
    b = refs[0].copy(); b[76:80] = np.array([3], "<u4").view(np.uint8); bad.append(b)  # unknown coding
    b = refs[0].copy(); b[-20:] ^= 0x5A; bad.append(b)                               # scrambled last bits
    for s in bad:
        ost = oracle.decompress_frame(s, geom)[0]
        for dp in dec_paths(geom, p):
            rec, dst = gpu_decompress([s], geom, p, dec_path=dp)
            assert dst[0] == ost, (dp, dst[0], ost)
    assert any(oracle.decompress_frame(s, geom)[0] == oracle.ERR_CORRUPT_STREAM for s in bad)


@pytest.mark.gpu
def test_roi_coder_cspad_frame():
    """One CSPAD-like frame with the widened npix cap (about 50 windows)."""
    r = RECIPES["cspad_single"]
    f = make_frame(r, 0)[None]
    st, nb, streams = assert_parity(f, rb.default_params(roi_coder=1, npix_max=49), rb.PATH_AUTO)
    h = oracle.parse_header(streams[0])
    assert h["roi_coding"] == 1 and h["roi_bytes"] < h["n_peaks"] * 17 * 17 * 4
