"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle,
byte for byte on the compressed streams and bit for bit on the
reconstructions, over seeded synthetic frames: small cases spanning several
tiles and ragged tails, the paper's detector shapes, and the edge cases."""
import numpy as np
import pytest

import oracle
import oracle_pins
import paper_2206_11297_gb300 as rb
from gpu_util import FUSED_DENSE, assert_parity, gpu_compress, gpu_decompress, oparams
from synthetic import RECIPES, FrameRecipe, make_frame

pytestmark = pytest.mark.gpu

PATHS2 = [rb.PATH_PLAIN, rb.PATH_FUSED]
PATHS = PATHS2 + [FUSED_DENSE]   # and the fused kernel's dense-peaks variant


def small_batch(geom, n, seed, peaks=("uniform", 2, 12), **kw):
    r = FrameRecipe(geom, peaks=peaks, seed=seed, **kw)
    return np.stack([make_frame(r, k) for k in range(n)])


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rb.library()
    oracle.lib()


def fused_or_skip(geom, params, path):
    """The fused path covers bin 2x2 with cols % 4 == 0; other shapes run the plain path."""
    if path not in (rb.PATH_FUSED, FUSED_DENSE):
        return
    with rb.Context(geom, params, max_frames=1) as ctx:
        ctx.set_path(rb.PATH_AUTO)
        if ctx.resolved_path != rb.PATH_FUSED:
            pytest.skip("fused path not available for this shape")


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("geom", [(2, 12, 13), (1, 7, 8), (3, 21, 27), (4, 37, 52), (2, 64, 100), (1, 3, 1),
                                  (5, 33, 400), (2, 21, 1024), (9, 10, 4), (3, 5, 96),
                                  (1, 19, 872), (1, 10, 1736)])
def test_small_geometries(geom, path):
    f = small_batch(geom, 3, seed=sum(geom))
    assert_parity(f, rb.default_params(atot_thr=300.0), path)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("change", [
    dict(bin_h=1, bin_w=1), dict(bin_h=3, bin_w=3), dict(bin_h=2, bin_w=3), dict(bin_h=4, bin_w=1),
    dict(abs_eb=1.0), dict(abs_eb=0.5), dict(abs_eb=90.0), dict(quant_radius=4), dict(quant_radius=64),
    dict(roi_h=5, roi_w=7), dict(roi_h=16, roi_w=16), dict(rank=1), dict(rank=2),
    dict(pix_nsigma=0.0, npix_max=49), dict(ring_r0=3, ring_dr=1), dict(max_peaks=0),
])
def test_parameters(change, path):
    f = small_batch((3, 45, 62), 2, seed=7, peaks=("uniform", 5, 20))
    p = rb.default_params(atot_thr=300.0)
    for k, v in change.items():
        setattr(p, k, v)
    assert_parity(f, p, path)


@pytest.mark.parametrize("path", PATHS)
def test_tiny_frames_with_planted_features(path):
    f = np.stack([oracle_pins.tiny_frame(s, shape=(2, 12, 13)) for s in range(4)])
    assert_parity(f, rb.default_params(atot_thr=300.0), path)


@pytest.mark.parametrize("path", PATHS)
def test_cspad_single_frame(path):
    f = make_frame(RECIPES["cspad_single"], 0)[None]
    st, nb, _ = assert_parity(f, rb.default_params(), path)
    assert st[0] == 0 and nb[0] < f.nbytes / 50


@pytest.mark.parametrize("path", PATHS)
def test_cspad_batch(path):
    r = RECIPES["cspad_batch"]
    f = np.stack([make_frame(r, k) for k in range(6)])
    assert_parity(f, rb.default_params(), path)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("eb", [1.0, 10.0, 50.0])
def test_epix_hot_pixels(eb, path):
    r = RECIPES["epix_hot"]
    f = np.stack([make_frame(r, k) for k in range(3)])
    assert_parity(f, rb.default_params(abs_eb=eb), path)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("eb", [1.0, 10.0, 50.0])
def test_epix_hot_pixels_round_trip(eb, path):
    """With room for their ~3,600 peaks the hot-pixel frames compress, and their
    streams decode on the dense decoder: no length-1 code at eb 1 and 10, and
    chunks too full of other symbols for the sparse way at eb 50."""
    r = RECIPES["epix_hot"]
    f = np.stack([make_frame(r, k) for k in range(2)])
    st, _, _ = assert_parity(f, rb.default_params(abs_eb=eb, max_peaks=8192), path)
    assert (st == 0).all()


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("hot", [0.001, 0.03, 0.2])
def test_many_candidates_per_item(hot, path):
    """A 1,024-column panel (one fused item, two column groups) with hot pixels:
    its candidates fit the shared list, spill past it to the CTA's list in
    global memory, or overflow both (a rescan of the item)."""
    f = small_batch((1, 64, 1024), 2, seed=int(hot * 1000), bg_mean=30.0, bg_sd=8.0, hot_fraction=hot)
    assert_parity(f, rb.default_params(max_peaks=8192, abs_eb=1.0), path)


@pytest.mark.parametrize("path", PATHS)
def test_jungfrau(path):
    r = RECIPES["jungfrau_mixed"]
    f = np.stack([make_frame(r, k) for k in range(2)])
    assert_parity(f, rb.default_params(), path)


@pytest.mark.parametrize("path", PATHS)
def test_special_frames(path):
    geom = (3, 40, 44)
    rng = np.random.default_rng(0)
    const = np.full(geom, 20.0, np.float32)
    zeros = np.zeros(geom, np.float32)
    bright = (400 + rng.normal(0, 5, geom)).astype(np.float32)  # every pixel >= amax: dense scan
    nonfinite = small_batch(geom, 1, 3)[0]
    nonfinite[0, 3, 4] = np.nan
    nonfinite[1, 10, 10:14] = np.inf
    nonfinite[2, 20, 20] = -np.inf
    nonfinite[2, 30, 30] = np.array([0xFFC01234], np.uint32).view(np.float32)[0]
    huge = small_batch(geom, 1, 4)[0]
    huge[0, :4, :4] = 1e30
    huge[1, 5:9, 5:9] = -3e9
    negative = (rng.normal(-50, 30, geom)).astype(np.float32)
    f = np.stack([const, zeros, bright, nonfinite, huge, negative])
    assert_parity(f, rb.default_params(atot_thr=300.0), path)


@pytest.mark.parametrize("path", PATHS)
def test_dense_candidate_fallback_large(path):
    # more pixels >= amax than the per-frame list holds (16384): the dense scan runs
    geom = (2, 150, 160)
    rng = np.random.default_rng(5)
    f = (350 + rng.normal(0, 20, (1, *geom))).astype(np.float32)
    assert_parity(f, rb.default_params(atot_thr=300.0, max_peaks=8192), path)


@pytest.mark.parametrize("path", PATHS)
def test_user_peaks(path):
    geom = (3, 30, 33)
    f = small_batch(geom, 3, 9)
    p = rb.default_params()
    peaks = np.zeros((3, p.max_peaks, 3), np.uint16)
    npk = np.array([3, 0, 2], np.uint32)
    peaks[0, :3] = [[2, 29, 32], [0, 0, 0], [1, 15, 16]]
    peaks[2, :2] = [[1, 3, 3], [1, 3, 3]]  # duplicates are kept
    assert_parity(f, p, path, peaks=peaks, npeaks=npk)
    bad = peaks.copy()
    bad[1, 0] = [3, 0, 0]  # panel out of range
    st, _, _ = gpu_compress(f, p, path=path, peaks=bad, npeaks=np.array([3, 1, 2], np.uint32))
    assert st.tolist() == [0, rb.ERR_INVALID_ARG, 0]
    st, _, _ = gpu_compress(f, p, path=path, peaks=peaks, npeaks=np.array([3, p.max_peaks + 1, 2], np.uint32))
    assert st[1] == rb.ERR_CAPACITY


@pytest.mark.parametrize("path", PATHS)
def test_capacity_errors(path):
    geom = (2, 40, 48)
    f = small_batch(geom, 2, 12, peaks=("fixed", 6))
    p = rb.default_params(atot_thr=300.0)
    ref_sizes = [len(oracle.compress_frame(f[k], oparams(p))[1]) for k in range(2)]
    stride = (min(ref_sizes) // 16) * 16
    st, nb, _ = gpu_compress(f, p, path=path, out_stride=stride)
    for k in range(2):
        if ref_sizes[k] > stride:
            assert st[k] == rb.ERR_CAPACITY and nb[k] == ref_sizes[k]
        else:
            assert st[k] == 0
    p2 = rb.default_params(atot_thr=300.0, max_peaks=1)
    st, nb, _ = gpu_compress(f, p2, path=path)
    for k in range(2):
        ost, _ = oracle.compress_frame(f[k], oparams(p2))
        assert st[k] == ost


def test_corrupt_streams_are_rejected():
    geom = (2, 24, 28)
    f = small_batch(geom, 1, 13)
    p = rb.default_params(atot_thr=300.0)
    st, ref = oracle.compress_frame(f[0], oparams(p))
    h = oracle.parse_header(ref)
    o = oracle.section_offsets(h)
    bad_magic = ref.copy()
    bad_magic[0] ^= 0xFF
    bad_total = ref.copy()
    bad_total[64] ^= 0x10
    bad_index = ref.copy()
    if h["n_chunks"] > 1:
        bad_index[o["chunk_index"] + 4:o["chunk_index"] + 8] = 0xFF
    bad_len = ref.copy()
    bad_len[o["lengths"]:o["lengths"] + 2 * h["quant_radius"]] = 0
    bad_bits = ref.copy()
    bad_bits[o["bitstream"]:o["end"]] = 0xFF
    for dp in (rb.DEC_PANEL, rb.DEC_MULTIPASS):
        rec, dst = gpu_decompress([bad_magic, bad_total, bad_len, bad_bits, ref], geom, p, dec_path=dp)
        assert dst.tolist()[:4] == [rb.ERR_CORRUPT_STREAM] * 4 and dst[4] == 0


def test_wide_rows_decompress_through_multipass():
    """Panels wider than 4096 bins per row have no panel decompression path:
    AUTO resolves to multi-pass and the round trip still matches the oracle."""
    geom = (1, 5, 8200)
    p = rb.default_params(atot_thr=300.0)
    with rb.Context(geom, p, max_frames=1) as ctx:
        assert ctx.resolved_decompress_path == rb.DEC_MULTIPASS
        with pytest.raises(rb.RoibinError):
            ctx.set_decompress_path(rb.DEC_PANEL)
    assert_parity(small_batch(geom, 2, 5), p, rb.PATH_PLAIN)


def test_wide_rows_decompress_one_bin_row_per_strip():
    """3100 bins per row: the panel path takes one binned row per strip."""
    geom = (2, 5, 6200)
    p = rb.default_params(atot_thr=300.0)
    with rb.Context(geom, p, max_frames=1) as ctx:
        assert ctx.resolved_decompress_path == rb.DEC_PANEL
    assert_parity(small_batch(geom, 2, 6), p, rb.PATH_PLAIN)


@pytest.mark.parametrize("dec_path", [rb.DEC_PANEL, rb.DEC_MULTIPASS])
def test_corrupt_outlier_lists_and_peaks_are_rejected(dec_path):
    """Outlier lists out of order, off their code-0 bins or past the frame, and a
    peak outside the frame: the oracle and both decompression paths reject each."""
    geom = (3, 24, 28)
    f = small_batch(geom, 1, 17)
    f[0, 0, 8:12, 8:12] = 60000.0   # Lorenzo outliers around a bright block
    f[0, 2, 4:8, 4:8] = -60000.0
    f[0, 1, 3, 3] = np.nan           # prequantisation outliers
    f[0, 2, 20, 20] = np.inf
    p = rb.default_params(atot_thr=300.0)
    st, ref = oracle.compress_frame(f[0], oparams(p))
    assert st == 0
    h = oracle.parse_header(ref)
    o = oracle.section_offsets(h)
    assert h["n_lorenzo"] >= 2 and h["n_prequant"] >= 2 and h["n_peaks"] >= 1
    u32 = lambda b, off: b[off:off + 4].view(np.uint32)
    bad = {}
    b = ref.copy()   # first two Lorenzo outliers swapped
    b[o["lorenzo"]:o["lorenzo"] + 16] = np.concatenate([ref[o["lorenzo"] + 8:o["lorenzo"] + 16],
                                                        ref[o["lorenzo"]:o["lorenzo"] + 8]])
    bad["lo_order"] = b
    b = ref.copy()   # first Lorenzo outlier moved to bin 0 (not a code-0 bin)
    u32(b, o["lorenzo"])[0] = 0
    bad["lo_place"] = b
    b = ref.copy()   # last Lorenzo outlier past the frame
    u32(b, o["lorenzo"] + 8 * (h["n_lorenzo"] - 1))[0] = 0xFFFFFFF0
    bad["lo_range"] = b
    b = ref.copy()   # prequantisation outliers out of order
    u32(b, o["prequant"] + 8)[0] = u32(ref, o["prequant"])[0]
    bad["pq_order"] = b
    b = ref.copy()   # last prequantisation outlier past the frame
    u32(b, o["prequant"] + 8 * (h["n_prequant"] - 1))[0] = 0xFFFFFFF0
    bad["pq_range"] = b
    b = ref.copy()   # first peak on a panel that does not exist
    b[o["peaks"]:o["peaks"] + 2].view(np.uint16)[0] = 7
    bad["peak_panel"] = b
    names = list(bad)
    for k in names:
        assert oracle.decompress_frame(bad[k], geom)[0] == oracle.ERR_CORRUPT_STREAM, k
    rec, dst = gpu_decompress([bad[k] for k in names] + [ref], geom, p, dec_path=dec_path)
    assert dict(zip(names, dst.tolist())) == {k: rb.ERR_CORRUPT_STREAM for k in names}
    assert dst[-1] == 0
    ost, orec = oracle.decompress_frame(ref, geom)
    assert np.array_equal(rec[-1].view(np.uint32), orec.view(np.uint32))


@pytest.mark.parametrize("path", PATHS2)
def test_roi_mask_and_peaks_match_oracle(path):
    import torch
    geom = (3, 50, 60)
    f = small_batch(geom, 3, 21, peaks=("uniform", 5, 15))
    p = rb.default_params(atot_thr=300.0)
    with rb.Context(geom, p, max_frames=3) as ctx:
        ctx.set_path(path)
        ctx.compress(torch.from_numpy(f).cuda())
        peaks, npk = ctx.last_peaks(3)
        mask = ctx.roi_mask(peaks, npk, 3)
        torch.cuda.synchronize()
        peaks = peaks.cpu().numpy().view(np.uint16)
        npk, mask = npk.cpu().numpy(), mask.cpu().numpy()
    for k in range(3):
        st, opk, n = oracle.find_peaks(f[k], oparams(p))
        assert npk[k] == n and np.array_equal(peaks[k, :n], opk)
        assert np.array_equal(mask[k], oracle.roi_mask(geom, oparams(p), opk))


@pytest.mark.parametrize("path", PATHS)
def test_batch_composition_invariance(path):
    """A frame compresses to the same bytes alone and inside any batch."""
    r = RECIPES["cspad_batch"]
    f = np.stack([make_frame(r, k) for k in range(4)])
    p = rb.default_params()
    _, _, together = gpu_compress(f, p, path=path)
    for k in (0, 3):
        _, _, alone = gpu_compress(f[k:k + 1], p, path=path)
        assert np.array_equal(alone[0], together[k])


@pytest.mark.parametrize("path", PATHS2)
def test_context_reuse_with_outliers_in_other_panels(path):
    """Prequantisation outliers in different panels on successive calls of one
    context: nothing left over from the first call may leak into the second."""
    import torch
    geom = (3, 40, 44)
    p = rb.default_params(atot_thr=300.0)
    fused_or_skip(geom, p, path)
    a = small_batch(geom, 2, 31)
    b = a.copy()
    a[:, 0, 5, 6] = np.nan       # outliers in panel 0 on the first call
    a[:, 0, 20:22, 8:12] = 1e30
    b[:, 2, 7, 9] = np.inf       # and only in panel 2 on the second
    with rb.Context(geom, p, max_frames=2) as ctx:
        ctx.set_path(path)
        for frames in (a, b):
            out, nb, st = ctx.compress(torch.from_numpy(frames).cuda())
            torch.cuda.synchronize()
            out, nb, st = out.cpu().numpy(), nb.cpu().numpy(), st.cpu().numpy()
            for k in range(2):
                ost, ref = oracle.compress_frame(frames[k], oparams(p))
                assert st[k] == ost == 0
                assert np.array_equal(out[k, :nb[k]], ref)


@pytest.mark.parametrize("path", PATHS)
def test_many_prequant_outliers(path):
    """More prequantisation outliers in one work item than any per-item list
    holds (the fused path then finds them again from the input)."""
    geom = (3, 40, 44)
    p = rb.default_params(atot_thr=300.0)
    fused_or_skip(geom, p, path)
    f = small_batch(geom, 2, 41)
    f[0, :, 4:24, 6:26] = np.nan          # 100 NaN bins in every panel
    f[1, 1, 10:30, 10:40] = 1e30          # 150 huge bins in one panel
    f[1, 2, 0:2, :] = -np.inf
    assert_parity(f, p, path)


def test_autotuner_picks_a_path_for_auto_and_keeps_the_bytes():
    """On AUTO with both paths the autotuner times both and AUTO takes the
    faster; the bytes are the oracle's whichever it is."""
    import torch
    geom = (4, 37, 52)
    f = small_batch(geom, 3, seed=78)
    p = rb.default_params(atot_thr=300.0)
    with rb.Context(geom, p, max_frames=3) as ctx:
        assert ctx.resolved_path == rb.PATH_FUSED
        shape, ms = ctx.autotune(torch.from_numpy(f).cuda())
        assert ms > 0 and ctx.resolved_path in (rb.PATH_FUSED, rb.PATH_PLAIN)
        out, nb, st = ctx.compress(torch.from_numpy(f).cuda())
        torch.cuda.synchronize()
        for k in range(3):
            ost, ref = oracle.compress_frame(f[k], oparams(p))
            assert int(st[k]) == ost == 0 and np.array_equal(out[k, :int(nb[k])].cpu().numpy(), ref)
        ctx.set_path(rb.PATH_FUSED)            # an explicit path still wins
        assert ctx.resolved_path == rb.PATH_FUSED


def test_plain_autotuner_and_shapes_write_the_same_bytes():
    """The plain path's autotuner keeps one of its shapes; a few fixed shapes,
    and the kept one, all write the oracle's bytes."""
    import torch
    geom = (2, 21, 1744)   # wider than the fused path takes (436 float4 columns)
    f = small_batch(geom, 2, seed=91)
    p = rb.default_params(atot_thr=300.0)
    refs = [oracle.compress_frame(f[k], oparams(p)) for k in range(2)]
    with rb.Context(geom, p, max_frames=2) as ctx:
        assert ctx.resolved_path == rb.PATH_PLAIN
        ft = torch.from_numpy(f).cuda()
        for rows, bands in [(1, 1), (4, 5), (16, 2), (0, 0)]:
            ctx.set_plain_shape(rows, bands)
            out, nb, st = ctx.compress(ft)
            torch.cuda.synchronize()
            for k in range(2):
                assert int(st[k]) == refs[k][0] == 0
                assert np.array_equal(out[k, :int(nb[k])].cpu().numpy(), refs[k][1]), (rows, bands, k)
        with pytest.raises(rb.RoibinError):
            ctx.set_plain_shape(17, 0)
        with pytest.raises(rb.RoibinError):
            ctx.set_plain_shape(0, 7)    # 11 binned rows: at most 6 bands
        shape, ms = ctx.autotune(ft)
        assert shape[0] >= 1 and shape[1] >= 1 and ms > 0
        out, nb, st = ctx.compress(ft)
        torch.cuda.synchronize()
        for k in range(2):
            assert np.array_equal(out[k, :int(nb[k])].cpu().numpy(), refs[k][1])


def test_autotuned_shape_writes_the_same_bytes():
    """The autotuner keeps one of the fused shapes; every shape writes the oracle's bytes."""
    import torch
    geom = (4, 37, 52)
    f = small_batch(geom, 3, seed=77)
    p = rb.default_params(atot_thr=300.0)
    with rb.Context(geom, p, max_frames=3) as ctx:
        if ctx.resolved_path != rb.PATH_FUSED:
            pytest.skip("no fused path for this shape")
        shape, ms = ctx.autotune(torch.from_numpy(f).cuda())
        assert shape is not None and ms > 0
        ctx.set_path(rb.PATH_FUSED)
        out, nb, st = ctx.compress(torch.from_numpy(f).cuda())
        torch.cuda.synchronize()
        out, nb, st = out.cpu().numpy(), nb.cpu().numpy(), st.cpu().numpy()
    for k in range(3):
        ost, ref = oracle.compress_frame(f[k], oparams(p))
        assert st[k] == ost == 0 and np.array_equal(out[k, :nb[k]], ref)


def test_new_entry_points_reject_bad_arguments():
    """The dense-peaks switch needs a fused path; decompression paths and plain
    shapes out of range are refused; the context keeps its settings."""
    import torch
    wide = (2, 21, 1744)   # no fused path
    p = rb.default_params(atot_thr=300.0)
    with rb.Context(wide, p, max_frames=1) as ctx:
        with pytest.raises(rb.RoibinError):
            ctx.set_fused_dense_peaks(True)
        assert not ctx.fused_dense_peaks
        with pytest.raises(rb.RoibinError):
            ctx.set_decompress_path(7)
        assert ctx.resolved_decompress_path == rb.DEC_PANEL
        with pytest.raises(rb.RoibinError):
            ctx.set_plain_shape(0, 100)
        assert ctx.plain_shape == (0, 0)
        f = torch.zeros((2, *wide), dtype=torch.float32, device="cuda")
        with pytest.raises(rb.RoibinError):
            ctx.autotune(f)                # more frames than the context takes
    with rb.Context((2, 12, 16), p, max_frames=1) as ctx:
        assert ctx.resolved_path == rb.PATH_FUSED
        ctx.set_fused_dense_peaks(True)
        assert ctx.fused_dense_peaks
        ctx.set_fused_dense_peaks(False)
        assert not ctx.fused_dense_peaks
