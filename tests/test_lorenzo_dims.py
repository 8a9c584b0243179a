"""The Lorenzo predictor's dimension (§6: the row of pixels, the panel, the
panel stack) on the GPU: dimension 1 and 3 streams equal the oracle's byte for
byte, their reconstructions equal the oracle's bit for bit on the multi-pass
decompression path, across plain-path shapes (bands that start inside a panel,
one row per step), parameters and the detector shapes.  Dimension 3 also runs
on the fused path (both variants), whose codebook stage stacks the streamed
2-D residuals; the paths that do not implement a dimension refuse it."""
import numpy as np
import pytest

import oracle
import paper_2206_11297_gb300 as rb
from gpu_util import FUSED_DENSE, assert_parity, gpu_compress, gpu_decompress, oparams
from synthetic import RECIPES, FrameRecipe, make_frame

pytestmark = pytest.mark.gpu

DIMS = [1, 3]
# (dimension, compression path): dimension 1 on the plain path, 3 on every path
CASES = [(1, rb.PATH_PLAIN), (3, rb.PATH_PLAIN), (3, rb.PATH_FUSED), (3, FUSED_DENSE)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rb.library()
    oracle.lib()


def small_batch(geom, n, seed, peaks=("uniform", 2, 12), **kw):
    r = FrameRecipe(geom, peaks=peaks, seed=seed, **kw)
    return np.stack([make_frame(r, k) for k in range(n)])


@pytest.mark.parametrize("dims,path", CASES)
@pytest.mark.parametrize("geom", [(2, 12, 13), (1, 7, 8), (3, 21, 27), (4, 37, 52), (5, 33, 400),
                                  (2, 21, 1024), (9, 10, 4), (1, 3, 1), (6, 20, 1736)])
def test_small_geometries(geom, dims, path):
    f = small_batch(geom, 3, seed=sum(geom) + dims)
    assert_parity(f, rb.default_params(atot_thr=300.0, lorenzo_dims=dims), path)


@pytest.mark.parametrize("dims,path", CASES)
@pytest.mark.parametrize("change", [dict(bin_h=1, bin_w=1), dict(bin_h=3, bin_w=3), dict(bin_h=2, bin_w=3),
                                    dict(abs_eb=0.5), dict(quant_radius=4), dict(quant_radius=200),
                                    dict(max_peaks=0)])
def test_parameters(change, dims, path):
    f = small_batch((3, 45, 62), 2, seed=17, peaks=("uniform", 5, 20))
    assert_parity(f, rb.default_params(atot_thr=300.0, lorenzo_dims=dims, **change), path)


@pytest.mark.parametrize("path", [rb.PATH_FUSED, FUSED_DENSE])
def test_stacked_residuals_with_chunks_roi_coder_and_rejection(path):
    """The fused path's 3-D residuals with chunk codebooks (the chunk's code
    from the stacked histograms), the ROI coder and non-hit rejection."""
    geom = (6, 40, 48)
    f = small_batch(geom, 5, seed=77, peaks=("uniform", 0, 12))
    p = rb.default_params(atot_thr=300.0, lorenzo_dims=3, chunk_frames=3, roi_coder=1, nhr_min_peaks=2)
    ost, orefs, _ = oracle.compress_frames(f, oparams(p))
    st, nb, streams = gpu_compress(f, p, path=path)
    assert st.tolist() == ost.tolist()
    for k in range(len(f)):
        if ost[k] == 0:
            assert np.array_equal(streams[k], orefs[k]), k
    ok = [orefs[k] for k in range(len(f)) if ost[k] == 0]
    rec, dst = gpu_decompress(ok, geom, p)
    _, orec = oracle.decompress_frames(ok, geom)
    assert (dst == 0).all() and np.array_equal(rec.view(np.uint32), orec.view(np.uint32))


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("shape", [(1, 1), (1, 4), (3, 2), (16, 8), (2, 10)])
def test_plain_shapes(shape, dims):
    """Rows per step and bands per panel: bands that start inside a panel take
    the row above (and, in 3-D, the previous panel's) from the frame; the 1-D
    predictor's first bin of a panel follows the previous panel's last."""
    geom = (4, 37, 52)
    f = small_batch(geom, 2, seed=29 + dims)
    p = rb.default_params(atot_thr=300.0, lorenzo_dims=dims)
    op = oparams(p)
    with rb.Context(geom, p, max_frames=2) as ctx:
        ctx.set_plain_shape(*shape)
        st, nb, streams = gpu_compress(f, p, path=rb.PATH_PLAIN, ctx=ctx)
    for k in range(2):
        ost, ref = oracle.compress_frame(f[k], op)
        assert st[k] == 0 and ost == 0 and np.array_equal(streams[k], ref), (shape, k)


@pytest.mark.parametrize("dims,path", CASES)
def test_epix_hot_pixels_eb1(dims, path):
    """Hot pixels at eb 1: many Lorenzo outliers, in every dimension."""
    r = RECIPES["epix_hot"]
    f = np.stack([make_frame(r, k) for k in range(2)])
    st, _, streams = assert_parity(f, rb.default_params(abs_eb=1.0, max_peaks=8192, lorenzo_dims=dims), path)
    assert (st == 0).all()
    assert all(oracle.parse_header(s)["n_lorenzo"] > 1000 for s in streams)


@pytest.mark.parametrize("dims,path", CASES)
def test_cspad_frame(dims, path):
    r = RECIPES["cspad_single"]
    f = make_frame(r, 0)[None]
    st, _, streams = assert_parity(f, rb.default_params(lorenzo_dims=dims), path)
    assert st[0] == 0 and oracle.parse_header(streams[0])["lorenzo_dims"] == dims


def test_paths_and_mismatched_streams():
    geom = (32, 185, 388)
    f = small_batch(geom, 1, seed=3)
    p1, p2, p3 = rb.default_params(lorenzo_dims=1), rb.default_params(), rb.default_params(lorenzo_dims=3)
    with rb.Context(geom, p1, max_frames=1) as ctx:   # dimension 1: the plain path only
        assert ctx.resolved_path == rb.PATH_PLAIN
        with pytest.raises(rb.RoibinError):
            ctx.set_path(rb.PATH_FUSED)
    with rb.Context(geom, p3, max_frames=1) as ctx:   # dimension 3: both, decoded by the multi-pass path
        assert ctx.resolved_path == rb.PATH_FUSED
        assert ctx.resolved_decompress_path == rb.DEC_MULTIPASS
        ctx.set_path(rb.PATH_PLAIN)
        with pytest.raises(rb.RoibinError):
            ctx.set_decompress_path(rb.DEC_PANEL)
    with rb.Context(geom, p2, max_frames=1) as ctx:
        assert ctx.resolved_path == rb.PATH_FUSED
    _, _, s3 = gpu_compress(f, p3)
    _, _, s2 = gpu_compress(f, p2)
    # each context decodes only streams of its own dimension
    _, st = gpu_decompress(s3, geom, p2)
    assert st[0] == rb.ERR_CORRUPT_STREAM
    _, st = gpu_decompress(s2, geom, p3)
    assert st[0] == rb.ERR_CORRUPT_STREAM
    rec, st = gpu_decompress(s3, geom, p3)
    ost, orec = oracle.decompress_frame(s3[0], geom)
    assert st[0] == 0 and ost == 0 and np.array_equal(rec[0].view(np.uint32), orec.view(np.uint32))


def test_autotune_keeps_the_bytes():
    import torch
    geom = (8, 64, 96)
    f = small_batch(geom, 4, seed=41)
    p = rb.default_params(atot_thr=300.0, lorenzo_dims=3)
    with rb.Context(geom, p, max_frames=4) as ctx:
        ctx.autotune(torch.from_numpy(f).cuda())
        assert ctx.resolved_path in (rb.PATH_PLAIN, rb.PATH_FUSED)
        st, nb, streams = gpu_compress(f, p, ctx=ctx)
    op = oparams(p)
    for k in range(4):
        ost, ref = oracle.compress_frame(f[k], op)
        assert st[k] == 0 and np.array_equal(streams[k], ref)
