"""roibin_compress_frame_static, the one entry point that allocates nothing:
it must give the same bytes as roibin_compress on a one-frame batch, call
after call, and refuse frames whose scratch does not fit its fixed area."""
import numpy as np
import pytest

import oracle
import paper_2206_11297_gb300 as rb
from synthetic import RECIPES, FrameRecipe, make_frame


def test_oversized_frame_is_refused_before_any_gpu_work():
    # 2 x 1024 x 1024 at bin 1x1: about 10 bytes per bin, well over the fixed area
    p = rb.default_params(bin_h=1, bin_w=1)
    g = rb.Geometry(2, 1024, 1024)
    assert rb.validate((2, 1024, 1024), p) == rb.OK
    lib = rb.library()
    fake = 1 << 20  # never dereferenced: the size check comes first
    code = lib.roibin_compress_frame_static(
        rb.ctypes.byref(g), rb.ctypes.byref(p), rb.ctypes.c_void_p(fake), None, None,
        rb.ctypes.c_void_p(fake), 1 << 20, rb.ctypes.c_void_p(fake), rb.ctypes.c_void_p(fake), None)
    assert code == rb.ERR_OUT_OF_BUDGET


def _static_vs_context(geometry, frame, params, peaks=None):
    """Static-scratch bytes == the context's one-frame bytes == the oracle's,
    on two calls in a row.  `peaks` (u16 [n, 3]) replaces the peak finder."""
    import torch
    d = torch.from_numpy(np.ascontiguousarray(frame)).cuda()
    dp = dn = None
    if peaks is not None:
        mp = max(int(params.max_peaks), 1)
        full = np.zeros((mp, 3), np.uint16)
        full[:len(peaks)] = peaks
        dp = torch.from_numpy(full.view(np.int16)).cuda()
        dn = torch.tensor([len(peaks)], dtype=torch.int32, device="cuda")
    with rb.Context(geometry, params, max_frames=1) as ctx:
        ctx.set_path(rb.PATH_PLAIN)
        ref, ref_n, ref_st = ctx.compress(d[None], peaks=None if dp is None else dp[None],
                                          npeaks=dn)
        torch.cuda.synchronize()
        cap = ctx.bound
    ref_n, ref_st = int(ref_n.item()), int(ref_st.item())
    assert ref_st == rb.OK
    expect = ref[0, :ref_n].cpu().numpy()
    ost, oref = oracle.compress_frame(frame, oracle.make_params(**params.as_dict()),
                                      user_peaks=None if peaks is None else np.asarray(peaks, np.uint16))
    assert ost == oracle.OK and np.array_equal(oref, expect), "context path differs from the oracle"
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    nb = torch.empty(1, dtype=torch.int64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    for call in range(2):  # two calls in a row reuse the same area
        out.fill_(0xAA)
        rb.compress_frame_static(geometry, params, d, out, nb, st, peaks=dp, npeaks=dn)
        torch.cuda.synchronize()
        assert int(st.item()) == rb.OK, f"call {call}"
        assert int(nb.item()) == ref_n, f"call {call}"
        got = out[:ref_n].cpu().numpy()
        assert np.array_equal(got, expect), f"call {call}: bytes differ from the context path"
        assert np.array_equal(got, oref), f"call {call}: bytes differ from the oracle"
    return ref_n


@pytest.mark.gpu
def test_static_scratch_matches_context_cspad():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = RECIPES["cspad_single"]
    _static_vs_context(r.geometry, make_frame(r, 0), rb.default_params())


@pytest.mark.gpu
def test_static_scratch_matches_context_small_and_odd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    geom = (3, 45, 62)
    r = FrameRecipe(geom, peaks=("uniform", 5, 20), seed=11)
    p = rb.default_params(atot_thr=300.0, bin_h=3, bin_w=2)
    _static_vs_context(geom, make_frame(r, 1), p)


@pytest.mark.gpu
def test_static_scratch_with_caller_peaks():
    """The caller-supplied peak list is its own branch of the call."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    geom = (4, 40, 56)
    r = FrameRecipe(geom, peaks=("uniform", 4, 10), seed=13)
    frame = make_frame(r, 2)
    p = rb.default_params(atot_thr=300.0, max_peaks=64)
    st, found, _ = oracle.find_peaks(frame, oracle.make_params(**p.as_dict()))
    assert st == oracle.OK
    # the finder's peaks in reverse plus two hand-placed ones (edge and corner)
    peaks = np.concatenate([found[::-1], np.array([[0, 0, 0], [3, 39, 55]], np.uint16)])
    _static_vs_context(geom, frame, p, peaks=peaks)


@pytest.mark.gpu
def test_static_scratch_capacity_error():
    """An output smaller than the frame's stream gives ERR_CAPACITY in the
    frame status, with the size the stream needs, as the context path does."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    geom = (3, 45, 64)
    r = FrameRecipe(geom, peaks=("uniform", 5, 20), seed=17)
    frame = make_frame(r, 0)
    p = rb.default_params(atot_thr=300.0)
    need = _static_vs_context(geom, frame, p)
    d = torch.from_numpy(frame).cuda()
    small = (need // 2) // 16 * 16
    out = torch.empty(small, dtype=torch.uint8, device="cuda")
    nb = torch.empty(1, dtype=torch.int64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    rb.compress_frame_static(geom, p, d, out, nb, st)
    torch.cuda.synchronize()
    assert int(st.item()) == rb.ERR_CAPACITY
    assert int(nb.item()) == need
    ost, osize = oracle.compress_frame(frame, oracle.make_params(**p.as_dict()), capacity=small)
    assert ost == oracle.ERR_CAPACITY and osize == need


@pytest.mark.gpu
def test_static_scratch_with_roi_coder():
    """The ROI coder's kernels run from the same fixed area."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = RECIPES["cspad_single"]
    _static_vs_context(r.geometry, make_frame(r, 0), rb.default_params(roi_coder=1, npix_max=49))
