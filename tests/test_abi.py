"""The C ABI library builds, loads and exports every symbol include/roibin.h
declares; host-side argument logic (no GPU compute) behaves as documented."""
import os
import re
import subprocess

import pytest

import oracle
import paper_2206_11297_gb300 as rb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "roibin.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(roibin_\w+)\s*\(", text)))


def test_library_builds_and_exports_header_symbols():
    lib = rb.library()
    declared = header_functions()
    assert declared == rb.EXPORTED_SYMBOLS, "binding and header disagree"
    nm = subprocess.run(["nm", "-D", "--defined-only", rb._build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (roibin_\w+)", nm))
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(lib, s)


def test_build_targets_sm103a_only():
    assert rb._build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "-fmad=false" in rb._build.FLAGS


def test_default_params_are_the_papers():
    p = rb.default_params()
    assert (p.amax_thr, p.atot_thr, p.son_min, p.npix_min, p.npix_max) == (300.0, 600.0, 10.0, 2, 30)
    assert (p.rank, p.roi_h, p.roi_w, p.bin_h, p.bin_w, p.max_peaks) == (3, 17, 17, 2, 2, 2048)
    assert p.lorenzo_dims == 2


@pytest.mark.parametrize("change,ok", [
    ({}, True), ({"bin_h": 0}, False), ({"bin_w": 9}, False), ({"roi_h": 64}, False),
    ({"rank": 0}, False), ({"quant_radius": 1}, False), ({"quant_radius": 513}, False),
    ({"abs_eb": 0.0}, False), ({"abs_eb": float("nan")}, False), ({"abs_eb": 3e38}, False),
    ({"pix_nsigma": -1.0}, False), ({"max_peaks": 8193}, False), ({"max_peaks": 0}, True),
    ({"npix_max": 1, "npix_min": 2}, False), ({"ring_r0": 10, "ring_dr": 7}, False),
    ({"lorenzo_dims": 0}, False), ({"lorenzo_dims": 1}, True), ({"lorenzo_dims": 3}, True),
    ({"lorenzo_dims": 4}, False),
])
def test_validate(change, ok):
    p = rb.default_params(**change)
    assert (rb.validate((32, 185, 388), p) == rb.OK) == ok


def test_validate_geometry_limits():
    p = rb.default_params()
    assert rb.validate((0, 10, 10), p) == rb.ERR_INVALID_ARG
    assert rb.validate((1, 65536, 10), p) == rb.ERR_INVALID_ARG
    assert rb.validate((1, 10, 2 * 8193), p) == rb.ERR_INVALID_ARG
    # binned size limit keeps every Huffman code within 32 bits
    assert rb.validate((100, 512, 1024), p) == rb.ERR_INVALID_ARG
    assert rb.validate((8, 512, 1024), p) == rb.OK


@pytest.mark.parametrize("geom", [(32, 185, 388), (16, 352, 384), (8, 512, 1024), (3, 17, 23)])
def test_compress_bound_matches_oracle(geom):
    p = rb.default_params()
    assert rb.compress_bound(geom, p) == oracle.compress_bound(geom, oracle.make_params())
    assert rb.compress_bound(geom, p) % 16 == 0
    assert rb.compress_bound((0, 1, 1), p) == 0


def test_status_strings():
    for code in range(0, -9, -1):
        assert rb.status_string(code) != "unknown status"
    assert rb.status_string(-99) == "unknown status"


def test_graph_create_rejects_bad_arguments_before_touching_the_device():
    """Argument checks of roibin_graph_create run on the host first: no jobs,
    and an unknown mode, are refused without a context or a GPU."""
    import ctypes
    lib = rb.library()
    h = ctypes.c_void_p()
    arr = (rb.Job * 1)()
    assert lib.roibin_graph_create(ctypes.byref(h), arr, 0, rb.GRAPH_SERIAL) == rb.ERR_INVALID_ARG
    assert lib.roibin_graph_create(ctypes.byref(h), None, 1, rb.GRAPH_SERIAL) == rb.ERR_INVALID_ARG
    assert lib.roibin_graph_create(ctypes.byref(h), arr, 1, 7) == rb.ERR_INVALID_ARG
    assert not h.value
    assert lib.roibin_graph_create(None, arr, 1, rb.GRAPH_SERIAL) == rb.ERR_INVALID_ARG


def test_static_call_wrapper_refuses_mismatched_buffers():
    """compress_frame_static checks dtype, device, layout and shape before the
    call: a mismatch would make the kernels index out of bounds."""
    import torch
    geom = (2, 16, 24)
    p = rb.default_params()
    frame = torch.zeros(geom, dtype=torch.float32)  # host memory: refused
    out = torch.zeros(rb.compress_bound(geom, p), dtype=torch.uint8)
    nb = torch.zeros(1, dtype=torch.int64)
    st = torch.zeros(1, dtype=torch.int32)
    with pytest.raises(AssertionError):
        rb.compress_frame_static(geom, p, frame, out, nb, st)
    with pytest.raises(AssertionError):  # wrong shape (checked before the device)
        rb.compress_frame_static((2, 16, 25), p, frame, out, nb, st)
    with pytest.raises(AssertionError):  # int32 frame_bytes would be overrun by the u64 store
        rb.compress_frame_static(geom, p, frame, out, nb.to(torch.int32), st)
