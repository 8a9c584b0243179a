"""Mixed-geometry batches under one CUDA graph (roibin_graph_*), with the jobs
chained or on concurrent branches: every job's bytes equal those of its own
compress call, on every launch, after the inputs are refilled in place."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2206_11297_gb300 as rb
from gpu_util import oparams
from synthetic import RECIPES, make_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rb.library()


MIX = [("cspad_mixed", 3), ("epix_mixed", 2), ("jungfrau_mixed", 2)]


def _frames(name, n, first):
    r = RECIPES[name]
    return np.stack([make_frame(r, first + k) for k in range(n)])


def _jobs(torch, params, first, tune):
    jobs = []
    for name, n in MIX:
        geom = RECIPES[name].geometry
        ctx = rb.Context(geom, params, max_frames=n)
        frames = torch.from_numpy(_frames(name, n, first)).cuda()
        out = torch.zeros((n, ctx.bound), dtype=torch.uint8, device="cuda")
        nb = torch.zeros(n, dtype=torch.int64, device="cuda")
        st = torch.zeros(n, dtype=torch.int32, device="cuda")
        if tune:
            ctx.autotune(frames)
        jobs.append(dict(ctx=ctx, frames=frames, out=out, frame_bytes=nb, status=st, name=name))
    return jobs


def _alone(job):
    """The same frames through the job's own context, one compress call."""
    out, nb, st = job["ctx"].compress(job["frames"])
    return out.cpu().numpy(), nb.cpu().numpy(), st.cpu().numpy()


def _check_against_alone(torch, jobs):
    torch.cuda.synchronize()
    for j in jobs:
        g_out, g_nb, g_st = j["out"].cpu().numpy(), j["frame_bytes"].cpu().numpy(), j["status"].cpu().numpy()
        a_out, a_nb, a_st = _alone(j)
        assert (g_st == a_st).all() and (g_st == 0).all(), (j["name"], g_st, a_st)
        assert (g_nb == a_nb).all(), j["name"]
        for k in range(len(g_nb)):
            assert np.array_equal(g_out[k, :g_nb[k]], a_out[k, :a_nb[k]]), (j["name"], k)


@pytest.mark.parametrize("concurrent", [False, True], ids=["serial", "concurrent"])
def test_graph_matches_separate_calls_and_refills(concurrent):
    import torch
    params = rb.default_params(max_peaks=8192)
    jobs = _jobs(torch, params, first=0, tune=True)
    paths = {j["name"]: j["ctx"].resolved_path for j in jobs}
    assert paths["cspad_mixed"] == rb.PATH_FUSED
    with rb.Context(RECIPES["jungfrau_mixed"].geometry, params, max_frames=1) as c:
        assert c.resolved_path == rb.PATH_FUSED   # 1,024-column panels: two column groups
    with rb.Graph(jobs, concurrent=concurrent) as g:
        assert g.launch_count >= len(jobs)
        g.launch()
        _check_against_alone(torch, jobs)
        # the oracle on one frame of each geometry
        for j in jobs:
            nb = int(j["frame_bytes"][0])
            ost, ref = oracle.compress_frame(j["frames"][0].cpu().numpy(), oparams(params))
            assert ost == 0 and np.array_equal(j["out"][0, :nb].cpu().numpy(), ref), j["name"]
        # refill the inputs in place with other frames and launch again
        for j, (name, n) in zip(jobs, MIX):
            j["frames"].copy_(torch.from_numpy(_frames(name, n, first=100)))
            j["status"].fill_(-99)
        g.launch()
        g.launch()
        _check_against_alone(torch, jobs)
    for j in jobs:
        j["ctx"].close()


def test_graph_rejects_shared_contexts_and_bad_jobs():
    import torch
    params = rb.default_params()
    geom = RECIPES["cspad_mixed"].geometry
    with rb.Context(geom, params, max_frames=1) as ctx:
        f = torch.zeros((1, *geom), dtype=torch.float32, device="cuda")
        out = torch.zeros((1, ctx.bound), dtype=torch.uint8, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        job = dict(ctx=ctx, frames=f, out=out, frame_bytes=nb, status=st)
        with pytest.raises(rb.RoibinError):
            rb.Graph([job, job])
        with pytest.raises(rb.RoibinError):
            rb.Graph([dict(job, out_stride=ctx.bound + 8)])
        # an unknown mode is refused through the C ABI
        lib, h = rb.library(), ctypes.c_void_p()
        arr = (rb.Job * 1)(rb.Job(ctx._h, f.data_ptr(), 1, None, None, out.data_ptr(), ctx.bound,
                                   nb.data_ptr(), st.data_ptr()))
        assert lib.roibin_graph_create(ctypes.byref(h), arr, 1, 7) == rb.ERR_INVALID_ARG and not h.value
        with rb.Graph([job]) as g:   # one job is a graph too
            g.launch()
            torch.cuda.synchronize()
            assert int(st[0]) == 0
