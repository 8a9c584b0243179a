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
    # untuned, every geometry of the mix takes the fused path (the 1,024-column
    # panels with two column groups); the autotuner may pick either path for
    # these few frames, and the graph takes each context as tuned
    for name, _ in MIX:
        with rb.Context(RECIPES[name].geometry, params, max_frames=1) as c:
            assert c.resolved_path == rb.PATH_FUSED, name
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


def _check_every_frame_against_oracle(jobs, params_of):
    """Every frame of every job: the oracle's status and bytes."""
    for j in jobs:
        p = oparams(params_of(j))
        frames = j["frames"].cpu().numpy()
        out, nb, st = j["out"].cpu().numpy(), j["frame_bytes"].cpu().numpy(), j["status"].cpu().numpy()
        for k in range(len(frames)):
            ost, ref = oracle.compress_frame(frames[k], p)
            assert st[k] == ost, (j["name"], k, st[k], ost)
            if ost == 0:
                assert nb[k] == len(ref) and np.array_equal(out[k, :nb[k]], ref), (j["name"], k)


def test_fused_graph_is_one_launch_and_matches_the_oracle():
    """CSPAD-, epix10k- (dense peaks, hot pixels) and 8 x 512 x 1024-shaped
    batches in ONE persistent launch: every frame equals the oracle's, on every
    launch and after the inputs are refilled in place."""
    import torch
    params = rb.default_params(max_peaks=8192)
    jobs = _jobs(torch, params, first=0, tune=True)
    for j in jobs:
        j["ctx"].set_path(rb.PATH_FUSED)
    jobs[1]["ctx"].set_fused_dense_peaks(True)   # the hot-pixel frames
    with rb.Graph(jobs, fused=True) as g:
        assert g.launch_count == 1
        g.launch()
        torch.cuda.synchronize()
        _check_every_frame_against_oracle(jobs, lambda j: params)
        _check_against_alone(torch, jobs)
        for j, (name, n) in zip(jobs, MIX):
            j["frames"].copy_(torch.from_numpy(_frames(name, n, first=50)))
            j["status"].fill_(-99)
        g.launch()
        g.launch()
        torch.cuda.synchronize()
        _check_every_frame_against_oracle(jobs, lambda j: params)
    for j in jobs:
        j["ctx"].close()


def test_fused_graph_mixes_parameters_features_and_paths():
    """One joint launch over jobs that differ in everything a context fixes:
    error bound, quant radius, the ROI coder, chunk codebooks, non-hit
    rejection, dense peaks, user peak lists, panel width and the 3-D predictor,
    next to jobs the persistent kernel does not take (cols % 4 != 0, the 1-D
    predictor), which follow it."""
    import torch
    from synthetic import FrameRecipe
    specs = [
        ("a", (4, 37, 52), dict(atot_thr=300.0, abs_eb=2.0), False),
        ("b", (3, 40, 44), dict(atot_thr=300.0, quant_radius=64, roi_coder=1), False),
        ("c", (2, 30, 1024), dict(atot_thr=300.0, chunk_frames=3, nhr_min_peaks=3), False),
        ("d", (4, 48, 64), dict(abs_eb=1.0, max_peaks=2048), True),
        ("e", (2, 21, 27), dict(atot_thr=300.0), False),                  # plain path: cols % 4 != 0
        ("f", (3, 40, 44), dict(atot_thr=300.0, lorenzo_dims=1), False),  # plain path: 1-D
        ("g", (2, 24, 32), dict(atot_thr=300.0, roi_coder=1, max_peaks=16), False),  # user peaks
        ("h", (5, 30, 64), dict(atot_thr=300.0, lorenzo_dims=3), False),  # the panel stack's predictor
    ]
    jobs, prm = [], {}
    for i, (name, geom, kw, hot) in enumerate(specs):
        extra = dict(bg_mean=30.0, bg_sd=8.0, hot_fraction=0.01) if hot else {}
        r = FrameRecipe(geom, peaks=("uniform", 0, 10), seed=200 + i, **extra)
        n = 4
        f = np.stack([make_frame(r, k) for k in range(n)])
        p = rb.default_params(**kw)
        prm[name] = p
        ctx = rb.Context(geom, p, max_frames=n)
        if hot:
            ctx.set_fused_dense_peaks(True)
        job = dict(ctx=ctx, frames=torch.from_numpy(f).cuda(),
                   out=torch.zeros((n, ctx.bound), dtype=torch.uint8, device="cuda"),
                   frame_bytes=torch.zeros(n, dtype=torch.int64, device="cuda"),
                   status=torch.zeros(n, dtype=torch.int32, device="cuda"), name=name)
        if name == "g":
            pk = np.zeros((n, 16, 3), np.uint16)
            pk[:, 0] = [0, 5, 6]
            pk[:, 1] = [1, 20, 30]
            job["peaks"] = torch.from_numpy(pk.view(np.int16)).cuda()
            job["npeaks"] = torch.tensor([2, 1, 0, 2], dtype=torch.int32, device="cuda")
            job["_pk"] = pk
        jobs.append(job)
    paths = [j["ctx"].resolved_path for j in jobs]
    assert paths[4] == rb.PATH_PLAIN and paths[5] == rb.PATH_PLAIN and paths[0] == paths[7] == rb.PATH_FUSED
    # the plain-path jobs' own launch counts, one call each
    chain = 0
    for j in jobs:
        if j["ctx"].resolved_path == rb.PATH_PLAIN:
            j["ctx"].compress(j["frames"], peaks=j.get("peaks"), npeaks=j.get("npeaks"))
            chain += j["ctx"].last_launch_count
    torch.cuda.synchronize()
    with rb.Graph(jobs, fused=True) as g:
        g.launch()
        torch.cuda.synchronize()
        joint_roi = sum(1 for j in jobs if prm[j["name"]].roi_coder and j["ctx"].resolved_path == rb.PATH_FUSED)
        assert g.launch_count == 1 + 3 * joint_roi + chain
        for j in jobs:
            p = oparams(prm[j["name"]])
            frames = j["frames"].cpu().numpy()
            out, nb, st = j["out"].cpu().numpy(), j["frame_bytes"].cpu().numpy(), j["status"].cpu().numpy()
            if j["name"] == "c":   # chunks: the oracle's call over the same frames
                ost, refs, _ = oracle.compress_frames(frames, p)
            for k in range(len(frames)):
                if j["name"] == "c":
                    o_st, ref = int(ost[k]), refs[k]
                elif j["name"] == "g":
                    cnt = int(j["npeaks"][k])
                    o_st, ref = oracle.compress_frame(frames[k], p, user_peaks=j["_pk"][k, :cnt])
                else:
                    o_st, ref = oracle.compress_frame(frames[k], p)
                assert st[k] == o_st, (j["name"], k, st[k], o_st)
                if o_st == 0:
                    assert nb[k] == len(ref) and np.array_equal(out[k, :nb[k]], ref), (j["name"], k)
    for j in jobs:
        j["ctx"].close()


def test_fused_graph_wait_limit_and_plain_only():
    """A job's wait limit reaches the joint launch (0: every frame of that job
    reports TIMEOUT, the other job is unaffected); a fused graph with no job
    on the fused path is the plain chains alone."""
    import torch
    from synthetic import FrameRecipe
    params = rb.default_params(atot_thr=300.0)
    jobs = []
    for i, geom in enumerate([(4, 37, 52), (3, 40, 44)]):
        r = FrameRecipe(geom, peaks=("uniform", 2, 8), seed=300 + i)
        f = np.stack([make_frame(r, k) for k in range(3)])
        ctx = rb.Context(geom, params, max_frames=3)
        jobs.append(dict(ctx=ctx, frames=torch.from_numpy(f).cuda(),
                         out=torch.zeros((3, ctx.bound), dtype=torch.uint8, device="cuda"),
                         frame_bytes=torch.zeros(3, dtype=torch.int64, device="cuda"),
                         status=torch.zeros(3, dtype=torch.int32, device="cuda"), name=str(geom)))
    jobs[0]["ctx"].set_wait_limit(0)
    with rb.Graph(jobs, fused=True) as g:
        assert g.launch_count == 1
        g.launch()
        torch.cuda.synchronize()
        assert (jobs[0]["status"].cpu().numpy() == rb.ERR_TIMEOUT).all()
        assert (jobs[0]["frame_bytes"].cpu().numpy() == 0).all()
        _check_every_frame_against_oracle(jobs[1:], lambda j: params)
    jobs[0]["ctx"].set_wait_limit(-1)
    chain = 0
    for j in jobs:
        j["ctx"].set_path(rb.PATH_PLAIN)
        j["ctx"].compress(j["frames"])
        chain += j["ctx"].last_launch_count
    torch.cuda.synchronize()
    with rb.Graph(jobs, fused=True) as g:
        g.launch()
        torch.cuda.synchronize()
        assert g.launch_count == chain
        _check_every_frame_against_oracle(jobs, lambda j: params)
    for j in jobs:
        j["ctx"].close()
