"""The serving loop: continuous batching across geometries, HBM-budget
admission, and each request's bytes equal to compressing it alone."""
import numpy as np
import pytest

import oracle
import paper_2206_11297_gb300 as rb
from paper_2206_11297_gb300 import serving
from synthetic import FrameRecipe, make_frame


def test_poisson_schedule_is_seeded_and_bounded():
    pools = {(2, 8, 8): np.zeros((10, 2, 8, 8), np.float32), (1, 4, 4): np.zeros((5, 1, 4, 4), np.float32)}
    a = serving.poisson_requests(pools, rate_hz=500, seconds=0.2, max_frames=4, seed=3)
    b = serving.poisson_requests(pools, rate_hz=500, seconds=0.2, max_frames=4, seed=3)
    assert a == b and 40 < len(a) < 200
    for t, g, n, first in a:
        assert 0 < t <= 0.2 and 1 <= n <= 4 and 0 <= first <= pools[g].shape[0] - n
    assert [x[0] for x in a] == sorted(x[0] for x in a)


def _pools(geoms, n=24):
    import torch
    pools = {}
    for i, g in enumerate(geoms):
        r = FrameRecipe(g, peaks=("uniform", 2, 10), seed=50 + i)
        pools[g] = torch.from_numpy(np.stack([make_frame(r, k) for k in range(n)])).pin_memory()
    return pools


def _alone(pools, req, params):
    import torch
    g = req.geometry
    with rb.Context(g, params, max_frames=req.frames.shape[0]) as ctx:
        out, nb, st = ctx.compress(req.frames.cuda().clone())  # a fresh, 16-byte aligned copy
        torch.cuda.synchronize()
        out, nb, st = out.cpu().numpy(), nb.cpu().numpy(), st.cpu().numpy()
    return [out[k, :nb[k]] if st[k] == 0 else None for k in range(len(nb))]


def _check_mixed(server, pools, schedule, params):
    reqs = serving.run(pools, schedule, server)
    assert len(reqs) == len(schedule)
    for r in reqs:
        assert r.done is not None and r.latency >= 0
        assert all(s == 0 for s in r.status)
        alone = _alone(pools, r, params)
        for mine, ref in zip(r.streams, alone):
            assert np.array_equal(mine, ref)
    # and against the oracle for one frame of each geometry
    seen = set()
    for r in reqs:
        if r.geometry in seen:
            continue
        seen.add(r.geometry)
        st, ref = oracle.compress_frame(r.frames[0].cpu().numpy(), oracle.make_params(**params.as_dict()))
        assert st == 0 and np.array_equal(r.streams[0], ref)
    return reqs


@pytest.mark.gpu
def test_mixed_geometries_same_bytes_alone_and_in_the_mix():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    geoms = [(3, 40, 44), (4, 37, 52), (2, 21, 27)]   # two fused shapes and one plain-path shape
    pools = _pools(geoms)
    params = rb.default_params(atot_thr=300.0)
    schedule = serving.poisson_requests(pools, rate_hz=2000, seconds=0.05, max_frames=8, seed=7)
    server = serving.Server(params, hbm_budget=4 << 30, lane_frames=16, lanes_per_geometry=2)
    try:
        reqs = _check_mixed(server, pools, schedule, params)
        assert {r.geometry for r in reqs} == set(geoms)
    finally:
        server.close()


@pytest.mark.gpu
def test_budget_admission_releases_idle_lanes():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    geoms = [(3, 40, 44), (4, 37, 52)]
    pools = _pools(geoms)
    params = rb.default_params(atot_thr=300.0)
    # room for one lane at a time: the other geometry waits until the first lane is released
    one = serving.Server(params, hbm_budget=1 << 40, lane_frames=16)
    for g in geoms:
        one._lane_for(g)
    lane_bytes = max(l.bytes for l in one.lanes)
    one.close()
    schedule = [(0.0, geoms[k % 2], 4, 4 * (k // 2)) for k in range(8)]
    server = serving.Server(params, hbm_budget=int(lane_bytes * 1.5), lane_frames=16, lanes_per_geometry=1)
    try:
        _check_mixed(server, pools, schedule, params)
        assert len(server.lanes) == 1 and server.held_bytes <= server.budget
    finally:
        server.close()


def test_queue_is_bounded():
    """Requests beyond max_queued_frames waiting frames are refused and counted;
    starting a batch frees their room (no GPU needed: nothing is scheduled)."""
    server = serving.Server(rb.default_params(), lane_frames=8, max_queued_frames=10)
    try:
        g = (1, 4, 4)
        mk = lambda rid, n: serving.Request(rid, np.zeros((n, *g), np.float32), 0.0)
        assert server.submit(mk(0, 6)) and server.submit(mk(1, 4))
        assert not server.submit(mk(2, 1)) and server.rejected == 1
        assert server.queued_frames == 10 and len(server.queues[g]) == 2
        with pytest.raises(ValueError):
            server.submit(mk(3, 9))   # larger than a lane's batch
    finally:
        server.close()


@pytest.mark.gpu
def test_packed_buffer_grows_and_streams_stay_exact(monkeypatch):
    """A lane's pinned buffer starts small here, so batches outgrow it and it is
    reallocated; every request's bytes still equal compressing it alone."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    monkeypatch.setattr(serving._Lane, "PACKED_START", 4096)
    geoms = [(3, 40, 44), (2, 21, 27)]
    pools = _pools(geoms)
    params = rb.default_params(atot_thr=300.0)
    schedule = serving.poisson_requests(pools, rate_hz=1000, seconds=0.05, max_frames=8, seed=11)
    server = serving.Server(params, hbm_budget=4 << 30, lane_frames=16)
    try:
        _check_mixed(server, pools, schedule, params)
        grown = [sl.h_packed.numel() for l in server.lanes for sl in l.slots if sl.h_packed is not None]
        assert grown and all(n > 4096 for n in grown)
    finally:
        server.close()


@pytest.mark.gpu
def test_requests_done_without_keeping_streams():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    geoms = [(3, 40, 44)]
    pools = _pools(geoms)
    params = rb.default_params(atot_thr=300.0)
    schedule = serving.poisson_requests(pools, rate_hz=1000, seconds=0.05, max_frames=8, seed=12)
    server = serving.Server(params, hbm_budget=4 << 30, lane_frames=16, keep_streams=False)
    try:
        reqs = serving.run(pools, schedule, server)
        assert len(reqs) == len(schedule) and server.rejected == 0
        assert all(r.done is not None and r.streams is None and all(s == 0 for s in r.status) for r in reqs)
    finally:
        server.close()


def _device_pools(geoms, n=24):
    return {g: t.cuda() for g, t in _pools(geoms, n).items()}


@pytest.mark.gpu
def test_device_resident_requests_same_bytes():
    """Frames already in device memory (a detector writing into HBM): a batch of
    one request is compressed where it lies, larger batches are gathered by
    device copies; every request's bytes still equal compressing it alone."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    geoms = [(3, 40, 44), (2, 21, 27)]   # the second has frames that are not 16-byte multiples
    pools = _device_pools(geoms)
    params = rb.default_params(atot_thr=300.0)
    schedule = serving.poisson_requests(pools, rate_hz=2000, seconds=0.05, max_frames=8, seed=13)
    server = serving.Server(params, hbm_budget=4 << 30, lane_frames=16)
    try:
        _check_mixed(server, pools, schedule, params)
    finally:
        server.close()


@pytest.mark.gpu
def test_device_output_and_a_second_batch_while_the_first_runs():
    """With output in device memory a request is done once its streams are on
    the GPU; a lane starts a second batch in its other slot while the first
    batch still runs, instead of waiting for it."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = (4, 37, 52)
    pools = _device_pools([g], n=40)
    params = rb.default_params(atot_thr=300.0)
    server = serving.Server(params, hbm_budget=4 << 30, lane_frames=16, lanes_per_geometry=1,
                            output="device")
    try:
        r1 = serving.Request(0, pools[g][0:16], 0.0)
        r2 = serving.Request(1, pools[g][16:32], 0.0)
        lane = server._lane_for(g)
        # a bounded spin (about 0.1 s) ahead of r1's kernels on the lane's
        # stream, so that r1 is certain to be running when r2 is scheduled
        with torch.cuda.stream(lane.stream):
            torch.cuda._sleep(200_000_000)
        assert server.submit(r1)
        server.step()
        assert server.submit(r2)
        server.step()   # r1's batch is still on the GPU: r2 goes to the other slot
        assert sum(sl.phase != "idle" for sl in lane.slots) == 2 and len(server.lanes) == 1
        server.drain()
        for r in (r1, r2):
            assert r.done is not None and r.streams is None and all(x == 0 for x in r.status)
        # the second slot's streams are the second request's, byte for byte
        sl = lane.slots[1]  # free_slot gave r1 the first slot and r2 the second
        alone = _alone(pools, r2, params)
        nb = sl.h_nb.numpy()
        for k in range(16):
            assert np.array_equal(sl.d_out[k, :nb[k]].cpu().numpy(), alone[k])
    finally:
        server.close()
