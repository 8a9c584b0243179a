"""A request loop for ROIBIN-SZ compression with continuous batching.

Requests of 1..N frames arrive on the host (pinned float32 [n, P, H, W]) for
any detector geometry.  The server keeps, per geometry, a few *lanes*: a
compression context with its device scratch, device buffers for one batch and
a CUDA stream.  Lanes are created on demand while the HBM budget allows and
the least recently used idle lane of another geometry is released when it
does not.  Whenever a lane is idle and requests of its geometry wait, the
waiting requests are packed into one batch (up to the lane's frame capacity),
copied to the device, compressed and copied back on the lane's stream, so
batches of different lanes overlap on the device and with the copies.  Each
frame has its own codebook, so a frame's bytes are the same whether it is
compressed alone or inside any batch.

Every step runs through the library's C ABI (roibin_compress); this module
only schedules.  Latency is measured from a request's arrival to the moment
its compressed frames are on the host.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import time

import numpy as np

from . import ERR_OUT_OF_BUDGET, Context, Params, RoibinError, compress_bound, default_params


@dataclasses.dataclass
class Request:
    rid: int
    frames: "object"          # pinned host float32 tensor [n, P, H, W]
    arrival: float            # time.perf_counter() seconds
    streams: list | None = None   # compressed frames (numpy uint8), filled on completion
    status: list | None = None
    done: float | None = None

    @property
    def geometry(self):
        return tuple(self.frames.shape[1:])

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


class _Lane:
    """One context, its batch buffers and its stream."""

    PACKED_START = 64 << 20  # pinned bytes for a batch's streams at first; grown on demand

    def __init__(self, geometry, params: Params, max_frames: int, device, budget: int, pool,
                 keep_streams: bool = True):
        """Raises RoibinError(ERR_OUT_OF_BUDGET) when the lane does not fit `budget` bytes."""
        import torch
        self.geometry = geometry
        self.max_frames = max_frames
        self.stride = compress_bound(geometry, params)
        buffers = max_frames * (int(np.prod(geometry)) * 4 + self.stride + 12)
        if buffers >= budget:
            raise RoibinError("lane buffers", ERR_OUT_OF_BUDGET)
        # the library refuses (without allocating) a scratch above the budget left
        self.ctx = Context(geometry, params, max_frames=max_frames, hbm_budget=budget - buffers,
                           device=device.index or 0)
        self.stream = torch.cuda.Stream(device=device)
        self.d_frames = torch.empty((max_frames, *geometry), dtype=torch.float32, device=device)
        self.d_out = torch.empty((max_frames, self.stride), dtype=torch.uint8, device=device)
        self.d_nb = torch.empty(max_frames, dtype=torch.int64, device=device)
        self.d_st = torch.empty(max_frames, dtype=torch.int32, device=device)
        self.h_nb = torch.empty(max_frames, dtype=torch.int64).pin_memory()
        self.h_st = torch.empty(max_frames, dtype=torch.int32).pin_memory()
        # the batch's streams come back packed, back to back, into one pinned
        # buffer; host copies out of it run on the server's thread pool
        self.h_packed = torch.empty(self.PACKED_START, dtype=torch.uint8).pin_memory()
        self.pool = pool
        self.keep_streams = keep_streams
        self.offsets: list = []
        self.futures: list = []
        self.batch: list[Request] = []
        self.n = 0
        # idle -> sizes (kernel + sizes copy in flight) -> bytes (streams copy in flight)
        #      -> host (copies out of the pinned buffer running) -> idle
        self.phase = "idle"
        self.event = None
        self.last_used = 0.0
        self.bytes = self.ctx.scratch_bytes + buffers

    def start(self, batch):
        import torch
        self.batch = batch
        self.n = sum(r.frames.shape[0] for r in batch)
        with torch.cuda.stream(self.stream):
            k = 0
            for r in batch:
                m = r.frames.shape[0]
                self.d_frames[k:k + m].copy_(r.frames, non_blocking=True)
                k += m
            self.ctx.compress(self.d_frames[:self.n], out=self.d_out, out_stride=self.stride,
                              frame_bytes=self.d_nb, status=self.d_st, stream=self.stream)
            self.h_nb[:self.n].copy_(self.d_nb[:self.n], non_blocking=True)
            self.h_st[:self.n].copy_(self.d_st[:self.n], non_blocking=True)
            self.event = torch.cuda.Event()
            self.event.record(self.stream)
        self.phase = "sizes"

    def advance(self):
        """Moves a running batch on when its copies are done; returns finished requests."""
        import torch
        if self.phase == "idle":
            return []
        if self.phase in ("sizes", "bytes") and not self.event.query():
            return []
        if self.phase == "sizes":
            nb, st = self.h_nb[:self.n].numpy(), self.h_st[:self.n].numpy()
            self.offsets, total = [], 0
            for k in range(self.n):
                m = int(nb[k]) if st[k] == 0 else 0
                self.offsets.append((total, m))
                total += m
            if total > self.h_packed.numel():
                self.h_packed = torch.empty(max(total, 2 * self.h_packed.numel()), dtype=torch.uint8).pin_memory()
            with torch.cuda.stream(self.stream):
                for k, (o, m) in enumerate(self.offsets):
                    if m:
                        self.h_packed[o:o + m].copy_(self.d_out[k, :m], non_blocking=True)
                self.event = torch.cuda.Event()
                self.event.record(self.stream)
            self.phase = "bytes"
            return []
        if self.phase == "bytes":
            if not self.keep_streams:  # the bytes are on the host: done
                now = time.perf_counter()
                st = self.h_st[:self.n].numpy()
                k = 0
                for r in self.batch:
                    m = r.frames.shape[0]
                    r.status = [int(x) for x in st[k:k + m]]
                    r.done = now
                    k += m
                finished, self.batch, self.phase = self.batch, [], "idle"
                self.last_used = now
                return finished
            # each request's streams are copied out of the pinned buffer in parallel
            packed = self.h_packed.numpy()
            st = self.h_st[:self.n].numpy().copy()
            k = 0
            self.futures = []
            for r in self.batch:
                m = r.frames.shape[0]
                spans = self.offsets[k:k + m]
                stats = [int(x) for x in st[k:k + m]]
                self.futures.append(self.pool.submit(
                    lambda spans=spans, stats=stats: (stats, [packed[o:o + n].copy() if s == 0 else None
                                                              for (o, n), s in zip(spans, stats)])))
                k += m
            self.phase = "host"
            return []
        if not all(f.done() for f in self.futures):
            return []
        now = time.perf_counter()
        for r, f in zip(self.batch, self.futures):
            r.status, r.streams = f.result()
            r.done = now
        finished, self.batch, self.futures, self.phase = self.batch, [], [], "idle"
        self.last_used = now
        return finished

    def close(self):
        self.ctx.close()


class Server:
    """Continuous-batching compression server (one GPU).

    hbm_budget: bytes of device memory the lanes may hold together;
    lane_frames: frames per batch of a lane; lanes_per_geometry: lanes a
    geometry may hold at once (more than one lets a batch start while the
    previous one of the same geometry is still copying back);
    max_queued_frames: frames that may wait (submit refuses a request beyond
    that, so an offered load above capacity is shed instead of queued without
    bound); keep_streams: hand each request a copy of its streams (False: a
    request is done once its bytes are in the lane's pinned host buffer, where
    a consumer would write them out)."""

    def __init__(self, params: Params | None = None, hbm_budget: int = 40 << 30, lane_frames: int = 128,
                 lanes_per_geometry: int = 2, device=None, host_threads: int = 8,
                 max_queued_frames: int = 1 << 20, keep_streams: bool = True):
        import torch
        self.params = params or default_params()
        self.budget = int(hbm_budget)
        self.lane_frames = int(lane_frames)
        self.lanes_per_geometry = int(lanes_per_geometry)
        self.device = torch.device(device or "cuda")
        self.queues: dict = collections.defaultdict(collections.deque)
        self.lanes: list[_Lane] = []
        self.finished: list[Request] = []
        self.pool = concurrent.futures.ThreadPoolExecutor(host_threads)
        self.max_queued_frames = int(max_queued_frames)
        self.keep_streams = bool(keep_streams)
        self.queued_frames = 0
        self.rejected = 0

    @property
    def held_bytes(self):
        return sum(lane.bytes for lane in self.lanes)

    def submit(self, req: Request) -> bool:
        """Queues the request; False (and counted in `rejected`) when the waiting
        frames would exceed max_queued_frames."""
        n = req.frames.shape[0]
        if n > self.lane_frames:
            raise ValueError(f"request of {n} frames exceeds lane_frames={self.lane_frames}")
        if self.queued_frames + n > self.max_queued_frames:
            self.rejected += 1
            return False
        self.queued_frames += n
        self.queues[req.geometry].append(req)
        return True

    def _lane_for(self, geometry):
        idle = [l for l in self.lanes if l.geometry == geometry and l.phase == "idle"]
        if idle:
            return idle[0]
        if sum(1 for l in self.lanes if l.geometry == geometry) >= self.lanes_per_geometry:
            return None
        while True:
            try:
                lane = _Lane(geometry, self.params, self.lane_frames, self.device,
                             self.budget - self.held_bytes, self.pool, self.keep_streams)
                self.lanes.append(lane)
                return lane
            except RoibinError as e:
                if e.code != ERR_OUT_OF_BUDGET:
                    raise
            # release the least recently used idle lane of a geometry nobody waits for
            victims = sorted((l for l in self.lanes if l.phase == "idle" and l.geometry != geometry
                              and not self.queues[l.geometry]), key=lambda l: l.last_used)
            if not victims:
                if not self.lanes:
                    raise RuntimeError(f"a lane for geometry {geometry} does not fit the HBM budget")
                return None   # admitted later, when memory frees up
            victims[0].close()
            self.lanes.remove(victims[0])

    def step(self):
        """One scheduling pass: finish copies, start batches.  Returns True if anything moved."""
        moved = False
        for lane in self.lanes:
            done = lane.advance()
            if done:
                self.finished.extend(done)
                moved = True
        for geometry, q in self.queues.items():
            while q:
                lane = self._lane_for(geometry)
                if lane is None:
                    break
                batch, n = [], 0
                while q and n + q[0].frames.shape[0] <= lane.max_frames:
                    r = q.popleft()
                    batch.append(r)
                    n += r.frames.shape[0]
                self.queued_frames -= n
                lane.start(batch)
                moved = True
        return moved

    def busy(self):
        return any(self.queues[g] for g in self.queues) or any(l.phase != "idle" for l in self.lanes)

    def drain(self):
        while self.busy():
            if not self.step():
                time.sleep(20e-6)

    def close(self):
        for lane in self.lanes:
            lane.close()
        self.lanes = []
        self.pool.shutdown(wait=True)


def poisson_requests(pools: dict, rate_hz: float, seconds: float, max_frames: int = 64, seed: int = 0):
    """(arrival offset, geometry, n_frames, first frame) of Poisson request arrivals: geometry
    uniform over the pools, 1..max_frames frames each (uniform)."""
    rng = np.random.default_rng(seed)
    t, out, geoms = 0.0, [], list(pools)
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > seconds:
            return out
        g = geoms[rng.integers(len(geoms))]
        n = int(rng.integers(1, max_frames + 1))
        first = int(rng.integers(0, pools[g].shape[0] - n + 1))
        out.append((t, g, n, first))


def run(pools: dict, schedule, server: Server):
    """Replays a request schedule in real time against the server; returns the accepted (and
    finished) requests; refused ones are counted in server.rejected."""
    t0 = time.perf_counter()
    pending = collections.deque(schedule)
    reqs = []
    rid = 0
    while pending or server.busy():
        now = time.perf_counter() - t0
        while pending and pending[0][0] <= now:
            at, g, n, first = pending.popleft()
            r = Request(rid, pools[g][first:first + n], t0 + at)
            rid += 1
            if server.submit(r):
                reqs.append(r)
        if not server.step():
            time.sleep(20e-6)
    return reqs


def main():
    import argparse
    import json
    import torch
    from synthetic import RECIPES, make_batch_threaded
    ap = argparse.ArgumentParser(description="ROIBIN-SZ serving loop on synthetic detector requests")
    ap.add_argument("--seconds", type=float, default=5.0)
    ap.add_argument("--rate", type=float, default=200.0, help="requests per second (Poisson)")
    ap.add_argument("--max-request-frames", type=int, default=64)
    ap.add_argument("--lane-frames", type=int, default=128)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--pool-frames", type=int, default=96)
    ap.add_argument("--max-peaks", type=int, default=8192)
    ap.add_argument("--max-queued-frames", type=int, default=8192)
    args = ap.parse_args()
    pools = {}
    for name in ("cspad_batch", "epix_hot", "jungfrau_mixed"):
        r = RECIPES[name]
        pools[r.geometry] = torch.from_numpy(make_batch_threaded(r, args.pool_frames)).pin_memory()
    # epix-like frames with 1% hot pixels hold about 3,600 accepted peaks (pairs of hot pixels pass
    # the tests), above the default list size: allow the largest
    params = default_params(max_peaks=args.max_peaks)
    server = Server(params, hbm_budget=int(args.budget_gb * 1e9), lane_frames=args.lane_frames,
                    max_queued_frames=args.max_queued_frames, keep_streams=False)
    warm = poisson_requests(pools, args.rate, 0.5, args.max_request_frames, seed=1)
    run(pools, warm, server)
    sched = poisson_requests(pools, args.rate, args.seconds, args.max_request_frames, seed=2)
    t0 = time.perf_counter()
    server.rejected = 0
    reqs = run(pools, sched, server)
    wall = time.perf_counter() - t0
    lat = np.array([r.latency for r in reqs]) * 1e3
    frames = sum(r.frames.shape[0] for r in reqs)
    in_bytes = sum(r.frames.numel() * 4 for r in reqs)
    ok = all(s == 0 for r in reqs for s in r.status)
    bad = collections.Counter((str(r.geometry), s) for r in reqs for s in r.status if s != 0)
    print(json.dumps({"requests": len(reqs), "frames": frames, "seconds": wall,
                      "offered_rate_hz": args.rate, "sustained_gbs": in_bytes / 1e9 / wall,
                      "frames_per_s": frames / wall,
                      "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                     "max": float(lat.max())},
                      "offered_requests": len(sched), "rejected_requests": server.rejected,
                      "lanes": len(server.lanes), "held_gb": server.held_bytes / 1e9, "all_ok": ok,
                      "errors": {f"{g} status {s}": c for (g, s), c in bad.items()}}))
    server.close()


if __name__ == "__main__":
    main()
