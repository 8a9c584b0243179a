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


class _Slot:
    """One batch's buffers in a lane: frames in, streams out, and the batch's
    progress (idle -> sizes -> bytes -> host -> idle)."""

    def __init__(self, geometry, max_frames, stride, device):
        import torch
        self.d_frames = torch.empty((max_frames, *geometry), dtype=torch.float32, device=device)
        self.d_out = torch.empty((max_frames, stride), dtype=torch.uint8, device=device)
        self.d_nb = torch.empty(max_frames, dtype=torch.int64, device=device)
        self.d_st = torch.empty(max_frames, dtype=torch.int32, device=device)
        self.h_nb = torch.empty(max_frames, dtype=torch.int64).pin_memory()
        self.h_st = torch.empty(max_frames, dtype=torch.int32).pin_memory()
        # the batch's streams come back packed, back to back, into one pinned
        # buffer; host copies out of it run on the server's thread pool
        self.h_packed = None
        self.offsets: list = []
        self.futures: list = []
        self.batch: list = []
        self.n = 0
        self.phase = "idle"
        self.event = None

    @property
    def bytes(self):
        return sum(t.numel() * t.element_size() for t in (self.d_frames, self.d_out, self.d_nb, self.d_st))


class _Lane:
    """One context and its streams, with two batch slots, so that a batch can
    start (its frames copied in and its kernels queued behind the running
    batch) while the previous batch's streams are still being copied out.
    Frames come in on `in_stream`, are compressed on `stream` and go out on
    `out_stream`; events order the three.  Requests whose frames are already in
    device memory (a detector writing into HBM) are gathered into the slot by
    device-to-device copies, or compressed where they are when the batch is a
    single request."""

    PACKED_START = 64 << 20  # pinned bytes for a batch's streams at first; grown on demand
    SLOTS = 2

    def __init__(self, geometry, params: Params, max_frames: int, device, budget: int, pool,
                 keep_streams: bool = True, output: str = "host"):
        """Raises RoibinError(ERR_OUT_OF_BUDGET) when the lane does not fit `budget` bytes."""
        import torch
        self.geometry = geometry
        self.max_frames = max_frames
        self.stride = compress_bound(geometry, params)
        buffers = self.SLOTS * max_frames * (int(np.prod(geometry)) * 4 + self.stride + 12)
        if buffers >= budget:
            raise RoibinError("lane buffers", ERR_OUT_OF_BUDGET)
        # the library refuses (without allocating) a scratch above the budget left
        self.ctx = Context(geometry, params, max_frames=max_frames, hbm_budget=budget - buffers,
                           device=device.index or 0)
        self.stream = torch.cuda.Stream(device=device)
        self.in_stream = torch.cuda.Stream(device=device)
        self.out_stream = torch.cuda.Stream(device=device)
        self.slots = [_Slot(geometry, max_frames, self.stride, device) for _ in range(self.SLOTS)]
        self.pool = pool
        self.keep_streams = keep_streams
        self.output = output
        self.last_used = 0.0
        self.bytes = self.ctx.scratch_bytes + buffers

    @property
    def phase(self):
        """"idle" when no slot holds a batch."""
        return "idle" if all(s.phase == "idle" for s in self.slots) else "busy"

    def free_slot(self):
        for s in self.slots:
            if s.phase == "idle":
                return s
        return None

    def start(self, batch, slot=None):
        import torch
        slot = slot or self.free_slot()
        slot.batch = batch
        slot.n = sum(r.frames.shape[0] for r in batch)
        frames = slot.d_frames[:slot.n]
        f0 = batch[0].frames
        if len(batch) == 1 and f0.is_cuda and f0.is_contiguous() and f0.data_ptr() % 16 == 0:
            frames = f0  # already in device memory: compressed where it is
        else:
            with torch.cuda.stream(self.in_stream):
                k = 0
                for r in batch:
                    m = r.frames.shape[0]
                    slot.d_frames[k:k + m].copy_(r.frames, non_blocking=True)
                    k += m
            self.stream.wait_stream(self.in_stream)
        with torch.cuda.stream(self.stream):
            self.ctx.compress(frames, out=slot.d_out, out_stride=self.stride, frame_bytes=slot.d_nb,
                              status=slot.d_st, stream=self.stream)
        # the sizes (and later the streams) leave on the output stream, so the
        # next batch's kernels can follow this one at once
        self.out_stream.wait_stream(self.stream)
        with torch.cuda.stream(self.out_stream):
            slot.h_nb[:slot.n].copy_(slot.d_nb[:slot.n], non_blocking=True)
            slot.h_st[:slot.n].copy_(slot.d_st[:slot.n], non_blocking=True)
            slot.event = torch.cuda.Event()
            slot.event.record(self.out_stream)
        slot.phase = "sizes"

    def _finish(self, slot, with_streams):
        now = time.perf_counter()
        st = slot.h_st[:slot.n].numpy()
        k = 0
        for r in slot.batch:
            m = r.frames.shape[0]
            r.status = [int(x) for x in st[k:k + m]]
            r.done = now
            k += m
        finished, slot.batch, slot.phase = slot.batch, [], "idle"
        self.last_used = now
        return finished

    def advance(self):
        """Moves the running batches on when their copies are done; returns finished requests."""
        out = []
        for slot in self.slots:
            out.extend(self._advance(slot))
        return out

    def _advance(self, slot):
        import torch
        if slot.phase == "idle":
            return []
        if slot.phase in ("sizes", "bytes") and not slot.event.query():
            return []
        if slot.phase == "sizes":
            if self.output == "device":  # the streams stay in the slot's device buffer
                return self._finish(slot, False)
            nb, st = slot.h_nb[:slot.n].numpy(), slot.h_st[:slot.n].numpy()
            slot.offsets, total = [], 0
            for k in range(slot.n):
                m = int(nb[k]) if st[k] == 0 else 0
                slot.offsets.append((total, m))
                total += m
            if slot.h_packed is None or total > slot.h_packed.numel():
                size = max(total, self.PACKED_START if slot.h_packed is None else 2 * slot.h_packed.numel())
                slot.h_packed = torch.empty(size, dtype=torch.uint8).pin_memory()
            with torch.cuda.stream(self.out_stream):
                for k, (o, m) in enumerate(slot.offsets):
                    if m:
                        slot.h_packed[o:o + m].copy_(slot.d_out[k, :m], non_blocking=True)
                slot.event = torch.cuda.Event()
                slot.event.record(self.out_stream)
            slot.phase = "bytes"
            return []
        if slot.phase == "bytes":
            if not self.keep_streams:  # the bytes are on the host: done
                return self._finish(slot, False)
            # each request's streams are copied out of the pinned buffer in parallel
            packed = slot.h_packed.numpy()
            st = slot.h_st[:slot.n].numpy().copy()
            k = 0
            slot.futures = []
            for r in slot.batch:
                m = r.frames.shape[0]
                spans = slot.offsets[k:k + m]
                stats = [int(x) for x in st[k:k + m]]
                slot.futures.append(self.pool.submit(
                    lambda spans=spans, stats=stats: (stats, [packed[o:o + n].copy() if s == 0 else None
                                                              for (o, n), s in zip(spans, stats)])))
                k += m
            slot.phase = "host"
            return []
        if not all(f.done() for f in slot.futures):
            return []
        now = time.perf_counter()
        for r, f in zip(slot.batch, slot.futures):
            r.status, r.streams = f.result()
            r.done = now
        finished, slot.batch, slot.futures, slot.phase = slot.batch, [], [], "idle"
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
    a consumer would write them out); output: "host" (streams copied to host
    memory) or "device" (a request is done once its streams are in device
    memory, as for a consumer on the GPU).  A request's frames may be in host
    memory (pinned) or already in device memory."""

    def __init__(self, params: Params | None = None, hbm_budget: int = 40 << 30, lane_frames: int = 128,
                 lanes_per_geometry: int = 2, device=None, host_threads: int = 8,
                 max_queued_frames: int = 1 << 20, keep_streams: bool = True, output: str = "host"):
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
        if output not in ("host", "device"):
            raise ValueError("output is 'host' or 'device'")
        self.output = output
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
        # a lane with a free slot takes the batch, even while its other slot runs
        free = [l for l in self.lanes if l.geometry == geometry and l.free_slot() is not None]
        if free:
            return free[0]
        if sum(1 for l in self.lanes if l.geometry == geometry) >= self.lanes_per_geometry:
            return None
        while True:
            try:
                lane = _Lane(geometry, self.params, self.lane_frames, self.device,
                             self.budget - self.held_bytes, self.pool, self.keep_streams, self.output)
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
    # pools: geometry -> frames (pinned host or device tensor [n, P, H, W])
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
    ap.add_argument("--input", choices=["host", "device"], default="host",
                    help="requests' frames in pinned host memory, or already in device memory")
    ap.add_argument("--output", choices=["host", "device"], default="host",
                    help="a request is done when its streams are in host memory, or in device memory")
    args = ap.parse_args()
    pools = {}
    for name in ("cspad_batch", "epix_hot", "jungfrau_mixed"):
        r = RECIPES[name]
        host = torch.from_numpy(make_batch_threaded(r, args.pool_frames))
        pools[r.geometry] = host.cuda() if args.input == "device" else host.pin_memory()
    # epix-like frames with 1% hot pixels hold about 3,600 accepted peaks (pairs of hot pixels pass
    # the tests), above the default list size: allow the largest
    params = default_params(max_peaks=args.max_peaks)
    server = Server(params, hbm_budget=int(args.budget_gb * 1e9), lane_frames=args.lane_frames,
                    max_queued_frames=args.max_queued_frames, keep_streams=False, output=args.output)
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
    print(json.dumps({"input": args.input, "output": args.output, "requests": len(reqs), "frames": frames,
                      "seconds": wall,
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
