"""Continuous-batching serving loop for FLD solves.

Requests (independent volumes of uneven size, each with its own medium,
albedo and light) arrive over time.  The loop admits a waiting request when
a solve slot is free and the GPU has room for its grid (free device memory
from the allocator, against the request's footprint), creates and bakes its
grid on the device, and hands it to a running `fld_server`: it joins the next
step, shares the device with the solves already in flight, and leaves as
soon as it converges.  Latency is completion time minus arrival time.

All device work happens in the library (`fld_server_*`, `fld_create_grid`,
`fld_bake_*`); this module only schedules.  The backend is injectable so the
scheduling logic can be tested without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

# bytes per padded voxel a grid holds on the device once admitted (the server
# allocates all of it at admission): the single-precision fields (sigma',
# sigma_a', j, phi hi/lo, D, fresh D: 28 B), the FP32 inputs (12 B), the
# safeguard snapshot (12 B), the FP64 fields of the FP64 stop test (sigma',
# sigma_a', j, phi, D, fresh D: 48 B) and their snapshot (16 B); Anderson
# mixing adds 12 B per history slot plus 8 B.  Half-row padding of the
# colour-split layout adds up to 2x at small edges (accounted for below).
BYTES_PER_VOXEL = 116
BYTES_PER_ANDERSON_SLOT = 12


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float              # seconds after the start of the stream
    n: int                      # cubic edge length
    medium: tuple               # (sigma_t, albedo) float32 arrays or tensors
    light: object               # fld_inputs.Light
    footprint: int = 0          # device bytes
    admitted: float = -1.0
    finished: float = -1.0
    result: object = None


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson stream: exponential gaps of mean 1/rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


class GpuBackend:
    """The library on one GPU."""

    def __init__(self, params, stream=None, device=0):
        import torch

        from . import Grid, Server
        self.torch = torch
        self.Grid = Grid
        self.device = torch.device("cuda", device)
        self.stream = stream
        self.params = params
        self.Server = Server
        self.server = Server(params, stream)

    def free_bytes(self) -> int:
        free, _ = self.torch.cuda.mem_get_info(self.device)
        return int(free)

    def admit(self, req: Request):
        n = req.n
        g = self.Grid(n, n, n, 1.0 / n, stream=self.stream)
        sig, alb = req.medium
        g.set_medium(sig, alb)
        lt = req.light
        if lt.kind == "point":
            g.bake_point(lt.pos, lt.power)
        else:
            g.bake_directional(lt.dir, lt.radiance)
        self.server.add(g, req.rid)
        return g

    def active(self) -> int:
        return self.server.active

    def step(self):
        return self.server.step()

    def updates(self) -> int:
        return self.server.updates

    def release(self, grid):
        grid.close()

    def reset(self):
        # a fresh server: grids released while in flight leave the old one
        self.server.close()
        self.server = self.Server(self.params, self.stream)

    def close(self):
        self.server.close()


def serve(requests, backend, max_active: int = 64, memory_fraction: float = 0.9, clock=time.perf_counter,
          sleep=time.sleep, keep_grids: bool = False, deadline: float | None = None):
    """Run the request stream to completion (or until `deadline` seconds after
    the start, for a stream one device cannot keep up with); returns
    (requests, stats).

    A request is admitted when it has arrived, fewer than `max_active` solves
    are in flight, and its footprint fits in `memory_fraction` of the free
    device memory.  Requests are admitted in arrival order (no overtaking).
    queue_depth_mean is time-weighted: the number of arrived, not yet
    admitted requests integrated over the run, divided by its length."""
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    waiting = collections.deque()
    grids = {}
    by_id = {r.rid: r for r in requests}
    t0 = clock()
    steps = 0
    max_in_flight = 0
    depth_max = 0
    depth_area = 0.0    # integral of the queue depth over time
    t_last, d_last = 0.0, 0
    stopped = False
    while pending or waiting or backend.active() > 0:
        now = clock() - t0
        if deadline is not None and now >= deadline:
            stopped = True
            break
        while pending and pending[0].arrival <= now:
            waiting.append(pending.popleft())
        while waiting and backend.active() < max_active:
            req = waiting[0]
            if req.footprint > memory_fraction * backend.free_bytes():
                break
            waiting.popleft()
            req.admitted = clock() - t0
            grids[req.rid] = backend.admit(req)
        max_in_flight = max(max_in_flight, backend.active())
        t_now = clock() - t0
        depth_area += d_last * (t_now - t_last)
        t_last, d_last = t_now, len(waiting)
        depth_max = max(depth_max, d_last)
        if backend.active() == 0:
            if pending:
                sleep(max(0.0, min(0.01, pending[0].arrival - (clock() - t0))))
                continue
            if waiting:
                raise RuntimeError(f"request {waiting[0].rid} does not fit on the device")
        for rid, res in backend.step():
            req = by_id[rid]
            req.finished = clock() - t0
            req.result = res
            g = grids.pop(rid)
            if keep_grids:
                req.grid = g
            else:
                backend.release(g)
        steps += 1
    t_end = clock() - t0
    depth_area += d_last * (t_end - t_last)
    work = backend.updates() if hasattr(backend, "updates") else None
    if stopped:      # release what the deadline left in flight: the server
        backend.reset()  # first (it hands its grids back), then the grids
        for rid, g in list(grids.items()):
            backend.release(g)
        grids.clear()
    done = [r for r in requests if r.finished >= 0]
    lat = np.array([r.finished - r.arrival for r in done])
    span = (max(r.finished for r in done) - min(r.arrival for r in done)) if done else 0.0
    arrived = [r for r in requests if r.arrival <= t_end]
    stats = {
        "requests": len(done),
        "arrived": len(arrived),
        "unfinished_at_deadline": len(requests) - len(done) if stopped else 0,
        "admitted_unfinished": sum(1 for r in requests if r.admitted >= 0 and r.finished < 0),
        "run_s": t_end,
        "voxel_updates": work,
        "steps": steps,
        "max_in_flight": max_in_flight,
        "latency_s_p50": float(np.percentile(lat, 50)) if len(lat) else None,
        "latency_s_p99": float(np.percentile(lat, 99)) if len(lat) else None,
        "latency_s_mean": float(lat.mean()) if len(lat) else None,
        "queue_s_p99": float(np.percentile([r.admitted - r.arrival for r in done], 99)) if done else None,
        "queue_depth_max": depth_max,
        "queue_depth_mean": depth_area / t_end if t_end > 0 else 0.0,
        "span_s": span,
        "throughput_req_s": len(done) / span if span > 0 else None,
    }
    return requests, stats


def footprint_bytes(n: int, anderson: int = 0) -> int:
    """Device bytes of an admitted n^3 grid: per padded voxel, with the
    colour-split layout's half rows rounded up to 32 elements."""
    hpx = (31 + (n + 2) // 2 + 1 + 31) // 32 * 32
    padded = 2 * hpx * (n + 2) * (n + 2)
    per = BYTES_PER_VOXEL + (BYTES_PER_ANDERSON_SLOT * anderson + 8 if anderson else 0)
    return per * padded
