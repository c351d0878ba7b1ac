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

# bytes per voxel a grid holds on the device: the single-precision fields
# (sigma', sigma_a', j, phi hi/lo, D, fresh D: 28 B, up to 2x for half-row
# padding at small sizes), the FP32 inputs (12 B) and the safeguard snapshot
# (12 B)
BYTES_PER_VOXEL = 80


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

    def release(self, grid):
        grid.close()

    def close(self):
        self.server.close()


def serve(requests, backend, max_active: int = 64, memory_fraction: float = 0.9, clock=time.perf_counter,
          sleep=time.sleep, keep_grids: bool = False):
    """Run the request stream to completion; returns (requests, stats).

    A request is admitted when it has arrived, fewer than `max_active` solves
    are in flight, and its footprint fits in `memory_fraction` of the free
    device memory.  Requests are admitted in arrival order (no overtaking)."""
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    waiting = collections.deque()
    grids = {}
    by_id = {r.rid: r for r in requests}
    t0 = clock()
    steps = 0
    max_in_flight = 0
    depth = []          # requests arrived but not admitted, after each admission round
    while pending or waiting or backend.active() > 0:
        now = clock() - t0
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
        depth.append(len(waiting))
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
    done = [r for r in requests if r.finished >= 0]
    lat = np.array([r.finished - r.arrival for r in done])
    span = (max(r.finished for r in done) - min(r.arrival for r in done)) if done else 0.0
    stats = {
        "requests": len(done),
        "steps": steps,
        "max_in_flight": max_in_flight,
        "latency_s_p50": float(np.percentile(lat, 50)) if len(lat) else None,
        "latency_s_p99": float(np.percentile(lat, 99)) if len(lat) else None,
        "latency_s_mean": float(lat.mean()) if len(lat) else None,
        "queue_s_p99": float(np.percentile([r.admitted - r.arrival for r in done], 99)) if done else None,
        "queue_depth_max": max(depth) if depth else 0,
        "queue_depth_mean": float(np.mean(depth)) if depth else 0.0,
        "span_s": span,
        "throughput_req_s": len(done) / span if span > 0 else None,
    }
    return requests, stats


def footprint_bytes(n: int) -> int:
    return BYTES_PER_VOXEL * (n + 2) ** 3
