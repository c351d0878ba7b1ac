"""Host logic of the continuous-batching serving loop, on a fake backend and
a fake clock (no GPU): arrivals, admission by free slots and free memory,
arrival-order admission, latency accounting."""
import numpy as np
import pytest

from paper_1403_8105_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeBackend:
    """Each admitted request needs `n // 8` steps; a step takes 0.01 s."""

    def __init__(self, clock, free=10_000, step_s=0.01):
        self.clock = clock
        self.free = free
        self.step_s = step_s
        self.inflight = {}
        self.log = []

    def free_bytes(self):
        return self.free

    def admit(self, req):
        self.free -= req.footprint
        self.inflight[req.rid] = [req.n // 8, req.footprint]
        self.log.append(("admit", req.rid, len(self.inflight)))
        return req.rid

    def active(self):
        return len(self.inflight)

    def step(self):
        self.clock.t += self.step_s
        out = []
        for rid in list(self.inflight):
            self.inflight[rid][0] -= 1
            if self.inflight[rid][0] <= 0:
                self.free += self.inflight.pop(rid)[1]
                out.append((rid, {"status": 0}))
        return out

    def release(self, grid):
        # a grid may only be released once the server no longer holds it
        assert grid not in self.inflight, "released a grid the server still holds"

    def reset(self):
        self.inflight.clear()
        self.log.append(("reset",))


def _requests(count=40, rate=50.0, seed=3, foot=100):
    arr = serve.poisson_arrivals(count, rate, seed)
    rng = np.random.default_rng(seed)
    return [serve.Request(rid=i, arrival=float(arr[i]), n=int(rng.integers(8, 64)), medium=None, light=None,
                          footprint=foot) for i in range(count)]


def test_poisson_arrivals_rate_and_order():
    a = serve.poisson_arrivals(20000, 200.0, 1)
    assert np.all(np.diff(a) > 0)
    assert abs(20000 / a[-1] - 200.0) < 6.0          # ~3 sigma of the rate estimate
    assert np.array_equal(a, serve.poisson_arrivals(20000, 200.0, 1))


def test_every_request_completes_with_consistent_times():
    clk = FakeClock()
    reqs, st = serve.serve(_requests(), FakeBackend(clk), max_active=8, clock=clk, sleep=clk.sleep)
    assert st["requests"] == 40
    for r in reqs:
        assert r.arrival <= r.admitted <= r.finished
    assert st["latency_s_p99"] >= st["latency_s_p50"] > 0


def test_admission_respects_slots_and_memory():
    clk = FakeClock()
    be = FakeBackend(clk, free=1000)
    reqs, st = serve.serve(_requests(foot=300), be, max_active=8, memory_fraction=1.0, clock=clk, sleep=clk.sleep)
    assert st["max_in_flight"] <= 3                      # 1000 B of room, 300 B each
    assert all(n <= 3 for kind, rid, n in be.log)
    clk = FakeClock()
    be = FakeBackend(clk, free=10 ** 9)
    reqs, st = serve.serve(_requests(), be, max_active=2, clock=clk, sleep=clk.sleep)
    assert st["max_in_flight"] <= 2


def test_admission_keeps_arrival_order():
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs, _ = serve.serve(_requests(), be, max_active=4, clock=clk, sleep=clk.sleep)
    admitted = [rid for kind, rid, n in be.log]
    arrival_order = [r.rid for r in sorted(reqs, key=lambda r: r.arrival)]
    assert admitted == arrival_order


def test_request_that_never_fits_is_reported():
    clk = FakeClock()
    with pytest.raises(RuntimeError):
        serve.serve(_requests(count=3, foot=10 ** 6), FakeBackend(clk, free=1000), clock=clk, sleep=clk.sleep)


def test_queue_depth_reflects_the_slot_limit():
    # one slot and a burst of arrivals: requests pile up while the slot is
    # busy; with many slots nobody waits
    clk = FakeClock()
    _, st1 = serve.serve(_requests(rate=500.0), FakeBackend(clk), max_active=1, clock=clk, sleep=clk.sleep)
    clk = FakeClock()
    _, st64 = serve.serve(_requests(rate=500.0), FakeBackend(clk, free=10 ** 9), max_active=64, clock=clk,
                          sleep=clk.sleep)
    assert st1["queue_depth_max"] > 5 and st1["queue_depth_mean"] > 1.0
    assert st64["queue_depth_max"] == 0 and st64["queue_depth_mean"] == 0.0
    # (with free slots a request still waits for the step in flight when it arrives)
    assert st64["queue_s_p99"] <= 0.0101
    assert st1["queue_s_p99"] > 10 * st64["queue_s_p99"]


def test_queue_depth_mean_is_time_weighted():
    # three requests at t = 0, one slot, two 0.01 s steps each: two wait for
    # 0.02 s, one more for another 0.02 s, then none -- the mean over the
    # 0.06 s run is (2 * 0.02 + 1 * 0.02) / 0.06 = 1, however often the loop
    # samples the queue
    clk = FakeClock()
    reqs = [serve.Request(rid=i, arrival=0.0, n=16, medium=None, light=None, footprint=1) for i in range(3)]
    _, st = serve.serve(reqs, FakeBackend(clk), max_active=1, clock=clk, sleep=clk.sleep)
    assert st["requests"] == 3 and st["queue_depth_max"] == 2
    assert st["queue_depth_mean"] == pytest.approx(1.0, rel=1e-9)


def test_deadline_stops_an_overloaded_stream():
    # a stream one slot cannot keep up with: the loop stops at the deadline,
    # counts what is unfinished, releases the solves in flight and resets
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs, st = serve.serve(_requests(count=200, rate=400.0), be, max_active=1, clock=clk, sleep=clk.sleep,
                           deadline=0.5)
    assert 0.5 <= st["run_s"] < 0.52
    assert 0 < st["requests"] < 200 and st["unfinished_at_deadline"] == 200 - st["requests"]
    assert st["arrived"] > st["requests"]
    assert ("reset",) in be.log and be.active() == 0
    assert all(r.finished < 0 or r.finished <= 0.52 for r in reqs)


def test_footprint_counts_the_padded_layout():
    # 64^3: half rows of 96 elements (31 + 33 + 1 = 65, rounded up to a
    # multiple of 32), 66 x 66 rows, two colours; 116 bytes per padded voxel,
    # 12 more per Anderson slot plus 8
    assert serve.footprint_bytes(64) == 116 * 2 * 96 * 66 * 66
    assert serve.footprint_bytes(64, anderson=8) == (116 + 12 * 8 + 8) * 2 * 96 * 66 * 66
