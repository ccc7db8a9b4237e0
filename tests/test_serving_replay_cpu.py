"""The served replay of the serving benchmark against a fake server: requests
are handed over at their arrival times, not a loop turn later, whether the
server is idle or busy, and every completion is collected.  The fake keeps
a clock that each call moves on, as host work does: a poll or a wait costs
a few microseconds, a clock read a fraction of one.  No GPU."""
import numpy as np
import pytest

from paper_2004_09883_gb300 import serving


class FakeServer:
    """fb_fft_server_* semantics on a simulated clock (seconds)."""

    def __init__(self, service_s, call_s=5e-6, tick_s=2e-7):
        self.t = 0.0
        self.call_s, self.tick_s = call_s, tick_s
        self.service = service_s
        self.running = []  # (completion time, tag)
        self.done = []
        self.submitted = {}

    def clock(self):
        self.t += self.tick_s
        return self.t

    def _retire(self):
        keep = []
        for td, tag in self.running:
            if td <= self.t:
                self.done.append((tag, 0, 0, self.submitted[tag], self.submitted[tag], self.t))
            else:
                keep.append((td, tag))
        self.running = keep

    def submit_many(self, reqs, first, count):
        self.t += self.call_s
        for k in range(first, first + count):
            self.submitted[k] = self.t
            self.running.append((self.t + self.service[k], k))
        return [0] * count

    def wait(self, until):
        # returns once a request has finished, nothing runs, or the clock reaches `until`
        self.t += self.call_s
        while True:
            self._retire()
            if self.done or not self.running or self.t >= until:
                return
            self.t += self.tick_s

    def poll(self):
        self.t += self.call_s
        self._retire()
        out, self.done = self.done, []
        return out

    def drain(self):
        while self.running:
            self.t += self.tick_s
            self._retire()


class FakeWorkload:
    def __init__(self, n):
        self.shapes = [(64,)] * n

    def requests(self, host_io=False):
        return None

    def bytes_moved(self):
        return 16 * 64 * len(self.shapes)


@pytest.mark.parametrize("gap_us", [1000.0, 200.0])
def test_idle_server_gets_each_request_at_its_arrival(gap_us):
    n = 200
    service = np.full(n, 20e-6)
    srv = FakeServer(service)
    arrivals = np.arange(n) * gap_us * 1e-6
    st = serving.run_served(srv, FakeWorkload(n), arrivals)
    assert st["requests"] == n
    sub = np.array([srv.submitted[k] for k in range(n)])
    late = sub - (arrivals + (sub[0] - arrivals[0]))
    # handed over within a clock read (plus the submit call) of the arrival,
    # not a poll/wait turn later
    assert late.max() <= srv.call_s + 3 * srv.tick_s
    # latency = the submit call + the service time (the wait watches it finish)
    assert st["p50_ms"] == pytest.approx((srv.call_s + 20e-6) * 1e3, abs=0.002)


def test_busy_server_collects_every_completion():
    n = 300
    rng = np.random.default_rng(3)
    service = rng.uniform(5e-6, 200e-6, n)
    srv = FakeServer(service)
    arrivals = np.cumsum(rng.exponential(20e-6, n))  # faster than it serves: queues build up
    st = serving.run_served(srv, FakeWorkload(n), arrivals)
    assert st["requests"] == n and np.isfinite(st["p99_ms"])
    assert not srv.running and not srv.done
