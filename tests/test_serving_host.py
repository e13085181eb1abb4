"""The open-loop serving driver (serving.poisson_run) on the CPU, against a
fake pool with a fixed service time and a bounded number of concurrent
requests: every arrival is either served once or rejected, latencies are at
least the service time, admission control rejects only when the wait queue
is full, and the arrival process is the seeded Poisson process."""
import time
from collections import deque
from types import SimpleNamespace

import numpy as np

from paper_2604_12902_gb300 import serving


class FakePool:
    """Requests run `service` seconds each, at most `slots` at a time; the
    rest wait first-in-first-out, like the device pool's admission."""

    def __init__(self, service: float, slots: int):
        self.service, self.slots = service, slots
        self.next_ticket = 1
        self.waiting = deque()
        self.running = {}          # ticket -> finish time
        self.done = deque()
        self.size = {}
        self.submitted = 0

    def _advance(self):
        now = time.perf_counter()
        for t, fin in sorted(self.running.items(), key=lambda kv: kv[1]):
            if fin <= now:
                del self.running[t]
                self.done.append(t)
        while self.waiting and len(self.running) < self.slots:
            self.running[self.waiting.popleft()] = time.perf_counter() + self.service

    def submit(self, wl, max_steps):
        t = self.next_ticket
        self.next_ticket += 1
        self.size[t] = wl.num_vms
        self.submitted += 1
        self.waiting.append(t)
        self._advance()
        return t

    def info(self):
        self._advance()
        return {"waiting": len(self.waiting), "running": len(self.running)}

    def next_done(self):
        self._advance()
        return self.done.popleft() if self.done else 0

    def read(self, t):
        return {"steps": np.full(self.size.pop(t), 3, np.uint64)}


def _arrivals(lam, duration, seed):
    """Number of arrivals of the seeded Poisson process within `duration`."""
    rng = np.random.default_rng(seed)
    t, n = rng.exponential(1.0 / lam), 0
    while t < duration:
        n += 1
        t += rng.exponential(1.0 / lam)
    return n


def test_every_arrival_is_served_once_with_latency_above_service():
    reqs = [SimpleNamespace(num_vms=n) for n in (5, 7, 11)]
    pool = FakePool(service=0.002, slots=64)
    out = serving.poisson_run(pool, reqs, lam=500.0, duration=0.3, seed=4, poll_interval=1e-4)
    want = _arrivals(500.0, 0.3, 4)
    assert out["requests"] == pool.submitted == want and out["rejected"] == 0
    assert not pool.size and not pool.running and not pool.waiting          # all read back
    assert (out["latencies"] >= 0.002).all()
    sizes = [reqs[k % 3].num_vms for k in range(want)]
    assert out["vm_steps"] == 3 * sum(sizes)
    assert abs(out["mean_vms"] - np.mean(sizes)) < 1e-9
    assert out["p50_ms"] <= out["p99_ms"]


def test_admission_control_rejects_only_when_the_wait_queue_is_full():
    reqs = [SimpleNamespace(num_vms=4)]
    pool = FakePool(service=0.02, slots=1)          # 50 requests/s capacity, offered 400/s
    out = serving.poisson_run(pool, reqs, lam=400.0, duration=0.3, seed=9, poll_interval=1e-4,
                              max_waiting=2)
    want = _arrivals(400.0, 0.3, 9)
    assert out["requests"] + out["rejected"] == want
    assert out["rejected"] > 0 and out["requests"] == pool.submitted
    assert (out["latencies"] >= 0.02).all()
    # at most 1 running + 2 waiting ahead of any served request
    assert out["latencies"].max() < 0.5
