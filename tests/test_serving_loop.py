"""Host logic of the continuous-batching loop, driven by a simulated pool (no GPU).

The fake pool admits by atom count, takes a fixed time per build and per
launch, and returns per-request values that depend only on the request, so
the loop's bookkeeping (arrivals, builder threads, refusals and releases,
slot reuse, batching) is checked against a closed-form expectation.
"""

from __future__ import annotations

import threading
import time

import numpy as np
import pytest

from paper_2505_06711_gb300.serving import Request, serve_stream


class _Event:
    def __init__(self, t_done):
        self.t_done = t_done

    def query(self):
        return time.perf_counter() >= self.t_done


class FakePool:
    def __init__(self, max_atoms, max_structures, builders=3, build_s=2e-4, launch_s=1e-3):
        self.max_atoms, self.max_structures = max_atoms, max_structures
        self.builds = [None] * builders
        self.build_s, self.launch_s = build_s, launch_s
        self.lock = threading.Lock()
        self.used = {}  # slot -> (request, pending)
        self.launched_batches = []
        self.concurrent_builds = 0
        self.max_concurrent_builds = 0

    def _atoms(self):
        return sum(r.n_atoms for r, _ in self.used.values())

    def submit(self, req, builder=0):
        with self.lock:
            self.concurrent_builds += 1
            self.max_concurrent_builds = max(self.max_concurrent_builds, self.concurrent_builds)
        time.sleep(self.build_s)
        with self.lock:
            self.concurrent_builds -= 1
            if len(self.used) >= self.max_structures or self._atoms() + req.n_atoms > self.max_atoms:
                return None
            slot = min(set(range(self.max_structures)) - set(self.used))
            self.used[slot] = (req, True)
            return slot

    def launch(self):
        with self.lock:
            slots = sorted(s for s, (_, p) in self.used.items() if p)
            for s in slots:
                self.used[s] = (self.used[s][0], False)
        self.launched_batches.append(len(slots))
        return slots, _Event(time.perf_counter() + self.launch_s)

    def collect(self, slots):
        with self.lock:
            return {s: (float(self.used[s][0].base.sum()), self.used[s][0].base * 2.0) for s in slots}

    def release(self, slot):
        with self.lock:
            del self.used[slot]

    def free_slots(self):
        with self.lock:
            return self.max_structures - len(self.used)


def _requests(n, rate, seed=0):
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for _ in range(n):
        t += rng.exponential(1.0 / rate)
        m = int(rng.integers(1, 40))
        out.append(Request(t, rng.normal(size=(m, 3)), np.zeros(m, np.int32), np.eye(3) * 10.0))
    return out


@pytest.mark.parametrize("rate", [500.0, 20000.0])
def test_every_request_answered_once_with_its_own_result(rate):
    reqs = _requests(300, rate)
    pool = FakePool(max_atoms=200, max_structures=8)
    res, st = serve_stream(pool, reqs)
    assert all(r is not None for r in res)
    for q, r in zip(reqs, res):
        assert r.energy == float(q.base.sum())
        assert np.array_equal(r.forces, q.base * 2.0)
        assert r.latency >= 0.0
    assert sum(pool.launched_batches) == len(reqs)
    assert st["launches"] == len(pool.launched_batches)
    assert pool.free_slots() == pool.max_structures  # everything released
    assert st["atoms"] == sum(q.n_atoms for q in reqs)


def test_batches_form_under_load_and_builders_overlap():
    reqs = _requests(400, 1e6)  # all arrive almost at once
    pool = FakePool(max_atoms=10_000, max_structures=64, builders=4, build_s=5e-4, launch_s=5e-3)
    res, st = serve_stream(pool, reqs)
    assert all(r is not None for r in res)
    assert st["mean_batch"] > 2.0
    assert pool.max_concurrent_builds > 1


def test_request_larger_than_the_pool_is_an_error():
    reqs = _requests(5, 1000.0)
    reqs[2] = Request(reqs[2].arrival, np.zeros((500, 3)), np.zeros(500, np.int32), np.eye(3) * 10.0)
    pool = FakePool(max_atoms=100, max_structures=4)
    with pytest.raises(RuntimeError, match="empty pool"):
        serve_stream(pool, reqs)
