"""Scheduling of the continuous-batching server on the host, with fake stream
operations (no GPU): each stream's requests run one at a time in submission
order, different streams run concurrently up to the slot count, a request
starts only when the memory budget allows it, waits while it does not, and
fails with LMS_ENOMEM when it never can."""
import threading
import time

import numpy as np

from paper_2111_04289_b300 import lmstream as lm


class FakeStreams:
    """Streams 1..k; a push sleeps a little and grows the stream's memory."""

    def __init__(self, grow_per_row=10, base=1000, seed=0):
        self.lock = threading.Lock()
        self.held = {}
        self.log = []  # (stream, n_rows, start, end)
        self.running = set()
        self.max_running = 0
        self.grow = grow_per_row
        self.base = base
        self.rng = np.random.default_rng(seed)
        self.violations = []
        self.budget = None

    def push(self, s, b):
        n = int(b.n_rows)
        with self.lock:
            assert s not in self.running, "two pushes of one stream at once"
            self.running.add(s)
            self.max_running = max(self.max_running, len(self.running))
            dt = float(self.rng.uniform(0.002, 0.01))
            t0 = time.perf_counter()
        time.sleep(dt)
        with self.lock:
            self.held[s] = self.held.get(s, self.base) + self.grow * n
            if self.budget is not None and sum(self.held.values()) > self.budget:
                self.violations.append(sum(self.held.values()))
            self.running.discard(s)
            self.log.append((s, n, t0, time.perf_counter()))
        return lm.LMS_OK

    def push_bytes(self, s, n, host):
        return 3 * self.grow * n  # what a push may allocate transiently

    def device_bytes(self, s):
        with self.lock:
            return self.held.get(s, self.base)

    def ops(self):
        return (self.push, self.push_bytes, self.device_bytes)


def _batch(n):
    b = lm.BatchC()
    b.n_rows = n
    return b


def test_per_stream_order_and_concurrency():
    f = FakeStreams()
    sv = lm.Server(slots=3, ops=f.ops())
    tickets = []
    for i in range(40):
        s = 1 + i % 5
        tickets.append((s, i, sv.submit(s, batch=_batch(100 + i))))
    for _, _, t in tickets:
        st, a, b = sv.wait(t)
        assert st == lm.LMS_OK and b >= a
    stats = sv.stats()
    sv.close()
    assert stats["completed"] == 40
    assert 2 <= stats["max_concurrent"] <= 3
    assert f.max_running <= 3
    for s in range(1, 6):
        mine = [n for (ss, n, _, _) in sorted(f.log, key=lambda x: x[2]) if ss == s]
        assert mine == sorted(mine), "a stream's batches ran out of submission order"


def test_memory_budget_admission_waits_and_holds():
    f = FakeStreams(grow_per_row=10, base=1000)
    # five streams of 1000 bytes; each push grows one by 2000 and reserves 6000:
    # two fit at first, then one at a time, and all five fit in the end
    budget = 19000
    f.budget = budget
    sv = lm.Server(slots=4, memory_budget_bytes=budget, ops=f.ops())
    ts = [sv.submit(1 + i, batch=_batch(200)) for i in range(5)]
    for t in ts:
        assert sv.wait(t)[0] == lm.LMS_OK
    stats = sv.stats()
    assert stats["memory_waits"] > 0
    assert stats["max_concurrent"] == 2
    assert stats["held_bytes"] == 15000 and stats["peak_bytes"] <= budget
    assert not f.violations
    # a request whose reserve alone exceeds what is left can never start
    t = sv.submit(1, batch=_batch(1000))
    assert sv.wait(t)[0] == lm.LMS_ENOMEM
    # a small one still can
    t = sv.submit(2, batch=_batch(10))
    assert sv.wait(t)[0] == lm.LMS_OK
    sv.close()


def test_wait_timeout_and_bad_ticket():
    f = FakeStreams()
    sv = lm.Server(slots=1, ops=f.ops())
    t = sv.submit(1, batch=_batch(5))
    st, _, _ = sv.wait(t)
    assert st == lm.LMS_OK
    try:
        sv.wait(t + 100)
        raise AssertionError("expected LMS_EINVAL")
    except lm.LmsError as e:
        assert e.status == lm.LMS_EINVAL
    sv.close()
