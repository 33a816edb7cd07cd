"""Host logic of the serving loop, driven by fake slots on a virtual clock."""
import math

import numpy as np
import pytest

from paper_2209_13711_gb300.serve import Request, Scheduler, SlotCapacity, poisson_arrivals, summarize


class VClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def idle(self, dt):
        assert math.isfinite(dt), "scheduler idled with nothing to wait for"
        self.t += max(dt, 1e-6)


class FakeSlot:
    """Serves a batch in base + per_event * n seconds of virtual time."""

    def __init__(self, clock, cap, base=2e-3, per_event=4e-4, nbytes=1000, log=None):
        self.clock = clock
        self.capacity = cap
        self.base, self.per = base, per_event
        self.device_bytes = nbytes
        self.finish = None
        self.batch = None
        self.log = log if log is not None else []

    def launch(self, batch):
        assert self.finish is None, "launch on a busy slot"
        self.batch = list(batch)
        self.finish = self.clock() + self.base + self.per * len(batch)
        self.log.append([r.rid for r in batch])

    def ready(self):
        return self.finish is not None and self.clock() >= self.finish

    def collect(self, n):
        assert n == len(self.batch)
        out = [("served", r.event) for r in self.batch]
        self.finish, self.batch = None, None
        return out


def run(reqs, cap=SlotCapacity(8, 10**6, 10**5), budget=10**9, max_slots=3, max_batch=8, nbytes=1000, **kw):
    ck = VClock()
    log = []
    made = []

    def make(i):
        s = FakeSlot(ck, cap, nbytes=nbytes, log=log, **kw)
        made.append(s)
        return s

    sch = Scheduler(make, budget, max_slots=max_slots, max_batch=max_batch, clock=ck, idle=ck.idle)
    out = sch.run(reqs)
    return out, sch, log, made


def reqs_at(times, hits=1000, seeds=100):
    return [Request(i, i % 5, float(t), hits, seeds) for i, t in enumerate(times)]


def test_every_request_served_once_in_arrival_order():
    t = poisson_arrivals(800.0, 300, seed=3)
    out, sch, log, _ = run(reqs_at(t))
    assert [r.rid for r in out] == list(range(300))
    flat = [rid for b in log for rid in b]
    assert sorted(flat) == list(range(300))
    assert flat == sorted(flat), "batches are launched first come, first served"
    for r in out:
        assert r.error is None and r.result == ("served", r.event)
        assert r.arrival <= r.launched <= r.done


def test_batches_respect_capacity_and_max_batch():
    rng = np.random.default_rng(0)
    reqs = [Request(i, 0, 0.0, int(rng.integers(100, 400)), int(rng.integers(10, 40))) for i in range(200)]
    cap = SlotCapacity(16, 1000, 90)
    out, sch, log, _ = run(reqs, cap=cap, max_batch=6)
    by_id = {r.rid: r for r in out}
    for b in log:
        assert 1 <= len(b) <= 6
        assert sum(by_id[i].n_hits for i in b) <= 1000
        assert sum(by_id[i].n_seeds for i in b) <= 90


def test_budget_limits_open_slots():
    reqs = reqs_at(np.zeros(100))
    _, sch, _, made = run(reqs, budget=2500, max_slots=4, nbytes=1000)
    assert len(made) == 2 and sch.used_bytes <= 2500
    _, sch, _, made = run(reqs_at(np.zeros(100)), budget=10**6, max_slots=4, nbytes=1000)
    assert len(made) == 4
    # the first slot opens even when it alone exceeds the budget
    _, sch, _, made = run(reqs_at(np.zeros(10)), budget=10, max_slots=4, nbytes=1000)
    assert len(made) == 1


def test_oversize_request_rejected_others_served():
    reqs = reqs_at(np.linspace(0, 0.01, 20))
    reqs[7].n_hits = 10**7
    out, _, log, _ = run(reqs)
    assert out[7].error is not None and out[7].result is None
    assert all(r.error is None for i, r in enumerate(out) if i != 7)
    assert 7 not in [rid for b in log for rid in b]
    assert summarize(out)["rejected"] == 1


def test_latency_equals_service_time_when_idle():
    # gaps far longer than a batch's service: each request runs alone and waits for nothing
    out, _, log, _ = run(reqs_at(np.arange(20) * 0.05), base=2e-3, per_event=4e-4)
    assert all(len(b) == 1 for b in log)
    lat = np.array([r.latency for r in out])
    # completion is seen at the next poll of a busy slot (every 50 us of waiting)
    assert np.all(lat >= 2.4e-3 - 1e-9) and np.all(lat <= 2.4e-3 + 5e-5 + 2e-6)


def test_continuous_batching_beats_one_event_per_launch_under_load():
    t = poisson_arrivals(3000.0, 600, seed=5)      # above what one-event launches can serve
    plain, _, plog, _ = run(reqs_at(t), max_slots=1, max_batch=1)
    batched, _, blog, _ = run(reqs_at(t), max_slots=3, max_batch=16)
    sp, sb = summarize(plain), summarize(batched)
    assert sp["mean_batch"] == 1.0
    assert sb["mean_batch"] > 2.0
    assert sb["events_per_s"] > 1.5 * sp["events_per_s"]
    assert sb["p99_ms"] < sp["p99_ms"]


def test_requests_wait_only_for_a_free_slot():
    # one slot: a request launches at its arrival when the slot is free, else when it frees
    out, sch, log, _ = run(reqs_at([0.0, 0.0005, 0.0006, 0.02]), max_slots=1, max_batch=8)
    assert log[0] == [0]
    assert log[1] == [1, 2]               # both waited for the first batch
    assert log[2] == [3]
    assert out[1].launched == pytest.approx(out[0].done, abs=2e-6)


def test_poisson_arrivals_rate():
    t = poisson_arrivals(500.0, 20000, seed=1)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 500.0) < 0.03 / 500.0
    # exponential gaps: standard deviation equals the mean
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03
    assert np.all(poisson_arrivals(math.inf, 5) == 0.0)
