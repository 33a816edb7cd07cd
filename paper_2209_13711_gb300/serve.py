"""Serving loop: Poisson event requests, continuous batching onto resident contexts.

Each slot is one library context (geometry and connectivity resident on the
device, object buffers sized for ``max_batch`` events) with its own CUDA
stream, so the batches of different slots overlap on the device. Slots are
opened while their object buffers fit the device-memory budget. Whenever a
slot is free and requests are waiting, the scheduler packs the oldest waiting
requests (up to the slot's event, hit and seed capacity) into one batch and
launches it at once; it never waits for a batch to fill. A request's latency
runs from its arrival to the moment its track candidates are on the host.

The paper runs one event per launch and overlaps events with several CUDA
streams (Section 2.2); batching several events into one graph launch is this
library's replacement, and this loop applies it to a live request stream.

The scheduler is pure host logic over an abstract slot (``launch``, ``ready``,
``collect``, ``capacity``, ``device_bytes``) and an injectable clock, so it can
be driven by fake slots on a virtual clock as well as by device slots.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    event: int               # index into the event pool
    arrival: float           # seconds on the scheduler clock
    n_hits: int = 0
    n_seeds: int = 0
    launched: float = math.nan
    done: float = math.nan
    slot: int = -1
    batch_size: int = 0
    result: object = None
    error: str | None = None

    @property
    def latency(self):
        return self.done - self.arrival


@dataclasses.dataclass
class SlotCapacity:
    max_events: int
    max_hits: int
    max_seeds: int


def poisson_arrivals(rate_hz, n, seed=0, start=0.0):
    """n arrival times of a Poisson process of the given rate (exponential gaps)."""
    rng = np.random.default_rng(seed)
    if rate_hz == math.inf:
        return np.full(n, float(start))
    return start + np.cumsum(rng.exponential(1.0 / rate_hz, n))


class Scheduler:
    """Continuous batching of requests onto slots under a memory budget.

    make_slot(i) -> slot; slots are opened on demand while the sum of their
    ``device_bytes`` stays within ``budget_bytes`` and their number within
    ``max_slots`` (at least one slot is always opened).
    """

    def __init__(self, make_slot, budget_bytes, max_slots=3, max_batch=16, clock=time.perf_counter,
                 idle=None, balance=True):
        self.make_slot = make_slot
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.max_batch = int(max_batch)
        self.clock = clock
        self.idle = idle or host_idle
        self.balance = balance
        self.slots = []
        self.busy = {}                 # slot index -> list of requests in flight
        self.used_bytes = 0
        self.batches = []              # (slot, size, launch time)

    # -- slots ------------------------------------------------------------
    def _can_open(self):
        if len(self.slots) >= self.max_slots:
            return False
        if not self.slots:
            return True
        per = self.slots[0].device_bytes
        return self.used_bytes + per <= self.budget

    def _open(self):
        s = self.make_slot(len(self.slots))
        if self.slots and self.used_bytes + s.device_bytes > self.budget:
            raise RuntimeError("slot does not fit the device-memory budget")
        self.slots.append(s)
        self.used_bytes += s.device_bytes
        return len(self.slots) - 1

    def _free_slots(self):
        return [i for i in range(len(self.slots)) if i not in self.busy]

    # -- batching ---------------------------------------------------------
    def _take(self, queue, slot, limit):
        """Oldest waiting requests that fit the slot's capacity (FIFO, no skipping)."""
        cap = slot.capacity
        batch, h, s = [], 0, 0
        limit = min(limit, cap.max_events, self.max_batch)
        while queue and len(batch) < limit:
            r = queue[0]
            if h + r.n_hits > cap.max_hits or s + r.n_seeds > cap.max_seeds:
                break
            batch.append(queue.popleft())
            h += r.n_hits
            s += r.n_seeds
        return batch

    def _now(self):
        return self.clock() - self._t0

    def _reject_oversize(self, queue, cap):
        kept = collections.deque()
        rejected = []
        for r in queue:
            if r.n_hits > cap.max_hits or r.n_seeds > cap.max_seeds:
                r.error = "event exceeds the slot capacity"
                r.done = self._now()
                rejected.append(r)
            else:
                kept.append(r)
        return kept, rejected

    def _collect(self, i):
        reqs = self.busy.pop(i)
        res = self.slots[i].collect(len(reqs))
        t = self._now()
        for r, out in zip(reqs, res):
            r.result = out
            r.done = t
        return reqs

    # -- the loop ---------------------------------------------------------
    def run(self, requests):
        """Serve requests (sorted by arrival) to completion; returns them with times filled."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue = collections.deque()
        finished = []
        k = 0
        n = len(pending)
        self._t0 = self.clock()
        if not self.slots:
            self._open()
        while len(finished) < n:
            now = self._now()
            while k < n and pending[k].arrival <= now:
                queue.append(pending[k])
                k += 1
            progressed = False
            for i in list(self.busy):
                if self.slots[i].ready():
                    finished.extend(self._collect(i))
                    progressed = True
            if queue:
                queue, rej = self._reject_oversize(queue, self.slots[0].capacity)
                finished.extend(rej)
            free = self._free_slots()
            if queue and not free and self._can_open():
                free = [self._open()]
            for j, i in enumerate(free):
                if not queue:
                    break
                share = len(queue)
                if self.balance:
                    share = -(-len(queue) // (len(free) - j))
                batch = self._take(queue, self.slots[i], share)
                if not batch:
                    break
                t = self._now()
                for r in batch:
                    r.launched = t
                    r.slot = i
                    r.batch_size = len(batch)
                self.slots[i].launch(batch)
                self.busy[i] = batch
                self.batches.append((i, len(batch), t))
                progressed = True
            if not progressed:
                nxt = pending[k].arrival - now if k < n else math.inf
                self.idle(min(nxt, 5e-5) if self.busy else nxt)
        return sorted(finished, key=lambda r: r.rid)


def host_idle(dt):
    """Wait on the host: sleep for long gaps, spin for short ones."""
    if dt > 2e-4:
        time.sleep(min(dt, 1e-3) - 1e-4)


def summarize(reqs, wall_s=None):
    """p50/p99/max latency (ms) and sustained throughput of served requests."""
    ok = [r for r in reqs if r.error is None]
    lat = np.array([r.latency for r in ok]) * 1e3
    first = min(r.arrival for r in reqs) if reqs else 0.0
    last = max(r.done for r in reqs) if reqs else 0.0
    span = wall_s if wall_s is not None else (last - first)
    sizes = np.array([r.batch_size for r in ok]) if ok else np.zeros(1)
    return dict(requests=len(reqs), served=len(ok), rejected=len(reqs) - len(ok),
                p50_ms=float(np.percentile(lat, 50)) if len(lat) else None,
                p99_ms=float(np.percentile(lat, 99)) if len(lat) else None,
                max_ms=float(lat.max()) if len(lat) else None,
                events_per_s=len(ok) / span if span > 0 else None,
                mean_batch=float(sizes.mean()))


# -- device slots ---------------------------------------------------------------

class EventPool:
    """Events held once in pinned host memory, with a per-event view of each array.

    Requests name an event of the pool; its inputs are already in pinned memory
    when the request arrives, so a batch's host-to-device copies are
    asynchronous.
    """

    def __init__(self, events):
        import torch
        from .lst import pack_events
        b = pack_events(list(events))
        self.hit_off = b["hit_off"].astype(np.int64)
        self.seed_off = b["seed_off"].astype(np.int64)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        f = {k: pin(b[k]) for k in ("x", "y", "z", "module", "side")}
        seeds = pin(b["seeds"])
        self.views = []
        for e in range(len(self.hit_off) - 1):
            a, c = int(self.hit_off[e]), int(self.hit_off[e + 1])
            v = {k: f[k][a:c] for k in f}
            v["seeds"] = seeds[9 * int(self.seed_off[e]):9 * int(self.seed_off[e + 1])]
            self.views.append(v)
        self._keep = (f, seeds)
        self.n_hits = np.diff(self.hit_off)
        self.n_seeds = np.diff(self.seed_off)

    def __len__(self):
        return len(self.n_hits)


class DeviceSlot:
    """A library context on its own stream. A batch's events are gathered from
    the pool's pinned views by the library (one asynchronous copy per array
    and event) and its track candidates come back packed, in two copies."""

    def __init__(self, module_table, maps, pool, cfg=None, max_events=16, hits_per_event=140000,
                 seeds_per_event=10000, device=0, fetch=True):
        import torch
        from . import lst as L
        self.L = L
        self.pool = pool
        self.fetch = fetch
        cap = L.default_capacity(max_events, max_hits=hits_per_event * max_events,
                                 max_seeds=seeds_per_event * max_events)
        self.ctx = L.Context(module_table, maps, cfg=cfg, capacity=cap, device=device)
        self.capacity = SlotCapacity(cap.max_events, cap.max_hits, cap.max_seeds)
        self.stream = torch.cuda.Stream(device=torch.device("cuda", device))
        self.device_bytes = self.ctx.device_bytes
        # results land in pinned host memory (a direct copy, not one staged through a driver buffer)
        self._rec_buf = torch.empty(cap.max_events * cap.tc_per_event * L.TC_DTYPE.itemsize,
                                    dtype=torch.uint8).pin_memory()
        self.records = self._rec_buf.numpy().view(L.TC_DTYPE)

    def launch(self, batch):
        self.ctx.run_events([self.pool.views[r.event] for r in batch], stream=self.stream.cuda_stream)

    def ready(self):
        return self.ctx.done()

    def collect(self, n):
        if not self.fetch:
            return [None] * n
        off, rec = self.ctx.batch_track_candidates(out=self.records)
        return [self.L.tc_dict(rec[off[j]:off[j + 1]]) for j in range(n)]

    def close(self):
        self.ctx.close()


def make_requests(pool_sizes, rate_hz, n, seed=0):
    """n requests with Poisson arrivals, each naming a random event of the pool."""
    n_hits, n_seeds = pool_sizes
    rng = np.random.default_rng(seed + 1)
    t = poisson_arrivals(rate_hz, n, seed)
    ev = rng.integers(0, len(n_hits), n)
    return [Request(i, int(ev[i]), float(t[i]), int(n_hits[ev[i]]), int(n_seeds[ev[i]])) for i in range(n)]


def serve(module_table, maps, pool, requests, cfg=None, budget_bytes=60 << 30, max_slots=3, max_batch=16,
          fetch=True, slots=None):
    """Run the serving loop on device slots; returns (requests, scheduler).

    slots: already-opened DeviceSlots to reuse (their graphs stay captured).
    """
    made = []

    def make(i):
        if slots is not None and i < len(slots):
            return slots[i]
        s = DeviceSlot(module_table, maps, pool, cfg=cfg, max_events=max_batch, fetch=fetch)
        made.append(s)
        return s

    sch = Scheduler(make, budget_bytes, max_slots=max_slots, max_batch=max_batch, idle=host_idle)
    out = sch.run(requests)
    return out, sch
