"""Continuous-batching server for FDM simulations.

Requests (grid side, step count, precision, initial U13) arrive over time.  The server owns
one ``Batch`` whose slots are grouped by (grid, precision); all resident simulations stay
on the device and advance together, ``tick_steps`` batched steps per tick.  Between ticks
it retires the simulations whose step budget is spent (reading their result back) and
admits waiting requests into free slots while the device memory of the resident set stays
within the HBM budget.  A request whose input is refused, or whose simulation stops being
finite, is retired as failed (``Server.failed``, with the library status) and its slot freed;
the others carry on.  Requests that arrive while others run are admitted as soon as a
slot and memory are free; their work then shares every launch with the running ones.
"""
import math
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

from .binding import Batch, FDMError, Params, FP64, MIXED, batch_device_bytes


@dataclass
class Request:
    rid: int
    n: int
    steps: int
    precision: int          # FP64 or MIXED
    arrival: float          # seconds after the start of the run
    up13: np.ndarray = field(repr=False, default=None)


@dataclass
class Result:
    rid: int
    n: int
    steps: int
    precision: int
    arrival: float
    admitted: float
    finished: float
    up13: Optional[np.ndarray] = field(repr=False, default=None)
    t: float = 0.0
    status: int = 0          # 0, or the library status that failed the request

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process with the given mean rate (seeded)."""
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=count)
    return np.cumsum(gaps)


class Server:
    """``classes`` maps (n, precision) -> number of slots; ``base`` gives every other
    parameter.  ``hbm_budget`` bounds the device bytes of the resident simulations."""

    def __init__(self, base: Params, classes: Dict[Tuple[int, int], int], hbm_budget: float,
                 tick_steps: int = 16, stream: Optional[int] = None, keep_fields: bool = True):
        self.tick_steps = tick_steps
        self.hbm_budget = hbm_budget
        self.keep_fields = keep_fields
        self.slot_class: List[Tuple[int, int]] = []
        params = []
        for (n, prec), k in sorted(classes.items()):
            for _ in range(k):
                q = Params(**{**base.__dict__, "n1": n, "n2": n, "precision": prec})
                params.append(q)
                self.slot_class.append((n, prec))
        self.params = params
        self.slot_bytes = [batch_device_bytes([q]) for q in params]
        self.batch = Batch(params, stream=stream)
        self.free: Dict[Tuple[int, int], deque] = {}
        for s, c in enumerate(self.slot_class):
            self.free.setdefault(c, deque()).append(s)
        self.bytes_in_use = 0
        self.resident: Dict[int, Tuple[Request, float]] = {}   # slot -> (request, admitted time)
        self.failed: List[Result] = []
        self.launched_steps = 0

    def _admit(self, queue: deque, now: float) -> None:
        """Admit every waiting request that has a free slot of its class and fits the
        budget (first come first served, skipping requests that cannot start yet)."""
        keep = deque()
        while queue:
            r = queue.popleft()
            c = (r.n, r.precision)
            slots = self.free.get(c)
            if not slots:
                keep.append(r)
                continue
            s = slots[0]
            if self.bytes_in_use + self.slot_bytes[s] > self.hbm_budget:
                keep.append(r)
                continue
            try:
                self.batch.set_plastic_distortion(s, r.up13)
            except FDMError as e:   # refused input (e.g. non-finite): fails alone, slot stays free
                self.failed.append(Result(r.rid, r.n, r.steps, r.precision, r.arrival, now, now, None, 0.0,
                                          e.status))
                continue
            slots.popleft()
            self.batch.set_budget(s, r.steps)
            self.bytes_in_use += self.slot_bytes[s]
            self.resident[s] = (r, now)
        queue.extend(keep)

    def run(self, requests: List[Request], clock: Callable[[], float] = None,
            max_seconds: float = 3600.0) -> Tuple[List[Result], dict]:
        """Serve `requests` (sorted by arrival) in real time; returns results and stats."""
        t0 = time.perf_counter()
        clock = clock or (lambda: time.perf_counter() - t0)
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queue: deque = deque()
        results: List[Result] = []
        max_queue = 0
        ticks = 0
        while pending or queue or self.resident:
            now = clock()
            if now > max_seconds:
                break
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            self._admit(queue, now)
            max_queue = max(max_queue, len(queue))
            if not self.resident:
                if pending:   # idle until the next arrival
                    time.sleep(max(0.0, min(pending[0].arrival - clock(), 0.01)))
                continue
            self.batch.enqueue_steps(self.tick_steps)
            self.launched_steps += self.tick_steps
            left, status = self.batch.sync_status()
            ticks += 1
            done_at = clock()
            for s in [s for s in self.resident if status[s] != 0]:
                # the simulation left the finite range: retire it as failed, free its slot
                r, adm = self.resident.pop(s)
                self.batch.set_budget(s, 0)
                self.failed.append(Result(r.rid, r.n, r.steps, r.precision, r.arrival, adm, done_at, None, 0.0,
                                          int(status[s])))
                self.free[(r.n, r.precision)].append(s)
                self.bytes_in_use -= self.slot_bytes[s]
            for s in [s for s in self.resident if left[s] == 0]:
                r, adm = self.resident.pop(s)
                f = self.batch.read_fields(s, "up13") if self.keep_fields else {}
                info = self.batch.info(s)
                if info.step != r.steps:
                    raise FDMError(0, "request %d took %d steps, expected %d" % (r.rid, info.step, r.steps))
                results.append(Result(r.rid, r.n, r.steps, r.precision, r.arrival, adm, done_at,
                                      f.get("up13"), info.t))
                self.free[(r.n, r.precision)].append(s)
                self.bytes_in_use -= self.slot_bytes[s]
        elapsed = clock()
        lat = np.array([r.latency for r in results]) if results else np.zeros(1)
        work = sum(r.n * r.n * r.steps for r in results)
        stats = {"completed": len(results), "failed": len(self.failed), "submitted": len(requests),
                 "elapsed_s": elapsed,
                 "cell_steps": work, "cell_steps_per_s": work / elapsed if elapsed > 0 else 0.0,
                 "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                 "max_queue": max_queue, "ticks": ticks, "tick_steps": self.tick_steps,
                 "launches": ticks * self.tick_steps * self.batch.launches_per_step()}
        return results, stats

    def close(self):
        self.batch.close()
