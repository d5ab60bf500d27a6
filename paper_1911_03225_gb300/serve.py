"""Continuous-batching server for FDM simulations.

Requests (grid side, step count, precision, initial U13) arrive over time.  Resident
simulations live in device *groups*: a group is a ``Batch`` of ``group_size`` slots of one
class (grid, precision), allocated when a request of that class finds no free slot and the
group's device bytes fit the HBM budget, and released again when it has no resident
simulation and its memory is wanted by another class (or when the server closes).  So the
budget is a ledger of device memory actually held: ``bytes_in_use`` is the sum of the
device bytes of the allocated groups at every moment, and a request waits when a new group
would take the ledger over the budget, even though its class still has slots to give.

Each group steps on its own CUDA stream; a tick enqueues ``tick_steps`` batched steps for
every group with residents, so the groups' work overlaps on the device, then retires the
simulations whose step budget is spent (reading their result back) and admits waiting
requests into free slots.  A request whose class is not served, whose group alone exceeds
the budget, or whose input is refused is retired at once as failed; one whose simulation
stops being finite is retired with the library's status and its slot freed; the others
carry on.
"""
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

from .binding import (Batch, FDMError, Params, FP64, MIXED, batch_device_bytes, FDM_ERR_INVALID_ARG,
                      FDM_ERR_OOM)


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


class _Group:
    """One device group: a Batch of `size` slots of one class on its own stream."""

    def __init__(self, cls, params: List[Params], nbytes: int, stream):
        self.cls = cls
        self.stream = stream
        self.batch = Batch(params, stream=stream.cuda_stream if stream is not None else None)
        self.nbytes = nbytes
        self.slots: List[Optional[Tuple[Request, float]]] = [None] * len(params)

    def free_slot(self) -> Optional[int]:
        for s, v in enumerate(self.slots):
            if v is None:
                return s
        return None

    def residents(self) -> int:
        return sum(v is not None for v in self.slots)


class Server:
    """``classes`` maps (n, precision) -> the most simulations of that class resident at
    once; ``base`` gives every other parameter.  Groups hold ``group_size`` slots (at most the
    class's limit).  ``hbm_budget`` bounds the device bytes of the allocated groups."""

    def __init__(self, base: Params, classes: Dict[Tuple[int, int], int], hbm_budget: float,
                 tick_steps: int = 16, keep_fields: bool = True, group_size: int = 8):
        self.base = base
        self.classes = dict(classes)
        self.tick_steps = tick_steps
        self.hbm_budget = hbm_budget
        self.keep_fields = keep_fields
        self.group_size = max(1, int(group_size))
        self.groups: List[_Group] = []
        self.bytes_in_use = 0                # device bytes of the allocated groups
        self.peak_bytes = 0
        self.groups_allocated = 0
        self.groups_released = 0
        self.failed: List[Result] = []
        self.launched_steps = 0
        self._bytes_cache: Dict[Tuple[int, int], int] = {}

    # ------------------------------------------------------------------ groups and ledger
    def _params(self, cls) -> Params:
        n, prec = cls
        return Params(**{**self.base.__dict__, "n1": n, "n2": n, "precision": prec})

    def _slots_per_group(self, cls) -> int:
        return max(1, min(self.group_size, self.classes.get(cls, 0)))

    def group_bytes(self, cls) -> int:
        """Device bytes one group of this class holds."""
        if cls not in self._bytes_cache:
            self._bytes_cache[cls] = batch_device_bytes([self._params(cls)] * self._slots_per_group(cls))
        return self._bytes_cache[cls]

    @property
    def resident(self) -> int:
        return sum(g.residents() for g in self.groups)

    def _resident_of(self, cls) -> int:
        return sum(g.residents() for g in self.groups if g.cls == cls)

    def _stream(self):
        try:
            import torch
            return torch.cuda.Stream() if torch.cuda.is_available() else None
        except ImportError:
            return None

    def _allocate(self, cls) -> Optional[_Group]:
        need = self.group_bytes(cls)
        if self.bytes_in_use + need > self.hbm_budget:
            # release idle groups (no resident simulation) until the new one fits
            for g in [g for g in self.groups if g.residents() == 0]:
                if self.bytes_in_use + need <= self.hbm_budget:
                    break
                self._release(g)
        if self.bytes_in_use + need > self.hbm_budget:
            return None
        g = _Group(cls, [self._params(cls)] * self._slots_per_group(cls), need, self._stream())
        self.groups.append(g)
        self.bytes_in_use += need
        self.peak_bytes = max(self.peak_bytes, self.bytes_in_use)
        self.groups_allocated += 1
        return g

    def _release(self, g: _Group) -> None:
        g.batch.close()
        self.groups.remove(g)
        self.bytes_in_use -= g.nbytes
        self.groups_released += 1

    def warm(self) -> int:
        """Allocates one group of every offered class while the budget allows (a server's
        start-up: the first request of a class then finds its group ready).  Returns the
        number of groups allocated."""
        k = 0
        for cls in sorted(self.classes):
            if self.classes[cls] > 0 and not any(g.cls == cls for g in self.groups):
                if self.bytes_in_use + self.group_bytes(cls) <= self.hbm_budget and self._allocate(cls):
                    k += 1
        return k

    # ------------------------------------------------------------------ admission
    def _reject_reason(self, r: Request) -> int:
        """A status if the request can never be served (class not offered, or one group of
        its class alone over the budget), else 0."""
        cls = (r.n, r.precision)
        if self.classes.get(cls, 0) < 1:
            return FDM_ERR_INVALID_ARG
        try:
            nbytes = self.group_bytes(cls)
        except FDMError:
            return FDM_ERR_INVALID_ARG
        if nbytes == 0:
            return FDM_ERR_INVALID_ARG
        return FDM_ERR_OOM if nbytes > self.hbm_budget else 0

    def _admit(self, queue: deque, now: float) -> None:
        """Admit, first come first served, every waiting request that finds a free slot of
        its class, or room in the budget for a new group of it; the others keep waiting."""
        keep = deque()
        while queue:
            r = queue.popleft()
            cls = (r.n, r.precision)
            g = next((g for g in self.groups if g.cls == cls and g.free_slot() is not None), None)
            if g is None:
                if self._resident_of(cls) >= self.classes[cls]:
                    keep.append(r)
                    continue
                g = self._allocate(cls)
                if g is None:
                    keep.append(r)
                    continue
            s = g.free_slot()
            try:
                g.batch.set_plastic_distortion(s, r.up13)
            except FDMError as e:   # refused input (e.g. non-finite): fails alone, slot stays free
                self.failed.append(Result(r.rid, r.n, r.steps, r.precision, r.arrival, now, now, None, 0.0,
                                          e.status))
                continue
            g.batch.set_budget(s, r.steps)
            g.slots[s] = (r, now)
        queue.extend(keep)

    # ------------------------------------------------------------------ serving loop
    def run(self, requests: List[Request], clock: Callable[[], float] = None, max_seconds: float = 3600.0,
            monitor: Callable[["Server"], None] = None) -> Tuple[List[Result], dict]:
        """Serve `requests` in real time; returns results and stats.  `monitor(server)`, if
        given, is called after every tick (with every group synchronised)."""
        t0 = time.perf_counter()
        clock = clock or (lambda: time.perf_counter() - t0)
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queue: deque = deque()
        results: List[Result] = []
        max_queue = 0
        max_resident = 0
        ticks = 0
        launches = 0
        while pending or queue or self.resident:
            now = clock()
            if now > max_seconds:
                break
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                why = self._reject_reason(r)
                if why:
                    self.failed.append(Result(r.rid, r.n, r.steps, r.precision, r.arrival, now, now, None, 0.0, why))
                else:
                    queue.append(r)
            self._admit(queue, now)
            max_queue = max(max_queue, len(queue))
            max_resident = max(max_resident, self.resident)
            active = [g for g in self.groups if g.residents() > 0]
            if not active:
                if queue and not pending:   # cannot happen: an empty device admits any servable request
                    raise RuntimeError("requests wait with no simulation resident")
                time.sleep(max(0.0, min(pending[0].arrival - clock(), 0.01)) if pending else 0.0)
                continue
            for g in active:
                g.batch.enqueue_steps(self.tick_steps)
                launches += self.tick_steps * g.batch.launches_per_step()
            self.launched_steps += self.tick_steps
            synced = [(g,) + tuple(g.batch.sync_status()) for g in active]
            ticks += 1
            done_at = clock()
            for g, left, status in synced:
                for s, v in enumerate(g.slots):
                    if v is None:
                        continue
                    r, adm = v
                    if status[s] != 0:
                        # the simulation left the finite range: retire it as failed, free its slot
                        g.batch.set_budget(s, 0)
                        self.failed.append(Result(r.rid, r.n, r.steps, r.precision, r.arrival, adm, done_at, None,
                                                  0.0, int(status[s])))
                        g.slots[s] = None
                    elif left[s] == 0:
                        f = g.batch.read_fields(s, "up13") if self.keep_fields else {}
                        info = g.batch.info(s)
                        if info.step != r.steps:
                            raise FDMError(0, "request %d took %d steps, expected %d" % (r.rid, info.step, r.steps))
                        results.append(Result(r.rid, r.n, r.steps, r.precision, r.arrival, adm, done_at,
                                              f.get("up13"), info.t))
                        g.slots[s] = None
            if monitor is not None:
                monitor(self)
        elapsed = clock()
        lat = np.array([r.latency for r in results]) if results else np.zeros(1)
        work = sum(r.n * r.n * r.steps for r in results)
        stats = {"completed": len(results), "failed": len(self.failed), "submitted": len(requests),
                 "elapsed_s": elapsed,
                 "cell_steps": work, "cell_steps_per_s": work / elapsed if elapsed > 0 else 0.0,
                 "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                 "max_queue": max_queue, "max_resident": max_resident, "ticks": ticks,
                 "tick_steps": self.tick_steps, "launches": launches,
                 "hbm_budget_bytes": self.hbm_budget, "peak_bytes": self.peak_bytes,
                 "groups_allocated": self.groups_allocated, "groups_released": self.groups_released}
        return results, stats

    def close(self):
        for g in list(self.groups):
            self._release(g)
