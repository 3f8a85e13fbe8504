"""Continuous batching of independent wake solves on one GPU.

Requests (a plasma column, beams and a xi window each) arrive over time.  A
request is admitted as soon as the device-memory budget allows (first come,
first served); its wake is created on the device without waiting for it
(WAKE_INIT_ASYNC) and joins the running batch at the next step.  Each step
advances every admitted wake through one batched launch per launch shape for
about `step_ns` of device time (wake_batch_step with a time budget, so wakes
of different sizes end a step together); one gathered progress read per step
tells which wakes finished (or stopped at a model breakdown).  Finished wakes
hand back the fields on their beam particles and free their memory, and the
next requests in line take their place.  Ring state and beams stay on the
device for the whole solve.

Everything on the device is the library's (libwake.so); this module only
schedules: admission, steps, retirement and latency bookkeeping.
"""
from __future__ import annotations

import collections
import concurrent.futures
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import wake as wm


def estimate_device_bytes(n_rings: int, n_beam: int, n_steps: int) -> int:
    """Upper bound of the device bytes a mixed-precision wake takes (the
    arrays wake_init allocates: ~180 B per ring, ~72 B per beam particle,
    16 B per slice, plus per-allocation rounding; a beam phase space for
    the push adds 40 B per particle, not counted here)."""
    return 192 * n_rings + 80 * n_beam + 16 * (n_steps + 1) + (64 << 10)


def sm_share(launch_config) -> float:
    """SM-equivalents a wake holds while it runs: its CTAs, each taking
    threads x 128 registers of an SM's 65,536."""
    threads, _, ctas = launch_config
    if threads <= 0:  # a one-CTA march of up to 512 threads
        return 1.0
    return ctas * min(1.0, threads / 512.0)


@dataclass
class Request:
    rid: int
    arrival: float            # seconds on the server clock
    edges: np.ndarray
    beams: Sequence           # objects with xi, r, w, q (numpy or pinned torch tensors)
    dxi: float
    n_steps: int
    out_ez: Optional[object] = None   # caller's result buffers (numpy or pinned torch), optional
    out_wr: Optional[object] = None
    # filled by the server
    admitted: float = float("nan")
    finished: float = float("nan")
    status: int = -1
    slices_done: int = 0
    sm_share: float = 0.0

    @property
    def n_rings(self) -> int:
        return int(self.edges.shape[0] - 1)

    @property
    def n_beam(self) -> int:
        return int(sum((b.xi.numel() if hasattr(b.xi, "numel") else b.xi.shape[0]) for b in self.beams))

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class ServeStats:
    completed: List[Request] = field(default_factory=list)
    steps: int = 0
    max_active: int = 0
    max_queue: int = 0
    peak_bytes: int = 0

    def records(self) -> List[tuple]:
        """(arrival, finished, ring-slices done, status) per completed request."""
        return [(r.arrival, r.finished, r.n_rings * r.slices_done, r.status) for r in self.completed]

    def counters(self) -> Dict[str, int]:
        return {"steps": self.steps, "max_active": self.max_active, "max_queue": self.max_queue,
                "peak_device_bytes": self.peak_bytes}

    def summary(self) -> Dict[str, float]:
        return summarize(self.records(), [self.counters()])


def summarize(records: Sequence[tuple], counters: Sequence[Dict[str, int]]) -> Dict[str, float]:
    """Latency percentiles and throughput of completed requests (records of
    ServeStats.records, from one server or several), with each server's
    counters summed (steps) or maximised (the rest)."""
    arr = np.array([r[0] for r in records])
    fin = np.array([r[1] for r in records])
    lat = fin - arr
    rs = sum(int(r[2]) for r in records)
    span = float(fin.max() - arr.min())
    stopped = np.array([r[3] == wm.WAKE_ENONFINITE for r in records], dtype=bool)

    def part(m):
        if not m.any():
            return {"requests": 0}
        return {"requests": int(m.sum()), "p50_ms": float(np.percentile(lat[m], 50) * 1e3),
                "p99_ms": float(np.percentile(lat[m], 99) * 1e3)}
    return {"requests": len(records), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "whole_window": part(~stopped), "stopped_at_breakdown": part(stopped),
            "ring_slices": int(rs), "ring_slices_per_s": rs / span, "span_s": span,
            "steps": int(sum(c["steps"] for c in counters)),
            "max_active": int(max(c["max_active"] for c in counters)),
            "max_queue": int(max(c["max_queue"] for c in counters)),
            "peak_device_bytes": int(max(c["peak_device_bytes"] for c in counters)),
            "stopped_by_breakdown": int(sum(r[3] == wm.WAKE_ENONFINITE for r in records))}


def dispatch(work: Sequence[float], n_ranks: int) -> np.ndarray:
    """The GPU (rank) that serves each request of an arrival-ordered stream
    when wakes are partitioned over n_ranks GPUs (a wake never spans GPUs,
    so the data path needs no collective): each request goes to the rank
    with the least work assigned so far (work: its ring-slices, rings x
    slices), ties to the lowest rank.  Deterministic, so every rank computes
    the same assignment from the same stream."""
    load = np.zeros(max(1, int(n_ranks)))
    owner = np.empty(len(work), dtype=np.int64)
    for i, w in enumerate(work):
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += float(w)
    return owner


def gather_summary(stats: ServeStats) -> Dict[str, float]:
    """summarize over the requests every rank of the default process group
    served (one object all-gather, after serving: off the data path); on a
    single process, stats.summary()."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return stats.summary()
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, (stats.records(), stats.counters()))
    out = summarize([r for recs, _ in parts for r in recs], [c for _, c in parts])
    out["ranks"] = len(parts)
    out["requests_per_rank"] = [len(recs) for recs, _ in parts]
    return out


class WakeServer:
    """Admits, steps and retires wakes; see the module docstring."""

    def __init__(self, memory_budget: int, step_ns: int = 4_000_000, stream=None,
                 clock: Optional[Callable[[], float]] = None, sm_budget: Optional[float] = None,
                 tuning=None, admit_threads: int = 8):
        self.budget = int(memory_budget)
        # Wakes admitted in one round are created concurrently: wake_init's
        # host work (argument checks over every beam particle, the densest
        # slice, allocations, queued uploads) runs in the library with the
        # interpreter lock released, and at a few hundred requests per second
        # it, not the device, would otherwise pace the loop.
        self.pool = concurrent.futures.ThreadPoolExecutor(admit_threads) if admit_threads > 1 else None
        # launch shapes from an autotune.TuningTable (None: the library's
        # automatic shapes)
        self.tuning = tuning
        # Admission also stops once the running wakes fill the SMs
        # (sm_budget SM-equivalents): beyond that every wake would only run
        # slower (they share the SMs), raising everyone's latency for no
        # throughput.  None: memory alone decides.
        self.sm_budget = sm_budget
        self.sm_used = 0.0
        self.step_ns = int(step_ns)
        self.stream = stream
        self.clock = clock or time.perf_counter
        self.queue: collections.deque = collections.deque()
        self.active: List[tuple] = []   # (request, Wake, estimated bytes)
        self.used = 0
        self.stats = ServeStats()

    def submit(self, req: Request):
        self.queue.append(req)
        self.stats.max_queue = max(self.stats.max_queue, len(self.queue))

    def _admit(self):
        # first in line first, while the memory and SM budgets allow
        picked = []
        while self.queue:
            req = self.queue[0]
            est = estimate_device_bytes(req.n_rings, req.n_beam, req.n_steps)
            busy = self.active or picked
            if busy and self.used + est > self.budget:
                break
            if busy and self.sm_budget is not None and self.sm_used >= self.sm_budget:
                break
            self.queue.popleft()
            shape = self.tuning.shape_for(req.n_rings, "mixed") if self.tuning is not None else {}
            req.sm_share = sm_share(wm.wake_launch_shape(req.n_rings, n_steps=req.n_steps, **shape))
            self.used += est
            self.sm_used += req.sm_share
            picked.append((req, est, shape))

        def create(item):
            req, est, shape = item
            return wm.Wake(req.edges, req.beams, req.dxi, req.n_steps, precision="mixed",
                           flags=wm.WAKE_INIT_ASYNC, stream=self.stream, **shape)
        if self.pool is not None and len(picked) > 1:
            made = list(self.pool.map(create, picked))
        else:
            made = [create(item) for item in picked]
        now = self.clock()
        for (req, est, _), w in zip(picked, made):
            req.admitted = now
            self.active.append((req, w, est))
        self.stats.max_active = max(self.stats.max_active, len(self.active))
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)

    def step(self) -> List[Request]:
        """One scheduling step: advance the running wakes, admit, retire.
        Returns the requests that finished in this step."""
        # the step is queued first, so that creating the newly admitted
        # wakes (host-side checks and uploads) overlaps it on the device
        stepped = [w for _, w, _ in self.active]
        if stepped:
            wm.wake_batch_step(stepped, 1 << 30, self.step_ns)
        self._admit()
        if not self.active:
            return []
        wakes = [w for _, w, _ in self.active]
        nxt, st = wm.wake_batch_progress(wakes)
        self.stats.steps += 1
        done, keep = [], []
        for (req, w, est), n, s in zip(self.active, nxt, st):
            if s != 0 or n >= req.n_steps:
                done.append((req, w, est, int(n), int(s)))
            else:
                keep.append((req, w, est))
        self.active = keep
        out = []
        for req, w, est, n, s in done:
            if req.out_ez is not None or req.out_wr is not None:
                ptr = lambda a: (a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data) if a is not None else None
                wm._check(wm.load().wake_get_beam_fields(w.handle, ptr(req.out_ez), ptr(req.out_wr), None, None, 0))
            req.finished = self.clock()
            req.status = s
            req.slices_done = min(n, req.n_steps)
            w.close()
            self.used -= est
            self.sm_used -= req.sm_share
            self.stats.completed.append(req)
            out.append(req)
        return out

    def idle(self) -> bool:
        return not self.queue and not self.active


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, n))


def run_stream(server: WakeServer, requests: Sequence[Request]) -> ServeStats:
    """Feeds requests to the server at their arrival times (server clock)
    and steps until all are done."""
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    while pending or not server.idle():
        now = server.clock()
        while pending and pending[0].arrival <= now:
            server.submit(pending.popleft())
        if server.idle():
            # nothing to do before the next arrival
            wait = pending[0].arrival - server.clock()
            if wait > 0:
                time.sleep(min(wait, 0.01))
            continue
        server.step()
    return server.stats
