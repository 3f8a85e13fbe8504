"""Launch-shape autotuner for batched wakes.

A mixed-precision wake runs on the on-chip march as one CTA (up to 2048
rings) or as a thread-block cluster of up to 16 CTAs; its rings per thread
(2, 4 or 8) and CTAs per wake fix the threads per CTA.  Fewer, wider CTAs mean
fewer cluster barriers per slice; more, narrower ones a shorter chain of
block-wide steps per slice and more CTAs resident per SM.  Which wins
depends on the ring count and on how full the GPU is, so the tuner measures
it: for each size class it builds a synthetic wake of that many rings,
fills the GPU with copies of it (about `fill` x the SM count in CTAs, as a
large batch does), times one batched march per candidate shape with CUDA
events and keeps the fastest in ring-slices per second.  The automatic
shape stays unless a candidate beats it by `min_gain`, so timing noise does
not churn the table.  The global-memory marches (FP64, mobile ions, RK4,
beam grids) are tuned the same way over their block size (block_threads),
and those with mobile ions, RK4 or beam grids also over their blocks per
wake (a thread-block cluster of 2, 4 or 8 blocks of the default size).

The candidates come from the library itself (wake_launch_shape: the shape
wake_init would give, computed on the host), so the tuner never proposes a
shape the library refuses.  A TuningTable maps ring counts to shapes; a
size class stores rings per thread and rings per CTA, and shape_for(n)
turns them into the CTAs per wake of an actual ring count n, checked again
by the library (the automatic shape if the stored one does not fit n).
The serving loop (serve.WakeServer(tuning=...)) and the bench
(--autotune) apply a table when they create wakes.

Everything on the device is the library's; this module only chooses
arguments of wake_init and times batched launches.
"""
from __future__ import annotations

import json
import math
from dataclasses import asdict, dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

from . import wake as wm
from . import workloads as W

# the kinds of march a table entry applies to: the on-chip march (mixed,
# electrons over the ion column) and the global-memory marches
KINDS = ("mixed", "fp64", "ions", "rk4", "grid")
BLOCK_THREADS = (64, 128, 256, 512)
# the block size wake_init takes when block_threads is 0 (timed as the
# automatic candidate, so not again as an explicit one)
DEFAULT_BLOCK_THREADS = {"fp64": 256, "grid": 256, "ions": 512, "rk4": 512}
# the global-memory marches that also run as thread-block clusters
GM_CLUSTER_KINDS = ("ions", "rk4", "grid")
DEFAULT_SIZES = (512, 1024, 2048, 3072, 4096, 6144, 8192, 12288, 16384, 32768, 65536)


@dataclass(frozen=True)
class Candidate:
    """Arguments of wake_init for one launch shape, with what they resolve
    to for the size they were made for."""
    rings_per_thread: int = 0   # on-chip march: 0 (automatic), 2, 4 or 8
    cluster_ctas: int = 0       # on-chip march: 0 (automatic) or 1-16; ions, RK4, grids: 0 or 1-8
    block_threads: int = 0      # global-memory marches: 0 (the library's default) or 64-512
    threads: int = 0            # resolved threads per CTA (on-chip march)
    ctas: int = 1               # resolved CTAs per wake

    @property
    def automatic(self) -> bool:
        return self.rings_per_thread == 0 and self.cluster_ctas == 0 and self.block_threads == 0

    def wake_kwargs(self) -> Dict[str, int]:
        out = {}
        if self.rings_per_thread or self.cluster_ctas:
            out["rings_per_thread"] = self.rings_per_thread
            out["cluster_ctas"] = self.cluster_ctas
        if self.block_threads:
            out["block_threads"] = self.block_threads
        return out


def max_rings(kind: str) -> int:
    if kind == "mixed":
        return wm.wake_max_rings("mixed")
    if kind == "ions":
        return 4096  # cells per species with mobile ions
    return wm.wake_max_rings("fp64")  # the other global-memory marches: 8192 rings


def candidates(n_rings: int, kind: str = "mixed", max_candidates: int = 8,
               min_threads: int = 64) -> List[Candidate]:
    """The shapes worth timing for a wake of n_rings rings: the automatic
    one first, then (on-chip march) every valid (rings per thread, CTAs per
    wake) with at least min_threads threads per CTA, thinned evenly to
    max_candidates; or (global-memory marches) the block sizes 64-512 and,
    with mobile ions, RK4 or beam grids, clusters of 2, 4 and 8 blocks of
    the default size."""
    if not 1 <= n_rings <= max_rings(kind):
        raise ValueError(f"{n_rings} rings: outside [1, {max_rings(kind)}] for the {kind} march")
    if kind != "mixed":
        out = [Candidate()] + [Candidate(block_threads=t, cluster_ctas=1 if kind in GM_CLUSTER_KINDS else 0)
                               for t in BLOCK_THREADS if t != DEFAULT_BLOCK_THREADS[kind]]
        if kind in GM_CLUSTER_KINDS:
            out += [Candidate(cluster_ctas=cl, ctas=cl) for cl in (2, 4, 8)]
        return out
    t0, k0, c0 = wm.wake_launch_shape(n_rings)
    auto = Candidate(threads=t0, ctas=c0)
    seen = {(t0, k0, c0)}
    rest = []
    for k in (2, 4, 8):
        for cl in range(1, 17):
            try:
                t, kk, cc = wm.wake_launch_shape(n_rings, k, cl)
            except wm.WakeError:
                continue
            if t < min_threads or (t, kk, cc) in seen:
                continue
            seen.add((t, kk, cc))
            rest.append(Candidate(rings_per_thread=k, cluster_ctas=cl, threads=t, ctas=cc))
    rest.sort(key=lambda c: (c.ctas, c.rings_per_thread))
    keep = max(0, max_candidates - 1)
    if len(rest) > keep:
        idx = sorted({round(i * (len(rest) - 1) / max(1, keep - 1)) for i in range(keep)}) if keep else []
        rest = [rest[i] for i in idx]
    return [auto] + rest


def probe_wake(n_rings: int, slices: int, kind: str = "mixed") -> W.Wake:
    """The synthetic wake a size class is timed on: uniform rings out to 6,
    a Gaussian driver (n_b0 = 1, sigma_r = 0.5, sigma_z = 1, 20k particles,
    centred at xi = 0.5), d xi = 0.01, the first `slices` slices."""
    drv = W.gaussian_beam(20_000, 1.0, 0.5, 1.0, 0.5, seed=5)
    extra = {"ions": {"ions": (1.0, 1836.0)}, "rk4": {"integrator": "rk4"}, "grid": {"grid_nr": 32}}.get(kind, {})
    return W.Wake(f"probe{n_rings}", W.edges_uniform(n_rings, 6.0), [drv], 0.01, slices, **extra)


def _precision(kind: str) -> str:
    return "fp64" if kind == "fp64" else "mixed"


def gpu_rate(n_rings: int, cand: Candidate, kind: str = "mixed", slices: int = 200, fill: float = 2.0,
             stream=None) -> float:
    """Ring-slices per second of one batched march over copies of the probe
    wake in this shape, enough copies for about fill x the SM count in
    CTAs; CUDA events around the march, after an untimed one."""
    import torch
    wk = probe_wake(n_rings, slices, kind)
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    copies = max(1, int(round(fill * sms / max(1, cand.ctas))))
    st = stream if stream is not None else torch.cuda.current_stream()
    gs = [wm.Wake.from_workload(wk, precision=_precision(kind), stream=st.cuda_stream, **cand.wake_kwargs())
          for _ in range(copies)]
    try:
        wm.wake_batch_run(gs)
        torch.cuda.synchronize()
        wm.wake_batch_reset(gs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        wm.wake_batch_run(gs)
        e1.record(st)
        torch.cuda.synchronize()
        species = 2 if kind == "ions" else 1
        done = sum(species * n_rings * g.progress()[0] for g in gs)
        return done / (e0.elapsed_time(e1) / 1e3)
    finally:
        for g in gs:
            g.close()


@dataclass
class SizeResult:
    n_rings: int
    kind: str
    rates: List[dict]           # one per candidate: its fields and ring_slices_per_s
    chosen: Candidate

    def to_json(self) -> dict:
        return {"n_rings": self.n_rings, "kind": self.kind, "rates": self.rates, "chosen": asdict(self.chosen)}


def tune_size(n_rings: int, kind: str = "mixed", rate: Optional[Callable[[int, Candidate], float]] = None,
              max_candidates: int = 8, min_gain: float = 0.03, **rate_kw) -> SizeResult:
    """Time every candidate shape of a size class (rate(n, candidate) ->
    ring-slices/s; the GPU by default) and choose the fastest, keeping the
    automatic shape unless another beats it by more than min_gain."""
    cands = candidates(n_rings, kind, max_candidates)
    if rate is None:
        def rate(n, c):
            return gpu_rate(n, c, kind, **rate_kw)
    rates = [float(rate(n_rings, c)) for c in cands]
    best = max(range(len(cands)), key=lambda i: rates[i])
    auto = next(i for i, c in enumerate(cands) if c.automatic)
    chosen = cands[best] if rates[best] > (1.0 + min_gain) * rates[auto] else cands[auto]
    rows = [dict(asdict(c), ring_slices_per_s=r) for c, r in zip(cands, rates)]
    return SizeResult(n_rings, kind, rows, chosen)


@dataclass
class TableEntry:
    kind: str
    n_max: int                  # applies to ring counts in (previous entry's n_max, n_max]
    rings_per_thread: int = 0
    rings_per_cta: int = 0      # 0: the automatic shape
    block_threads: int = 0


@dataclass
class TuningTable:
    entries: List[TableEntry] = field(default_factory=list)
    results: List[dict] = field(default_factory=list)

    def entry_for(self, n_rings: int, kind: str = "mixed") -> Optional[TableEntry]:
        for e in sorted((e for e in self.entries if e.kind == kind), key=lambda e: e.n_max):
            if n_rings <= e.n_max:
                return e
        return None

    def shape_for(self, n_rings: int, kind: str = "mixed") -> Dict[str, int]:
        """Keyword arguments of Wake for a wake of n_rings rings: the size
        class's rings per thread and CTAs of its rings per CTA, if the
        library accepts them for n_rings; {} (the automatic shape)
        otherwise."""
        e = self.entry_for(n_rings, kind)
        if e is None:
            return {}
        if kind != "mixed":
            out = {"block_threads": e.block_threads} if e.block_threads else {}
            if kind in GM_CLUSTER_KINDS and (e.rings_per_cta or e.block_threads):
                # the stored blocks per wake for this size (1 with a block size alone;
                # n_rings counts cells per species with ions)
                out["cluster_ctas"] = max(1, min(8, math.ceil(n_rings / e.rings_per_cta))) if e.rings_per_cta else 1
            return out
        if not e.rings_per_cta:
            return {}
        cl = max(1, math.ceil(n_rings / e.rings_per_cta))
        try:
            wm.wake_launch_shape(n_rings, e.rings_per_thread, cl)
        except wm.WakeError:
            return {}
        return {"rings_per_thread": e.rings_per_thread, "cluster_ctas": cl}

    def to_json(self) -> str:
        return json.dumps({"entries": [asdict(e) for e in self.entries], "results": self.results}, indent=1)

    @classmethod
    def from_json(cls, text: str) -> "TuningTable":
        d = json.loads(text)
        return cls([TableEntry(**e) for e in d.get("entries", [])], d.get("results", []))

    def save(self, path: str):
        with open(path, "w") as f:
            f.write(self.to_json())

    @classmethod
    def load(cls, path: str) -> "TuningTable":
        with open(path) as f:
            return cls.from_json(f.read())


def entry_from(result: SizeResult, n_max: int) -> TableEntry:
    c = result.chosen
    if result.kind != "mixed":
        per_cta = math.ceil(result.n_rings / c.ctas) if c.cluster_ctas > 1 else 0
        return TableEntry(result.kind, n_max, rings_per_cta=per_cta, block_threads=c.block_threads)
    if c.automatic:
        return TableEntry("mixed", n_max)
    return TableEntry("mixed", n_max, c.rings_per_thread, math.ceil(result.n_rings / c.ctas))


def tune(sizes: Sequence[int] = DEFAULT_SIZES, kind: str = "mixed",
         rate: Optional[Callable[[int, Candidate], float]] = None, **kw) -> TuningTable:
    """A table over size classes: each size in `sizes` is timed and its
    choice applies to ring counts from just above the previous size up to
    it (the last one to the march's maximum)."""
    sizes = sorted(s for s in set(sizes) if 1 <= s <= max_rings(kind))
    table = TuningTable()
    for i, n in enumerate(sizes):
        res = tune_size(n, kind, rate, **kw)
        n_max = n if i + 1 < len(sizes) else max_rings(kind)
        table.entries.append(entry_from(res, n_max))
        table.results.append(res.to_json())
    return table


def _class_bounds(sizes: Sequence[int], kind: str = "mixed") -> List[int]:
    """Upper ring counts of the size classes: each size, the last one
    extended to the march's maximum."""
    sizes = sorted(s for s in set(sizes) if 1 <= s <= max_rings(kind))
    return sizes[:-1] + [max_rings(kind)] if sizes else []


def tune_batch(wakes: Sequence, sizes: Sequence[int] = DEFAULT_SIZES, max_candidates: int = 6,
               min_gain: float = 0.02, make: Optional[Callable] = None, run: Optional[Callable] = None,
               repeats: int = 2) -> TuningTable:
    """A table for one batch of wakes (mixed path), chosen on the batch's
    own step time: a synthetic probe misses what makes a workload's slices
    costly (ring crossings, dense beam slices), and a batch is done when its
    longest wake is, so the objective is the time of the whole batched step
    (wake_batch_reset_run over every wake) rather than any one wake's rate.
    Coordinate descent over the size classes, the class of the longest wake
    (rings x slices) first: for each class, every candidate shape of its largest
    member is tried on the class's wakes with the other classes as chosen so
    far, and kept if it shortens the step by more than min_gain.

    make(wake, shape_kwargs) -> handle and run(handles) -> seconds of one
    step are the GPU by default (a Wake per workload wake; CUDA events
    around wake_batch_reset_run); the best of `repeats` runs counts.  The
    wakes must be on-chip-march wakes (electrons over the ion column, AB2,
    no beam grids): the other marches take no rings per thread or CTAs."""
    for wk in wakes:
        if (getattr(wk, "ions", None) is not None or getattr(wk, "integrator", "ab2") != "ab2"
                or getattr(wk, "grid_nr", 0)):
            raise ValueError(f"{wk.name}: not a wake of the on-chip march (ions, RK4 or beam grids)")
    bounds = _class_bounds(sizes)
    table = TuningTable([TableEntry("mixed", b) for b in bounds])
    if make is None or run is None:
        make, run = _gpu_batch_fns()

    def cls(n):
        return next(i for i, b in enumerate(bounds) if n <= b)

    members: Dict[int, List[int]] = {}
    for i, wk in enumerate(wakes):
        members.setdefault(cls(wk.n_rings), []).append(i)
    handles = [make(wk, table.shape_for(wk.n_rings)) for wk in wakes]

    def timed():
        return min(float(run(handles)) for _ in range(max(1, repeats)))

    def rebuild(idx, tab):
        for i in idx:
            old = handles[i]
            handles[i] = make(wakes[i], tab.shape_for(wakes[i].n_rings))
            close = getattr(old, "close", None)
            if close is not None:
                close()

    base = timed()
    # the classes of the longest wakes first: the step ends with its longest wake
    longest = {c: max(wakes[i].n_rings * wakes[i].n_steps for i in idx) for c, idx in members.items()}
    for c in sorted(members, key=lambda c: -longest[c]):
        idx = members[c]
        n_rep = max(wakes[i].n_rings for i in idx)
        tried = [{"shape": "automatic", "step_s": base}]
        best_t, best_entry = base, table.entries[c]
        for cand in candidates(n_rep, "mixed", max_candidates)[1:]:
            entry = entry_from(SizeResult(n_rep, "mixed", [], cand), bounds[c])
            trial = TuningTable(list(table.entries))
            trial.entries[c] = entry
            rebuild(idx, trial)
            t = timed()
            tried.append({"shape": asdict(cand), "step_s": t})
            if t < best_t:
                best_t, best_entry = t, entry
        if best_entry is not table.entries[c] and best_t < (1.0 - min_gain) * base:
            table.entries[c] = best_entry
            base = best_t
        rebuild(idx, table)
        table.results.append({"class_n_max": bounds[c], "wakes": len(idx), "largest": n_rep, "tried": tried,
                              "chosen": asdict(table.entries[c])})
    for h in handles:
        close = getattr(h, "close", None)
        if close is not None:
            close()
    return table


def _gpu_batch_fns(stream=None):
    """make and run of tune_batch on the GPU: mixed-precision Wakes on the
    current stream; one pipelined batched solve (wake_batch_reset_run)
    between CUDA events, after one untimed solve of a new set of handles."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    state = {"warm": None}

    def make(wk, shape):
        return wm.Wake.from_workload(wk, precision="mixed", stream=st.cuda_stream, **shape)

    def run(handles):
        key = tuple(id(h) for h in handles)
        if state["warm"] != key:
            wm.wake_batch_reset_run(list(handles))
            torch.cuda.synchronize()
            state["warm"] = key
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        wm.wake_batch_reset_run(list(handles))
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    return make, run
