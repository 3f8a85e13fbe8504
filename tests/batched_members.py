"""Members of the 256-wake batched workload compared with the oracle one by
one: the stratified sample and the oracle runs (in spawned worker
processes: the parent holds a CUDA context).

The sample: the ring counts (log-uniform in [500, 8000]) split into eight
log-spaced classes; from each class the member with the strongest driver,
the one with the longest window and the two lowest-numbered others; and the
four strongest drivers of the whole batch.  So every launch shape of the
batch (one CTA up to 2048 rings, clusters of 2-8 CTAs above) and the wakes
that break down earliest are in it.
"""
import math

import numpy as np

N_MEMBERS = 256
# whole-window comparison: the first slices of each member, before the
# trajectories of two correct implementations part (they are chaotic
# behind the first bubble: the FP64 GPU path and the oracle differ only in
# summation order and still part by 1e-3 after ~1000 slices)
WINDOW = 300
# slices of the oracle's run kept whole (state with AB2 history, fields):
# fractions of the window, each with the slice after it
SNAP_FRACTIONS = (0.05, 0.15, 0.25, 0.35, 0.45, 0.55, 0.65, 0.75, 0.85, 0.95)


def stratified_sample():
    """Member indices of the sample, ascending."""
    from paper_2603_16623_gb300 import workloads as W
    ps = [W.batched_params(k) for k in range(N_MEMBERS)]
    lo, hi = math.log(500), math.log(8000)
    classes = {}
    for k, p in enumerate(ps):
        c = min(7, int((math.log(p.n_rings) - lo) / (hi - lo) * 8))
        classes.setdefault(c, []).append(k)
    pick = set()
    for c, ks in classes.items():
        pick.add(max(ks, key=lambda k: ps[k].n_b0))
        pick.add(max(ks, key=lambda k: ps[k].n_steps))
        for k in sorted(ks):
            if len([j for j in pick if j in ks]) >= 4:
                break
            pick.add(k)
    pick.update(sorted(range(N_MEMBERS), key=lambda k: -ps[k].n_b0)[:4])
    return sorted(pick)


def snapshot_slices(n_steps):
    """Snapshot slices: each fraction of the window from slice WINDOW on,
    with the slice after it."""
    out = []
    for f in SNAP_FRACTIONS:
        s = max(WINDOW, min(n_steps - 2, WINDOW + int(f * (n_steps - WINDOW))))
        out += [s, s + 1]
    return sorted(set(out))


def one_step_picks(snaps, status, fail_slice, slices_run):
    """Three snapshot slices s >= WINDOW (first, middle, last) whose state
    and the next are both kept and that were solved without a stop."""
    last = fail_slice if status != 0 else slices_run
    cand = [s for s in sorted(snaps) if s + 1 in snaps and s + 1 <= last and s >= WINDOW]
    return sorted({cand[0], cand[len(cand) // 2], cand[-1]}) if cand else []


def oracle_member(k):
    """The oracle on member k: the first WINDOW slices with ring radii and
    the beam fields; the whole window for where it stops, with the state,
    AB2 history and ring fields at three slices spread over its run (and
    the state after each) and the beam fields of those slices' particles."""
    import oracle
    from paper_2603_16623_gb300 import workloads as W
    wk = W.batched_wake(k)
    head = W.Wake(wk.name, wk.edges, wk.beams, wk.dxi, min(WINDOW, wk.n_steps))
    r1 = oracle.run_wake(head, ring_dumps=("r",), beam_fields=("ez", "wr"))
    r2 = oracle.run_wake(wk, beam_fields=("ez", "wr", "bt"), snapshots=snapshot_slices(wk.n_steps))
    picks = one_step_picks(r2.snapshots, r2.status, r2.fail_slice, r2.slices_run)
    xi = np.concatenate([b.xi for b in wk.beams])
    sl = np.floor(xi / wk.dxi + 0.5)
    sel = np.nonzero(np.isin(sl, picks))[0]
    return {"k": k, "head_status": r1.status, "head_r": r1.rings["r"], "head_beam": r1.beam,
            "status": r2.status, "fail_slice": r2.fail_slice, "slices_run": r2.slices_run,
            "picks": picks, "snapshots": {s: r2.snapshots[s] for p in picks for s in (p, p + 1)},
            "beam_idx": sel, "beam": {f: v[sel] for f, v in r2.beam.items()}}


def oracle_members(ks, workers=None):
    """oracle_member over ks in spawned processes, as {k: result}."""
    import concurrent.futures
    import multiprocessing
    import os
    workers = workers or max(1, min(len(ks), os.cpu_count() or 1))
    ctx = multiprocessing.get_context("spawn")
    # largest work first, so the long members do not finish last
    from paper_2603_16623_gb300 import workloads as W
    order = sorted(ks, key=lambda k: -W.batched_params(k).n_rings * W.batched_params(k).n_steps)
    with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        return {r["k"]: r for r in ex.map(oracle_member, order)}


def nerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b)) if b.size else 0.0
    d = np.max(np.abs(a - b)) if b.size else 0.0
    return float(d / den) if den > 0 else float(d)
