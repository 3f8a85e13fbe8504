"""Benchmark of the gridless quasistatic wake hot path on one or more GPUs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one pass of the whole hot path over the batched workload: 256
independent wakes (log-uniform 500-8000 rings, 1000-6000 slices), each
prepared on the device (ring initialisation, nearest-slice binning and radial
sort of its beam) and then marched through its window in one persistent
launch (sort, prefix sums, psi and derivatives, B_theta, fields on the beam
particles, AB2 push).  The metric is ring-slice updates per second: one ring
advanced one slice, summed over the slices each wake actually ran (a wake
stops early if its quasistatic model breaks down, psibar <= 0).

With torchrun (N > 1) every rank solves its own batch of 256 wakes (weak
scaling, no collective on the data path) and rank 0 prints one JSON line.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.

Besides the timed step the line carries: the same step end to end from
pinned host beams (e2e), beam-particle field evaluations per second, the
ALU roofline of the march, the plain FP64 one-wake-per-launch baseline,
serving latencies under a Poisson stream, the beam push, mobile ions and a
density profile, RK4, beam grids, the single-wake workloads, the oracle on
the host cores, and the SM clocks sampled during the timed region.  Each
leg has a --skip-* flag; --autotune batch|probe picks the launch shapes by
a tuning run first.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_16623_gb300 import workloads as W  # noqa: E402

METRIC = "ring-slice updates/s (batched FP32 vs plain FP64, 1 GB300); p50/p99 wake latency"
UNIT = "ring-slices/s"
# algorithmic floating-point operations per ring-slice update of the march:
# the arithmetic of steps a3-a10 as the oracle writes it (each +, -, *, /
# and log counted once): beam field 2, prefix sums 4, psi/d_rho psi/psibar/
# gamma/t 21, d_zeta psi 6, A/B/C 27, B_theta^(p) recursion and value 44,
# AB2 push 13
FLOPS_PER_RING_SLICE = 117
# the same count for the two-species march with mobile ions (orc_run_ions):
# per ring of either species beam field 2, prefix sums 4, own psi/d_rho psi
# 5, their gather from the other species and the totals 11, psibar/gamma/t
# 11, d_zeta psi (prefix, own, gather, total) 13, AB2 push 13; per electron
# ring A/B/C 27 and B^(p) 44; per ion ring the B^(p) gather 6
FLOPS_PER_RING_SLICE_IONS = (130 + 65) / 2
# and for the RK4 integrator (orc_run with integrator rk4): four field
# evaluations of a3-a8 and B^(p) at the rings (104 each, +2 for the second
# source at the two half steps), the derivatives (5 per stage), three stage
# states (4 each), the weighted sums (4 per later stage) and the update (4)
FLOPS_PER_RING_SLICE_RK4 = 4 * 104 + 2 * 2 + 4 * 5 + 3 * 4 + 3 * 4 + 4
# FP32 ALU peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x clock
SMS, FP32_LANES = 152, 128


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def _clock_summary(path, gpu_index):
    try:
        rows = [l.strip().split(",") for l in open(path) if l.strip()]
    except Exception:
        return None
    rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(gpu_index)]
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    reasons = set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        for name, v in zip(names, r[5:9]):
            if v.lower() in ("active", "1"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(rows)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _workload(n_wakes, rank):
    """Rank r's share: its own n_wakes wakes (weak scaling, no overlap)."""
    return [W.batched_wake(k + 256 * rank) for k in range(n_wakes)]


def _reduce_max_sum(tot_ms, ring_slices, device):
    """Across ranks: the largest timed milliseconds and the total ring-slices."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([tot_ms, float(ring_slices)], device=device, dtype=torch.float64)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm_ = t.clone()
    dist.all_reduce(sm_, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm_[1])


def _shape(n_rings, args):
    """Launch shape of a wake: the library's automatic one, or with
    --rings-per-cta R, clusters of ceil(n / R) CTAs of 4 rings per thread."""
    if not args.rings_per_cta or n_rings <= 2048:
        return {}
    cl = -(-n_rings // args.rings_per_cta)
    return {"rings_per_thread": 4, "cluster_ctas": cl} if cl <= 16 else {}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2603_16623_gb300 import wake as wm

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    stream = torch.cuda.current_stream()
    wakes = _workload(args.n_wakes, rank)
    tuning = None
    if args.autotune:
        # launch shapes timed on this GPU: on this batch's own step time
        # (batch), or per size class on synthetic probe wakes (probe)
        from paper_2603_16623_gb300 import autotune
        t_tune = time.perf_counter()
        sizes = [int(v) for v in args.autotune_sizes.split(",")]
        if args.autotune == "batch":
            table = autotune.tune_batch(wakes, sizes)
        else:
            table = autotune.tune(sizes, "mixed", slices=200, fill=args.autotune_fill)
        tuning = {"mode": args.autotune, "entries": [dataclasses.asdict(e) for e in table.entries],
                  "tuning_s": time.perf_counter() - t_tune}
        if args.autotune == "probe":
            tuning["fill"] = args.autotune_fill
        shape = lambda n: table.shape_for(n)  # noqa: E731
    else:
        shape = lambda n: _shape(n, args)  # noqa: E731
    gs = [wm.Wake.from_workload(wk, precision="mixed", stream=stream.cuda_stream, **shape(wk.n_rings))
          for wk in wakes]
    torch.cuda.synchronize()
    # one march launch per distinct (threads, rings per thread, blocks per wake)
    n_march_launches = len({g.launch_config() for g in gs})

    def step(ev=None):
        # a0/a1 preparation and the march of every wake, pipelined: each
        # launch shape's march starts once its own wakes are prepared
        if ev is not None:
            ev[0].record(stream)
        wm.wake_batch_reset_run(gs)
        if ev is not None:
            ev[1].record(stream)

    def phase_step(ev):
        # the two phases one after the other (for their times)
        ev[0].record(stream)
        wm.wake_batch_reset(gs)
        ev[1].record(stream)
        wm.wake_batch_run(gs)
        ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # work actually done per step (wakes may stop at a model breakdown)
    ring_slices = 0
    stopped = 0
    nexts = []
    for g, wk in zip(gs, wakes):
        nxt, st, fl = g.progress()
        ring_slices += wk.n_rings * nxt
        stopped += int(st != 0)
        nexts.append(nxt)
    evals = beam_evaluations(wakes, nexts)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    clk_path = os.path.join(tempfile.gettempdir(), f"bench_clocks_{os.getpid()}.csv")
    proc, fh = _clock_sampler(clk_path) if rank == 0 else (None, None)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(evs[k])
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall = time.perf_counter() - t0
    if proc is not None:
        proc.terminate()
        proc.wait()
        fh.close()
    step_ms = [e[0].elapsed_time(e[1]) for e in evs]
    # the last timed step's schedule: each wake's march from its own device
    # times (when its launch began on it, when it finished)
    wt = [g.march_times() for g in gs]
    t_first = min(t[0] for t in wt)
    # the throughput bound: each wake's SM share (its CTAs' share of an SM's
    # registers at 128 per thread, or of its 2048 thread slots) x its march
    # time in the batch, summed and spread over the SMs
    sms = torch.cuda.get_device_properties(0).multi_processor_count

    def sm_share(g):
        threads, _, ctas = g.launch_config()
        per_sm = max(1, min(65536 // (128 * threads), 2048 // threads))
        return ctas / per_sm

    schedule = {"longest_wake_ms": max(t[1] - t[0] for t in wt) / 1e6,
                "march_span_ms": (max(t[1] for t in wt) - t_first) / 1e6,
                "sm_time_bound_ms": sum(sm_share(g) * (t[1] - t[0]) for g, t in zip(gs, wt)) / 1e6 / sms,
                "latest_start_of_the_10_longest_ms": sorted(
                    ((t[1] - t[0], t[0] - t_first) for t in wt), reverse=True)[9][1] / 1e6 if len(wt) >= 10 else None,
                "note": "device times (globaltimer) of the last timed step; the longest wake is the critical path, "
                        "sm_time_bound the throughput bound (SM shares by registers x in-batch march times / SMs)"}
    try:  # the critical-path wake's shape and slices (for the latency roofline)
        i_long = max(range(len(wt)), key=lambda i: wt[i][1] - wt[i][0])
        t_c, k_c, c_c = gs[i_long].launch_config()
        schedule["critical_wake"] = {"rings": wakes[i_long].n_rings, "slices": nexts[i_long], "threads": t_c,
                                     "rings_per_thread": k_c, "ctas": c_c}
    except Exception as e:  # reported, never fatal to the bench
        schedule["critical_wake"] = {"unavailable": repr(e)}
    pev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    phase_step(pev)
    torch.cuda.synchronize()
    march_ms = [pev[1].elapsed_time(pev[2])]
    prep_ms = [pev[0].elapsed_time(pev[1])]
    tot_ms = sum(step_ms)
    if ws > 1:
        tot_ms_max, rs_all = _reduce_max_sum(tot_ms, ring_slices, "cuda")
    else:
        tot_ms_max = tot_ms
        rs_all = float(ring_slices)
    value = rs_all * args.steps / (tot_ms_max / 1e3)
    if ws > 1:
        _, evals_all = _reduce_max_sum(tot_ms, evals, "cuda")
    else:
        evals_all = float(evals)

    # pinned host copies of the beams (end-to-end and serving runs)
    pinned = []
    h2d = 0
    if not (args.skip_e2e and args.skip_serve):
        for wk in wakes:
            pinned.append(_pinned_beams(wk))
            h2d += sum(3 * 8 * b.n for b in wk.beams)

    # ---- end to end through the C ABI with host buffers (pinned), rank-local
    e2e = None
    if not args.skip_e2e:
        outs = [{k: torch.empty(g.n_beam, dtype=torch.float32).pin_memory() for k in ("ez", "wr")} for g in gs]
        d2h = sum(g.n_beam for g in gs) * 2 * 4
        def e2e_step():
            # pinned host beams up, preparation and march pipelined, E_z and
            # W_r of every beam particle back to pinned host buffers
            wm.wake_batch_solve(gs, pinned)
            wm.wake_batch_get_beam_fields(gs, [o["ez"] for o in outs], [o["wr"] for o in outs])

        e2e_step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t1 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 3))
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t1) / n_e2e
        if ws > 1:
            t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t[0])
        e2e = {"value": rs_all / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e2e_s * 1e3}

    # ---- every batched member against the oracle (host cores), rank 0; the
    # handles still hold the march of the workload's own beams (the push leg
    # below moves them)
    parity = None
    if not args.skip_parity_sample and rank == 0 and ws == 1:
        parity = parity_sample_bench(gs, wakes, _host_cores(), stream)

    # ---- beam push (the step after a solve): Boris step of every beam particle
    push = None
    if not args.skip_push:
        push = push_bench(args, gs, wakes, stream)

    # ---- the beam stage: the batched march with each slice's beam staged in
    # shared memory by bulk copies (the default) against plain global loads
    stage_ab = None
    if not args.skip_stage_ab:
        stage_ab = stage_ab_bench(gs, wakes, stream)

    # ---- mobile ions: the two-species march on batched wakes
    ions = None
    if not args.skip_ions:
        ions = ions_bench(args, wakes, stream)

    # ---- the RK4 ring integrator on batched wakes
    rk4 = None
    if not args.skip_rk4:
        rk4 = rk4_bench(args, wakes, stream)

    # ---- adaptive beam grids against the gridless coupling (FP64)
    grid = None
    if not args.skip_grid:
        grid = grid_bench(args, wakes, stream)

    # ---- serving: Poisson arrivals of batched-workload wakes, continuous batching
    serving = None
    if not args.skip_serve:
        serving = serve_bench(args, wakes, pinned, stream, rank, ws)

    # ---- plain FP64 one-wake-per-launch on a bounded sample (the plain GPU baseline)
    plain = None
    if not args.skip_plain and rank == 0:
        sample = wakes[: args.plain_wakes]
        hs = [wm.Wake.from_workload(wk, precision="fp64", stream=stream.cuda_stream) for wk in sample]
        for h in hs:
            h.step_slices(20)
        torch.cuda.synchronize()
        for h in hs:
            h.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for h in hs:
            h.step_slices(args.plain_slices)
        e1.record(stream)
        torch.cuda.synchronize()
        done = sum(wk.n_rings * h.progress()[0] for wk, h in zip(sample, hs))
        plain_v = done / (e0.elapsed_time(e1) / 1e3)
        plain = {"value": plain_v, "unit": UNIT,
                 "sample": f"first {args.plain_slices} slices of wakes 0-{len(sample) - 1}, one wake per launch",
                 "ratio_batched_mixed_over_plain_fp64": value / ws / plain_v}
        for h in hs:
            h.close()

    # ---- the single-wake workloads (linear, blowout, large) alone on the GPU
    singles = None
    if not args.skip_singles and rank == 0:
        singles = single_wakes_bench(args, stream)

    # ---- CPU baseline: the oracle on a bounded sample, rank 0 only
    cpu = None
    if not args.skip_cpu and rank == 0 and ws == 1:
        cpu = cpu_sample(args.cpu_seconds)
        # and single-threaded on the single-wake workloads
        cpu["single_wakes"] = oracle_single_wakes(args.large_oracle_slices)
        # and on every host core (independent wakes in spawned processes)
        pool = OraclePool(_host_cores())
        cpu["all_cores"] = pool.sample(args.cpu_seconds / 2)
        pool.close()

    peaks = _peaks()
    clocks = _clock_summary(clk_path, local) if rank == 0 else None
    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    # the on-chip peaks measured on this GPU by the library's microbenchmarks
    onchip = wm.measure_peaks()
    peak_tflops = onchip["fp32_tflops"]
    march_avg_ms = sum(march_ms) / len(march_ms)
    achieved = FLOPS_PER_RING_SLICE * ring_slices / (march_avg_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": None,
                "kernel": "march_fast_kernel<4> + march_cluster_kernel<4> (batched march)",
                "peak_basis": "measured: FP32 FMA throughput microbenchmark (wake_measure_peaks), "
                              f"{onchip['sm_clock_mhz']:.0f} MHz",
                "nominal_fp32_tflops": SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12,
                "onchip_peaks": onchip, "schedule": schedule,
                "latency_roofline": latency_roofline(schedule, onchip)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff (mixed)", "data": "synthetic",
            "config": {"workload": f"batched: {args.n_wakes} independent wakes per GPU, log-uniform 500-8000 "
                                   "rings, 1000-6000 slices of 0.01, 50k-500k beam particles",
                       "n_wakes": args.n_wakes, "precision": "mixed",
                       "launches": sorted({g.launch_config() for g in gs}),
                       "launch_shapes": "autotuned" if tuning else "automatic",
                       "autotune": tuning,
                       "ring_slices_per_step": ring_slices, "wakes_stopped_by_breakdown": stopped,
                       "l2": "inputs larger than L2 (device-resident beams ~1.7 GB per batch)"},
            "serving": serving, "parity_sample": parity,
            "beam_evaluations": {"value": evals_all * args.steps / (tot_ms_max / 1e3),
                                 "unit": "beam-particle field evaluations/s", "per_step": evals_all,
                                 "note": "step a9: each beam particle binned into a slice its wake marched"},
            "e2e": e2e, "gpu_launches": args.steps * (len(gs) * 7 + n_march_launches),
            "roofline": roofline, "cpu_baseline": cpu, "plain_fp64": plain,
            "beam_push": push, "beam_stage": stage_ab,
            "mobile_ions": _ions_roofline(ions, peak_tflops, sm_mhz),
            "rk4": _alu_roofline(rk4, peak_tflops, sm_mhz, FLOPS_PER_RING_SLICE_RK4, "march_rk4_kernel<PrecMixed>", 1),
            "beam_grid": grid,
            "single_wakes": singles,
            "clocks": clocks,
            "phases_ms": {"prepare_a0_a1": sum(prep_ms) / len(prep_ms), "march": march_avg_ms,
                          "note": "one untimed step with the two phases in sequence; the timed steps pipeline them"},
            "wall_s": wall,
        }
        print(json.dumps(line))
    for g in gs:
        g.close()
    if ws > 1:
        dist.destroy_process_group()


# algorithmic HBM bytes per beam particle of one push (one fused kernel):
# read x, y, xi, u_x, u_y, u_z (48), its sorted position (4) and E_z, W_r,
# B_theta there (12); write x, y, xi, r, u_x, u_y, u_z (56)
PUSH_BYTES_PER_PARTICLE = 48 + 4 + 12 + 56


def push_bench(args, gs, wakes, stream):
    """wake_batch_push_beam over the whole batch after a solve, timed with
    CUDA events; HBM-bound (one pass over the particle arrays)."""
    import torch
    from paper_2603_16623_gb300 import wake as wm
    n_part = 0
    for g, wk in zip(gs, wakes):
        b = np.concatenate([bm.r for bm in wk.beams])
        n = b.shape[0]
        g.set_beam_phase_space(b, np.zeros(n), np.zeros(n), np.zeros(n), np.full(n, 2000.0))
        n_part += n
    wm.wake_batch_push_beam(gs, 0.1)  # warm-up
    torch.cuda.synchronize()
    reps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        wm.wake_batch_push_beam(gs, 0.1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    peak = _peaks().get("hbm_gbs", 6800.0)
    gbs = PUSH_BYTES_PER_PARTICLE * n_part / (ms / 1e3) / 1e9
    # one coupled stage step (Sec. V): bin the pushed beams again (the
    # densest slice read back from the device), solve every wake, push
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    wm.wake_batch_reset(gs)
    wm.wake_batch_run(gs)
    wm.wake_batch_push_beam(gs, 0.1)
    s1.record(stream)
    torch.cuda.synchronize()
    stage_ms = s0.elapsed_time(s1)
    stage_rs = sum(wk.n_rings * g.progress()[0] for g, wk in zip(gs, wakes))
    return {"particles": n_part, "ms_per_push": ms, "particles_per_s": n_part / (ms / 1e3),
            "stage_step": {"ms": stage_ms, "ring_slices_per_s": stage_rs / (stage_ms / 1e3),
                           "steps": "batched reset of the pushed beams + march + push"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "bytes_per_particle": PUSH_BYTES_PER_PARTICLE, "peak_basis": "measured copy (MEASURED_PEAKS.json)"}}


def stage_ab_bench(gs, wakes, stream, reps=3):
    """The batched march (after a batched preparation, CUDA-event timed) of
    the same wakes with the beam staged by bulk copies and with plain
    global loads (WAKE_NO_STAGE handles), alternated; best of reps each."""
    import torch
    from paper_2603_16623_gb300 import wake as wm
    plain = [wm.Wake.from_workload(wk, precision="mixed", stream=stream.cuda_stream, flags=wm.WAKE_NO_STAGE)
             for wk in wakes]
    out = {"staged_ms": [], "global_ms": []}
    for _ in range(reps):
        for key, hs in (("staged_ms", gs), ("global_ms", plain)):
            wm.wake_batch_reset(hs)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            wm.wake_batch_run(hs)
            e1.record(stream)
            torch.cuda.synchronize()
            out[key].append(e0.elapsed_time(e1))
    longest = {}
    for key, hs in (("staged", gs), ("global", plain)):
        wt = [h.march_times() for h in hs]
        longest[key] = max(t[1] - t[0] for t in wt) / 1e6
    for h in plain:
        h.close()
    out["staged_over_global"] = min(out["staged_ms"]) / min(out["global_ms"])
    out["longest_wake_ms"] = longest
    return out


def ions_bench(args, wakes, stream):
    """A batch of the workload's wakes of <= 4096 rings with mobile hydrogen
    ions (Z = 1, M = 1836) in place of the ion column: batched reset + march,
    CUDA-event timed; ring-slices count both species.  The same wakes with
    the immobile ion column (the on-chip AB2 march) give the per-ring-slice
    comparison."""
    base = [wk for wk in wakes if wk.n_rings <= 4096][: args.ion_wakes]
    sel = [dataclasses.replace(wk, ions=(1.0, 1836.0)) for wk in base]
    res = _ions_batch(sel, stream)
    res["ions"] = "Z = 1, M = 1836 (hydrogen), same cells as the electrons"
    ref = _ions_batch(base, stream, species=1)
    res["electron_only_same_wakes"] = {k: ref[k] for k in ("ring_slices", "ms_per_step", "value", "unit")}
    res["electron_only_over_ions_per_ring_slice"] = ref["value"] / res["value"]
    # a radial profile changes only the ring weights: the parabolic channel
    # n = 1 + 4 r^2 / w0^4 (w0 = 3) with static ion rings
    prof = [dataclasses.replace(wk, ions=(1.0, float("inf")), cell_density=W.parabolic_profile(wk.edges, 1.0, 3.0))
            for wk in sel]
    res["parabolic_static_ions"] = _ions_batch(prof, stream)
    return res


def rk4_bench(args, wakes, stream):
    """The batched workload's wakes of <= 8192 rings with the RK4 ring
    integrator (blocks of 512 threads, a cluster of up to 8 for the wide
    wakes): batched reset + march, CUDA-event timed.  The same wakes with
    AB2 (the on-chip march) give the per-ring-slice comparison."""
    base = [wk for wk in wakes if wk.n_rings <= 8192][: args.rk4_wakes]
    sel = [dataclasses.replace(wk, integrator="rk4") for wk in base]
    res = _ions_batch(sel, stream, species=1)
    res["integrator"] = "classical RK4 per slice (four field evaluations), electrons over the ion column"
    ref = _ions_batch(base, stream, species=1)
    res["ab2_same_wakes"] = {k: ref[k] for k in ("ring_slices", "ms_per_step", "value", "unit")}
    res["ab2_over_rk4_per_ring_slice"] = ref["value"] / res["value"]
    return res


# warp instructions per ring-slice of the on-chip marches, from the ncu
# captures summarised in profiles/ (one CTA: 2048 rings, 512 threads x 4;
# cluster: 6000 rings, 6 CTAs of 256 x 4), and their barriers per slice
WARP_INSTR_PER_RING_SLICE = {"one_cta": 39.7, "cluster": 48.2}
BLOCK_BARRIERS_PER_SLICE = {"one_cta": 11, "cluster": 8}
CLUSTER_BARRIERS_PER_SLICE = 6


def latency_roofline(schedule, onchip):
    """A lower bound of the critical-path wake's march time, whose slices run
    in sequence: per slice its CTA's instructions at the issue rate its
    warps can sustain on dependent float-float chains (a scheduler with w
    warps issues at most min(1, w / FMA latency) per cycle, 4 schedulers per
    SM, the CTA alone on its SM) plus the latency of its barriers, from the
    measured on-chip peaks.  frac = bound / the wake's measured time."""
    try:
        cw = schedule["critical_wake"]
        kind = "cluster" if cw["ctas"] > 1 else "one_cta"
        warps_per_scheduler = cw["threads"] / 32 / 4
        ipc = 4 * min(1.0, warps_per_scheduler / onchip["fma_latency_cycles"])
        instr = WARP_INSTR_PER_RING_SLICE[kind] * cw["threads"] * cw["rings_per_thread"]
        issue_us = instr / ipc / onchip["sm_clock_mhz"]
        barrier_us = BLOCK_BARRIERS_PER_SLICE[kind] * onchip["syncthreads_ns"] / 1e3
        if kind == "cluster":
            barrier_us += CLUSTER_BARRIERS_PER_SLICE * onchip["cluster_barrier_ns"] / 1e3
        bound_ms = cw["slices"] * (issue_us + barrier_us) / 1e3
        return {"bound_ms": bound_ms, "measured_ms": schedule["longest_wake_ms"],
                "frac": bound_ms / schedule["longest_wake_ms"], "kind": kind,
                "per_slice_us": {"issue": issue_us, "barriers": barrier_us},
                "basis": "warp instructions per ring-slice from the ncu captures in profiles/; FMA latency, "
                         "barrier latencies and SM clock measured by wake_measure_peaks"}
    except Exception as e:  # reported, never fatal to the bench
        return {"unavailable": repr(e)}


def grid_bench(args, wakes, stream):
    """The paper's grid coupling (adaptive beam grids of 32 radial cells per
    beam) against the gridless one on the same batched wakes of <= 8192
    rings over a bounded window (their first args.grid_slices slices):
    FP64 on the global-memory march, both on one block per wake (the grid's
    own cost), and the grids on their automatic clusters; mixed, the grids
    on their automatic clusters against the gridless on-chip march; batched
    reset + step, CUDA-event timed."""
    import torch
    from paper_2603_16623_gb300 import wake as wm
    sel = [wk for wk in wakes if wk.n_rings <= 8192][: args.grid_wakes]
    out = {"wakes": len(sel), "slices": args.grid_slices, "grid_nr": 32,
           "note": "fp64: gridless and grid on one block per wake, grid_clusters on the automatic clusters; "
                   "mixed: grids on the automatic clusters, gridless on the on-chip march"}
    # (name, grid cells, precision, blocks per wake: 1, or 0 = automatic)
    for name, nr, prec, cl in (("gridless", 0, "fp64", 0), ("grid", 32, "fp64", 1), ("grid_clusters", 32, "fp64", 0),
                               ("mixed_gridless", 0, "mixed", 0), ("mixed_grid", 32, "mixed", 0)):
        shape = {"cluster_ctas": cl} if nr else {}
        gs = [wm.Wake.from_workload(dataclasses.replace(wk, grid_nr=nr), precision=prec, stream=stream.cuda_stream,
                                    **shape) for wk in sel]
        wm.wake_batch_reset(gs)
        wm.wake_batch_step(gs, args.grid_slices)  # warm-up
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        wm.wake_batch_reset(gs)
        wm.wake_batch_step(gs, args.grid_slices)
        ev[1].record(stream)
        torch.cuda.synchronize()
        rs = sum(wk.n_rings * g.progress()[0] for g, wk in zip(gs, sel))
        ms = ev[0].elapsed_time(ev[1])
        blocks = [g.launch_config()[2] for g in gs]
        out[name] = {"ring_slices": rs, "ms_per_step": ms, "value": rs / (ms / 1e3), "unit": UNIT,
                     "blocks_per_wake": [min(blocks), max(blocks)]}
        for g in gs:
            g.close()
    out["grid_over_gridless_time"] = out["grid"]["ms_per_step"] / out["gridless"]["ms_per_step"]
    out["mixed_grid_over_gridless_time"] = out["mixed_grid"]["ms_per_step"] / out["mixed_gridless"]["ms_per_step"]
    return out


def _alu_roofline(res, peak_tflops, sm_mhz, flops, kernel, species):
    if res is None:
        return None
    achieved = flops * res["ring_slices"] / (res["march_ms"] / 1e3) / 1e12
    res["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                       "frac": achieved / peak_tflops, "traffic": None, "kernel": kernel, "flops_per_ring_slice": flops,
                       "peak_basis": "measured: FP32 FMA throughput microbenchmark (wake_measure_peaks)"}
    return res


def _ions_batch(sel, stream, species=2):
    import torch
    from paper_2603_16623_gb300 import wake as wm
    gs = [wm.Wake.from_workload(wk, precision="mixed", stream=stream.cuda_stream) for wk in sel]
    wm.wake_batch_reset(gs)
    wm.wake_batch_run(gs)  # warm-up
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    wm.wake_batch_reset(gs)
    ev[1].record(stream)
    wm.wake_batch_run(gs)
    ev[2].record(stream)
    torch.cuda.synchronize()
    ring_slices, stopped, blocks = 0, 0, []
    for g, wk in zip(gs, sel):
        nxt, st, _ = g.progress()
        ring_slices += species * wk.n_rings * nxt
        stopped += int(st != 0)
        blocks.append(g.launch_config()[2])
        g.close()
    march_ms = ev[1].elapsed_time(ev[2])
    step_ms = ev[0].elapsed_time(ev[2])
    return {"wakes": len(sel), "cells": [min(wk.n_rings for wk in sel), max(wk.n_rings for wk in sel)],
            "ring_slices": ring_slices, "wakes_stopped_by_breakdown": stopped,
            "blocks_per_wake": [min(blocks), max(blocks)], "blocks": sum(blocks),
            "ms_per_step": step_ms, "march_ms": march_ms, "value": ring_slices / (step_ms / 1e3), "unit": UNIT}


def _ions_roofline(ions, peak_tflops, sm_mhz):
    if ions is None:
        return None
    achieved = FLOPS_PER_RING_SLICE_IONS * ions["ring_slices"] / (ions["march_ms"] / 1e3) / 1e12
    ions["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                        "frac": achieved / peak_tflops, "traffic": None, "kernel": "march_ions_kernel<PrecMixed>",
                        "flops_per_ring_slice": FLOPS_PER_RING_SLICE_IONS,
                        "peak_basis": "measured: FP32 FMA throughput microbenchmark (wake_measure_peaks)"}
    return ions


def _pinned_beams(wk):
    """The wake's beams as pinned float64 host tensors (for asynchronous
    uploads inside the timed regions)."""
    import torch
    out = []
    for b in wk.beams:
        t = [torch.from_numpy(a).pin_memory() for a in (b.xi, b.r, b.w)]
        out.append(type("B", (), {"xi": t[0], "r": t[1], "w": t[2], "q": b.q}))
    return out


def serve_bench(args, wakes, pinned, stream, rank, ws=1):
    """Continuous batching under a Poisson stream: requests drawn (seeded)
    from the batched workload's first len(wakes) members arrive at
    args.serve_rate per second per GPU; the server admits them under a
    device-memory budget and steps the running batch; latency = result on
    the host minus arrival.  With N GPUs one stream of N times the requests
    at N times the rate is dispatched over the ranks (serve.dispatch: the
    rank with the least work assigned so far), each rank serves its share on
    its own GPU, and the latencies of all ranks are gathered afterwards
    (serve.gather_summary)."""
    import torch
    from paper_2603_16623_gb300 import serve
    n_pool = len(wakes)
    rng = np.random.Generator(np.random.PCG64(4))
    n_req = args.serve_requests * ws
    pick = rng.integers(0, n_pool, n_req)
    arrivals = serve.poisson_arrivals(n_req, args.serve_rate * ws, 4)
    params = [W.batched_params(k) for k in range(n_pool)]
    work = [params[int(k)].n_rings * params[int(k)].n_steps for k in pick]
    owner = serve.dispatch(work, ws)
    mine = np.nonzero(owner == rank)[0]
    # this rank's requests: rank 0's own wakes are the pool members; other
    # ranks draw the members they were given
    pool = {}
    for k in sorted({int(pick[i]) for i in mine}):
        if rank == 0:
            pool[k] = (wakes[k], pinned[k])
        else:
            wk = W.batched_wake(k)
            pool[k] = (wk, _pinned_beams(wk))
    # one pinned result buffer per distinct wake: requests for the same wake
    # compute the same fields, so they may share it
    outs = {k: (torch.empty(wk.n_beam, dtype=torch.float32).pin_memory(),
                torch.empty(wk.n_beam, dtype=torch.float32).pin_memory()) for k, (wk, _) in pool.items()}
    reqs = []
    for i in mine:
        k = int(pick[i])
        wk, pb = pool[k]
        reqs.append(serve.Request(rid=int(i), arrival=float(arrivals[i]), edges=wk.edges, beams=pb, dxi=wk.dxi,
                                  n_steps=wk.n_steps, out_ez=outs[k][0], out_wr=outs[k][1]))
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sm_budget = args.serve_sm_fill * sms if args.serve_sm_fill > 0 else None
    srv = serve.WakeServer(int(args.serve_budget_gb * (1 << 30)), step_ns=int(args.serve_step_us * 1e3),
                           stream=stream.cuda_stream, clock=lambda: time.perf_counter() - t0, sm_budget=sm_budget)
    stats = serve.run_stream(srv, reqs)
    torch.cuda.synchronize()
    out = serve.gather_summary(stats)
    out.update({"arrival_rate_per_s": args.serve_rate * ws, "memory_budget_gb": args.serve_budget_gb,
                "sm_budget": sm_budget,
                "step_us": args.serve_step_us,
                "requests_from": f"{n_pool} batched-workload wakes, drawn with seed 4"
                                 + (f", dispatched over {ws} GPUs by least assigned work" if ws > 1 else ""),
                "offered_ring_slices_per_s": float(sum(work) / arrivals[-1])})
    return out


def beam_evaluations(wakes, nexts):
    """Beam particles whose fields one solve evaluates (step a9): those
    binned into a slice their wake marched, 0 <= floor(xi / dxi + 1/2) <
    the wake's next slice."""
    n = 0
    for wk, nxt in zip(wakes, nexts):
        for b in wk.beams:
            s = np.floor(np.asarray(b.xi) / wk.dxi + 0.5)
            n += int(np.count_nonzero((s >= 0) & (s < nxt)))
    return n


def _single_workloads(large_slices=None):
    """The three single-wake workloads: linear (200 rings, 1000 slices),
    blowout (2000 refined rings, 250k particles, 4000 slices) and large
    (65,536 log-spaced rings, 4M particles, 8000 slices, or its first
    large_slices)."""
    lg = W.large_wake() if large_slices is None else W.large_wake(n_steps=large_slices)
    return [W.linear_wake(), W.blowout_wake(), lg]


def single_wakes_bench(args, stream):
    """Each single-wake workload alone on the GPU, one wake per launch: the
    mixed path over the whole window, and the plain FP64 path (at most 8192
    rings: the large wake has no FP64 line), CUDA-event timed after one
    untimed solve."""
    import torch
    from paper_2603_16623_gb300 import wake as wm
    out = {}
    for wk in _single_workloads():
        row = {"rings": wk.n_rings, "slices": wk.n_steps, "beam_particles": wk.n_beam}
        for prec in ("mixed", "fp64"):
            if wk.n_rings > wm.wake_max_rings(prec):
                row[prec] = None
                continue
            g = wm.Wake.from_workload(wk, precision=prec, stream=stream.cuda_stream)
            g.step_slices(wk.n_steps)  # warm-up solve
            torch.cuda.synchronize()
            g.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.step_slices(wk.n_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            nxt, st, _ = g.progress()
            row[prec] = {"ms": ms, "slices_run": nxt, "status": st, "launch": list(g.launch_config()),
                         "value": wk.n_rings * nxt / (ms / 1e3), "unit": UNIT}
            g.close()
        out[wk.name] = row
    return out


def oracle_single_wakes(large_slices: int):
    """The FP64 oracle, as it stands, on one host core on each single-wake
    workload: the whole window of the linear and blowout wakes, the first
    large_slices slices of the large one (its beam binning included)."""
    import oracle
    out = {}
    for wk in _single_workloads(large_slices):
        t0 = time.perf_counter()
        res = oracle.run_wake(wk, beam_fields=())
        dt = time.perf_counter() - t0
        out[wk.name] = {"rings": wk.n_rings, "slices_run": res.slices_run, "s": dt, "cores": 1,
                        "value": wk.n_rings * res.slices_run / dt, "unit": UNIT}
    return out


def cpu_sample(seconds: float):
    """The FP64 oracle, as it stands, on the first slices of the batched
    wakes until about `seconds` of single-core CPU time."""
    import oracle
    done = 0
    t0 = time.perf_counter()
    used = []
    k = 0
    slices = 400
    while time.perf_counter() - t0 < seconds and k < 256:
        wk = W.batched_wake(k)
        res = oracle.run_wake(wk, max_slices=slices, beam_fields=())
        done += wk.n_rings * res.slices_run
        used.append(k)
        k += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {slices} slices of batched wakes 0-{used[-1]} ({done} ring-slices, {dt:.1f} s)"}


def _oracle_member_parity(k):
    """The oracle on batched member k (runs in a spawned process): its
    status and stopping slice over the whole window, the laminar part of its
    first 300 slices (before any two rings cross), and for the beam
    particles of that part E_z, W_r and the number of rings strictly below
    each (where the particle sits among the rings)."""
    import oracle
    wk = W.batched_wake(k)
    full = oracle.run_wake(wk, beam_fields=())
    head = W.Wake(wk.name, wk.edges, wk.beams, wk.dxi, min(300, wk.n_steps))
    r = oracle.run_wake(head, ring_dumps=("r",), beam_fields=("ez", "wr"))
    rr = r.rings["r"]
    crossed = np.nonzero(np.any(np.diff(rr, axis=1) <= 0.0, axis=1))[0]
    lam = int(crossed[0]) if crossed.size else rr.shape[0]
    if r.status:
        lam = min(lam, r.fail_slice + 1)
    xi = np.concatenate([b.xi for b in wk.beams])
    rb = np.concatenate([b.r for b in wk.beams])
    sl = np.floor(xi / wk.dxi + 0.5).astype(np.int64)
    sel = np.nonzero((sl >= 0) & (sl < lam))[0]
    below = np.empty(sel.shape[0], dtype=np.int32)
    order = np.argsort(sl[sel], kind="stable")
    srt = sel[order]
    bounds = np.searchsorted(sl[srt], np.arange(lam + 1))
    for s_ in range(lam):
        a, b = bounds[s_], bounds[s_ + 1]
        if a < b:
            below[order[a:b]] = np.searchsorted(np.sort(rr[s_]), rb[srt[a:b]], side="left")
    return {"k": k, "status": full.status, "fail": full.fail_slice, "laminar": lam, "idx": sel,
            "ez": r.beam["ez"][sel], "wr": r.beam["wr"][sel], "below": below}


def parity_sample_bench(gs, wakes, cores, stream):
    """Every member of the batch against the oracle (all host cores): the
    stop (status, slice) of the last march of the handles, and E_z, W_r on
    the beam particles of each member's laminar head slices (the first 300
    slices before any two rings cross), norm-wise per member.  A particle
    is compared where the GPU (in FP32) and the oracle (in FP64) place it
    among the same number of rings; the few within rounding of a ring, which
    either side may place on the other side (where d_zeta psi and B^(p) jump
    by that ring's share), are counted apart."""
    import concurrent.futures
    import multiprocessing
    import torch
    from paper_2603_16623_gb300 import wake as wm
    t0 = time.perf_counter()
    ks = list(range(len(wakes)))
    ex = concurrent.futures.ProcessPoolExecutor(max_workers=cores, mp_context=multiprocessing.get_context("spawn"))
    futs = [ex.submit(_oracle_member_parity, k) for k in sorted(ks, key=lambda k: -wakes[k].n_rings * wakes[k].n_steps)]
    stops = [g.progress() for g in gs]
    # the head window again, with the ring radii kept
    heads = [wm.Wake.from_workload(W.Wake(wk.name, wk.edges, wk.beams, wk.dxi, min(300, wk.n_steps)),
                                   precision="mixed", flags=wm.WAKE_DUMP_RING_R, stream=stream.cuda_stream)
             for wk in wakes]
    wm.wake_batch_run(heads)
    torch.cuda.synchronize()
    ref = {}
    for f in futs:
        r = f.result()
        ref[r["k"]] = r
    ex.shutdown()
    same_status, diffs, errs, left_out = 0, [], {"ez": [], "wr": []}, []
    for k, (nxt, st, fail), g, wk in zip(ks, stops, heads, wakes):
        r = ref[k]
        same_status += int(st == r["status"])
        if st == r["status"] == 4:
            diffs.append(fail - r["fail"])
        if r["idx"].size == 0:
            g.close()
            continue
        rr = g.ring_dumps(which=("r",))["r"]
        bf = g.beam_fields(which=("ez", "wr"))
        xi = np.concatenate([b.xi for b in wk.beams])
        rb = np.concatenate([b.r for b in wk.beams]).astype(np.float32)
        sl = np.floor(xi / wk.dxi + 0.5).astype(np.int64)
        sel = r["idx"]
        below = np.empty(sel.shape[0], dtype=np.int32)
        order = np.argsort(sl[sel], kind="stable")
        srt = sel[order]
        bounds = np.searchsorted(sl[srt], np.arange(r["laminar"] + 1))
        for s_ in range(r["laminar"]):
            a, b = bounds[s_], bounds[s_ + 1]
            if a < b:
                below[order[a:b]] = np.searchsorted(np.sort(rr[s_]), rb[srt[a:b]], side="left")
        ok = below == r["below"]
        left_out.append(1.0 - ok.mean())
        for f in ("ez", "wr"):
            den = float(np.max(np.abs(r[f][ok]))) if ok.any() else 0.0
            d = float(np.max(np.abs(bf[f][sel][ok] - r[f][ok]))) if ok.any() else 0.0
            errs[f].append(d / den if den > 0 else d)
        g.close()
    q = lambda v, p: float(np.percentile(v, p)) if len(v) else None  # noqa: E731
    return {"members": len(ks), "same_status": same_status,
            "stopped_at_guard_in_oracle": int(sum(ref[k]["status"] != 0 for k in ks)),
            "stop_slice_minus_oracles": {"min": min(diffs) if diffs else None, "median": q(diffs, 50),
                                         "max": max(diffs) if diffs else None, "n": len(diffs)},
            "laminar_head_errors": {f: {"max": max(v) if v else None, "median": q(v, 50), "p90": q(v, 90)}
                                    for f, v in errs.items()},
            "particles_on_a_ring_left_out": {"max": max(left_out) if left_out else None,
                                             "median": q(left_out, 50)},
            "note": "mixed path vs the FP64 oracle, norm-wise per member; laminar head = the first 300 "
                    "slices before any two rings cross", "oracle_s": time.perf_counter() - t0, "cores": cores}


def _oracle_share(task):
    """One host core's share of the oracle sample (runs in a spawned
    process): wakes first, first + stride, ... until `seconds` have passed."""
    first, stride, seconds, slices = task
    import oracle
    done = used = 0
    k = first
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds and k < 256:
        wk = W.batched_wake(k)
        res = oracle.run_wake(wk, max_slices=slices, beam_fields=())
        done += wk.n_rings * res.slices_run
        used += 1
        k += stride
    return done, used


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The oracle, as it stands, on every host core: independent wakes in
    spawned worker processes (spawn, never fork: the parent may hold a CUDA
    context)."""

    def __init__(self, cores: int):
        import concurrent.futures
        import multiprocessing
        self.cores = cores
        self.ex = concurrent.futures.ProcessPoolExecutor(max_workers=cores,
                                                         mp_context=multiprocessing.get_context("spawn"))
        list(self.ex.map(_oracle_share, [(c, cores, 0.0, 1) for c in range(cores)]))  # start the workers

    def sample(self, seconds: float, slices: int = 400):
        t0 = time.perf_counter()
        res = list(self.ex.map(_oracle_share, [(c, self.cores, seconds, slices) for c in range(self.cores)]))
        dt = time.perf_counter() - t0
        done = sum(r[0] for r in res)
        used = sum(r[1] for r in res)
        return {"value": done / dt, "unit": UNIT, "cores": self.cores, "kind": "oracle",
                "sample": f"first {slices} slices of {used} batched wakes in {self.cores} processes "
                          f"({done} ring-slices, {dt:.1f} s)"}

    def close(self):
        self.ex.shutdown()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    # each step: the oracle on a bounded sample of the workload, on every
    # host core (independent wakes in parallel processes)
    import oracle
    oracle.build()
    per_step = max(2.0, args.cpu_seconds / max(1, args.steps))
    pool = OraclePool(_host_cores())
    for _ in range(args.warmup):
        pool.sample(0.5)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = pool.sample(per_step)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    pool.close()
    value = statistics.mean(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batched: {args.n_wakes} independent wakes, log-uniform 500-8000 rings, "
                                   "1000-6000 slices of 0.01, 50k-500k beam particles",
                       "n_wakes": args.n_wakes},
            "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": last["cores"], "sample": last["sample"], "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_uniform(args):
    """A batch of identical wakes (--uniform RINGS,SLICES,COPIES): one batched
    march, timed with CUDA events; the small, fixed case the kernel profiles
    are taken on.  Driver: n_b0 = 1, sigma_r = 0.5, sigma_z = 1, 20k particles;
    uniform rings out to 6; d xi = 0.01.  --uniform-kind: the AB2 march
    ("ab2"), mobile hydrogen ions ("ions", RINGS per species) or RK4."""
    import torch
    from paper_2603_16623_gb300 import wake as wm
    n, slices, copies = (int(v) for v in args.uniform.split(","))
    drv = W.gaussian_beam(20_000, 1.0, 0.5, 1.0, 0.5, seed=5)
    kind = {"ab2": {}, "ions": {"ions": (1.0, 1836.0)}, "rk4": {"integrator": "rk4"}}[args.uniform_kind]
    wk = W.Wake(f"uniform{n}", W.edges_uniform(n, 6.0), [drv], 0.01, slices, **kind)
    n = n * (2 if args.uniform_kind == "ions" else 1)
    flags = wm.WAKE_NO_STAGE if args.no_stage else 0
    shape = {}
    if args.uniform_shape:
        k, cl = (int(v) for v in args.uniform_shape.split(","))
        shape = {"rings_per_thread": k, "cluster_ctas": cl}
    gs = [wm.Wake.from_workload(wk, precision="mixed", flags=flags, **shape) for _ in range(copies)]
    wm.wake_batch_run(gs)
    torch.cuda.synchronize()
    wm.wake_batch_reset(gs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    wm.wake_batch_run(gs)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"case": "uniform", "kind": args.uniform_kind, "staged": not args.no_stage,
                      "rings": n, "slices": slices, "copies": copies,
                      "launch": gs[0].launch_config(), "march_ms": ms, "us_per_slice": ms * 1e3 / slices,
                      "ring_slices_per_s": n * slices * copies / (ms / 1e3)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-wakes", type=int, default=256)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--plain-wakes", type=int, default=4)
    ap.add_argument("--plain-slices", type=int, default=300)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--skip-push", action="store_true")
    ap.add_argument("--skip-ions", action="store_true")
    ap.add_argument("--ion-wakes", type=int, default=152)
    ap.add_argument("--skip-rk4", action="store_true")
    ap.add_argument("--skip-grid", action="store_true")
    ap.add_argument("--skip-singles", action="store_true")
    ap.add_argument("--large-oracle-slices", type=int, default=300)
    ap.add_argument("--grid-wakes", type=int, default=64)
    ap.add_argument("--grid-slices", type=int, default=300)
    ap.add_argument("--rk4-wakes", type=int, default=152)
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=500.0)
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--serve-step-us", type=float, default=10000.0)
    ap.add_argument("--serve-sm-fill", type=float, default=2.0,
                    help="admit while running wakes hold fewer than this many SMs' worth (x SM count); 0: no cap")
    ap.add_argument("--uniform", default=None, help="RINGS,SLICES,COPIES: one batch of identical wakes")
    ap.add_argument("--uniform-kind", default="ab2", choices=["ab2", "ions", "rk4"])
    ap.add_argument("--uniform-shape", default=None,
                    help="--uniform: RINGS_PER_THREAD,CTAS (the on-chip march's launch shape; default automatic)")
    ap.add_argument("--no-stage", action="store_true",
                    help="--uniform: read each slice's beam from global memory (no bulk-copy staging)")
    ap.add_argument("--skip-stage-ab", action="store_true")
    ap.add_argument("--skip-parity-sample", action="store_true")
    ap.add_argument("--rings-per-cta", type=int, default=0, help="cluster wakes: at most this many rings per CTA")
    ap.add_argument("--autotune", default=None, choices=["batch", "probe"],
                    help="launch shapes of the batched wakes from a tuning run on this GPU: on the batch's own "
                         "step time (autotune.tune_batch) or per size class on probe wakes (autotune.tune)")
    ap.add_argument("--autotune-sizes", default="512,1024,2048,3072,4096,6144,8192",
                    help="ring counts of the tuned size classes")
    ap.add_argument("--autotune-fill", type=float, default=2.0,
                    help="probe tuning: CTAs in flight while a shape is timed, in SMs (2: throughput of a "
                         "full GPU; small: one wake alone, its latency)")
    args = ap.parse_args()
    if args.uniform:
        run_uniform(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
