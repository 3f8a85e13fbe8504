"""The bench's multi-rank host logic on CPU with gloo, world size 2: each
rank takes a disjoint share of the batched workload (weak scaling) and the
reported time is the maximum over ranks, the work the sum."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    names = [w.name for w in bench._workload(3, rank)]
    t_max, rs_sum = bench._reduce_max_sum(10.0 + 5.0 * rank, 1000 * (rank + 1), "cpu")
    out.put((rank, names, t_max, rs_sum))
    dist.destroy_process_group()


def test_two_ranks_shard_wakes_and_reduce_max_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, t0, s0), (r1, n1, t1, s1) = res
    assert not set(n0) & set(n1)
    assert n0 == ["batched[0]", "batched[1]", "batched[2]"]
    assert t0 == t1 == 15.0
    assert s0 == s1 == 3000.0


def test_beam_evaluations_count_the_particles_of_marched_slices():
    """Step a9 evaluates each beam particle binned into a slice its wake
    marched: floor(xi / dxi + 1/2) in [0, next slice)."""
    import numpy as np

    import bench
    from paper_2603_16623_gb300 import workloads as W
    xi = np.array([-0.006, -0.004, 0.0, 0.0049, 0.005, 0.0151, 0.02, 0.5])
    beam = W.Beam(xi, np.full(xi.shape, 0.3), np.full(xi.shape, 1e-3), -1.0)
    wk = W.Wake("evals", W.edges_uniform(10, 2.0), [beam, beam], 0.01, 3)
    # slices: -1, 0, 0, 0, 1, 2, 2, 50 (two beams of each)
    assert bench.beam_evaluations([wk], [0]) == 0
    assert bench.beam_evaluations([wk], [1]) == 2 * 3
    assert bench.beam_evaluations([wk], [3]) == 2 * 6
    assert bench.beam_evaluations([wk, wk], [3, 2]) == 2 * 6 + 2 * 4


def _fake_served(rank, world, n_req=40):
    """The requests this rank serves of one dispatched stream, completed
    with made-up latencies (no GPU): (owner array, ServeStats)."""
    import numpy as np

    from paper_2603_16623_gb300 import serve
    from paper_2603_16623_gb300 import workloads as W
    rng = np.random.Generator(np.random.PCG64(4))
    pick = rng.integers(0, 256, n_req)
    arrivals = serve.poisson_arrivals(n_req, 500.0 * world, 4)
    work = [W.batched_params(int(k)).n_rings * W.batched_params(int(k)).n_steps for k in pick]
    owner = serve.dispatch(work, world)
    st = serve.ServeStats()
    for i in np.nonzero(owner == rank)[0]:
        p = W.batched_params(int(pick[i]))
        r = serve.Request(rid=int(i), arrival=float(arrivals[i]), edges=np.linspace(0, 6, p.n_rings + 1), beams=(),
                          dxi=0.01, n_steps=p.n_steps)
        r.finished = r.arrival + 0.001 * (1 + i % 7)
        r.slices_done = p.n_steps
        r.status = 0
        st.completed.append(r)
    st.steps, st.max_active, st.max_queue, st.peak_bytes = 10 + rank, 3 + rank, 2, 1000 * (rank + 1)
    return owner, st


def _serve_rank_main(rank, world, port, out):
    import torch.distributed as dist

    from paper_2603_16623_gb300 import serve
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    owner, st = _fake_served(rank, world)
    out.put((rank, owner.tolist(), serve.gather_summary(st)))
    dist.destroy_process_group()


def test_two_ranks_dispatch_one_stream_and_gather_the_latencies():
    """Every rank computes the same assignment of one request stream; the
    gathered summary covers the union of both ranks' requests (percentiles
    over all latencies, steps summed, peaks maximised)."""
    import numpy as np
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_serve_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, own0, s0), (_, own1, s1) = res
    assert own0 == own1 and set(own0) == {0, 1}
    assert s0 == s1
    lat = [0.001 * (1 + i % 7) for i in range(len(own0))]
    assert s0["requests"] == len(own0) and s0["requests_per_rank"] == [own0.count(0), own0.count(1)]
    assert abs(s0["p50_ms"] - np.percentile(lat, 50) * 1e3) < 1e-9
    assert abs(s0["p99_ms"] - np.percentile(lat, 99) * 1e3) < 1e-9
    assert s0["steps"] == 21 and s0["max_active"] == 4 and s0["peak_device_bytes"] == 2000


def test_dispatch_balances_work_and_one_rank_takes_everything():
    import numpy as np

    from paper_2603_16623_gb300 import serve
    rng = np.random.Generator(np.random.PCG64(9))
    work = rng.uniform(1.0, 10.0, 500)
    for n in (2, 3, 8):
        owner = serve.dispatch(work, n)
        load = np.bincount(owner, weights=work, minlength=n)
        assert load.max() - load.min() <= work.max()
        assert np.array_equal(owner, serve.dispatch(work, n))
    assert not serve.dispatch(work, 1).any()
    # one server's summary is the summary of its records
    _, st = _fake_served(0, 1)
    assert st.summary() == serve.summarize(st.records(), [st.counters()])


def test_batched_params_are_the_members_parameters():
    from paper_2603_16623_gb300 import workloads as W
    for k in (0, 5, 77):
        p, wk = W.batched_params(k), W.batched_wake(k)
        assert (p.n_rings, p.n_steps, p.n_mp) == (wk.n_rings, wk.n_steps, wk.beams[0].n)
        assert wk.edges[-1] == p.r_max


def test_latency_roofline_of_the_critical_wake():
    """The bench's latency bound: per slice, the critical wake's block's
    warp instructions at min(1, warps per scheduler / FMA latency) per
    scheduler-cycle plus its barriers' latency, times its slices; a missing
    input is reported, not raised."""
    import bench
    onchip = {"fma_latency_cycles": 4.0, "syncthreads_ns": 20.0, "cluster_barrier_ns": 200.0, "sm_clock_mhz": 2000.0}
    # one block of 512 threads x 4 rings: 4 warps per scheduler, full rate
    one = {"critical_wake": {"rings": 2048, "slices": 100, "threads": 512, "rings_per_thread": 4, "ctas": 1},
           "longest_wake_ms": 4.0}
    r = bench.latency_roofline(one, onchip)
    issue = bench.WARP_INSTR_PER_RING_SLICE["one_cta"] * 2048 / 4.0 / 2000.0
    barriers = bench.BLOCK_BARRIERS_PER_SLICE["one_cta"] * 20.0 / 1e3
    assert r["kind"] == "one_cta"
    assert abs(r["per_slice_us"]["issue"] - issue) < 1e-12
    assert abs(r["bound_ms"] - 100 * (issue + barriers) / 1e3) < 1e-12
    assert abs(r["frac"] - r["bound_ms"] / 4.0) < 1e-12
    # a cluster of 256-thread blocks: 2 warps per scheduler, half rate, and the cluster barriers
    cl = {"critical_wake": {"rings": 6000, "slices": 10, "threads": 256, "rings_per_thread": 4, "ctas": 6},
          "longest_wake_ms": 1.0}
    r = bench.latency_roofline(cl, onchip)
    issue = bench.WARP_INSTR_PER_RING_SLICE["cluster"] * 1024 / (4 * 2 / 4.0) / 2000.0
    barriers = (bench.BLOCK_BARRIERS_PER_SLICE["cluster"] * 20.0 + bench.CLUSTER_BARRIERS_PER_SLICE * 200.0) / 1e3
    assert r["kind"] == "cluster"
    assert abs(r["bound_ms"] - 10 * (issue + barriers) / 1e3) < 1e-12
    assert "unavailable" in bench.latency_roofline({"critical_wake": {"unavailable": "x"}}, onchip)
