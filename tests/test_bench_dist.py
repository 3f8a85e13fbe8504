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
