"""GPU parity of the RK4 ring integrator (march_rk4.cuh) against the
oracle's RK4 march (orc_run with integrator "rk4"): classical RK4 over each
slice, the beam source at the half step the mean of slices n and n+1, stage
states below the axis evaluated mirrored.  Tolerances as for AB2 wakes:
1e-10 norm-wise (FP64), 1e-5 (mixed) on ring radii and on E_z, W_r at beam
particles whose place among the rings is unambiguous; strong wakes slice by
slice from the oracle's state."""
import numpy as np
import pytest

import oracle
from paper_2603_16623_gb300 import workloads as W
from test_gpu_parity import FP64_TOL, MIXED_FIELD_TOL, MIXED_TOL, nerr, unambiguous

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2603_16623_gb300 import wake
    wake.load()
    yield


def rk4_wake(n=300, steps=500, nb0=1.5, sig_r=0.3, seed=81, edges=None):
    drv = W.gaussian_beam(40_000, nb0, sig_r, 0.6, 1.8, seed=seed)
    e = W.edges_uniform(n, 5.0) if edges is None else edges
    return W.Wake(f"rk4_{seed}", e, [drv], 0.01, steps, integrator="rk4")


def gpu_run(wk, precision, threads=0, dumps=True):
    from paper_2603_16623_gb300 import wake as wm
    g = wm.Wake.from_workload(wk, precision=precision, block_threads=threads,
                              flags=wm.WAKE_DUMP_RING_FIELDS if dumps else 0)
    st, _, _, _ = g.run()
    out = {"status": st, "progress": g.progress(), "beam": g.beam_fields(), "final": g.ring_state()}
    if dumps:
        out["rings"] = g.ring_dumps()
    g.close()
    return out


def oracle_run(wk, dumps=True):
    keys = ("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb") if dumps else ()
    return oracle.run_wake(wk, ring_dumps=keys)


@pytest.mark.parametrize("threads", [64, 512])
def test_fp64_rk4_wake_matches_oracle(threads):
    wk = rk4_wake()
    ref = oracle_run(wk)
    assert ref.status == 0
    got = gpu_run(wk, "fp64", threads)
    assert got["status"] == 0
    for k in ("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt", "psi"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k
    assert nerr(got["final"][0], ref.final_r) < FP64_TOL


def test_fp64_rk4_axis_crossings_match_oracle():
    """A dense narrow driver: rings cross each other and the axis (stage
    states mirrored), on refined cells with a ragged ring count."""
    wk = rk4_wake(steps=450, nb0=5.0, sig_r=0.15, seed=82, edges=W.edges_refined(140, 1.0, 157, 5.0))
    ref = oracle_run(wk)
    assert ref.status == 0
    assert np.any(np.diff(np.sign(ref.rings["ur"]), axis=0) != 0)
    got = gpu_run(wk, "fp64", 256)
    assert got["status"] == 0
    for k in ("r", "ur", "psi", "dpsidz", "bp"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k


def test_mixed_rk4_wake_within_tolerance():
    wk = rk4_wake(n=600, steps=600, seed=83)
    ref = oracle_run(wk)
    got = gpu_run(wk, "mixed")
    assert got["status"] == ref.status == 0
    assert nerr(got["rings"]["r"], ref.rings["r"]) < MIXED_TOL
    ok = unambiguous(wk, ref.rings["r"], got["rings"]["r"])
    assert ok.mean() > 0.95
    for k in ("ez", "wr"):
        assert nerr(got["beam"][k][ok], ref.beam[k][ok]) < MIXED_TOL, k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_step_parity_on_a_strong_rk4_wake(precision):
    from paper_2603_16623_gb300 import wake as wm
    drv = W.gaussian_beam(60_000, 10.0, 0.15, 0.5, 2.0, seed=84)
    wk = W.Wake("strong_rk4", W.edges_uniform(400, 4.0), [drv], 0.01, 800, integrator="rk4")
    ref = oracle.run_wake(wk, ring_dumps=("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"))
    R = ref.rings
    bad = []
    # from slice 60 on: before the driver the fields are rounding noise, so
    # a norm-wise relative error there measures nothing
    for n in range(60, ref.slices_run - 1, 60):
        g = wm.Wake.from_workload(wk, precision=precision, flags=wm.WAKE_DUMP_RING_FIELDS)
        g.set_ring_state(n, R["r"][n], R["ur"][n])
        g.step_slices(1)
        assert g.progress()[:2] == (n + 1, 0)
        d = g.ring_dumps()
        rho, ur = g.ring_state()
        keep = np.ones(wk.n_rings, dtype=bool)
        if precision == "mixed":
            order = np.argsort(R["r"][n], kind="stable")
            rs = R["r"][n][order]
            close = np.diff(rs) <= 5e-7 * rs[1:]
            keep[order[1:][close]] = False
            keep[order[:-1][close]] = False
            assert keep.mean() > 0.99
        e = {k: nerr(d[k][n][keep], R[k][n][keep]) for k in ("psi", "dpsidr", "dpsidz", "bp", "bb")}
        e["r"] = nerr(rho[keep], R["r"][n + 1][keep])
        e["ur"] = nerr(ur[keep], R["ur"][n + 1][keep])
        g.close()
        for k, v in e.items():
            tol = FP64_TOL if precision == "fp64" else MIXED_FIELD_TOL.get(k, MIXED_TOL)
            if k == "ur":
                tol = max(tol, 1e-14)
            if not v < tol:
                bad.append((n, k, v))
    assert not bad, bad


def test_rk4_wakes_batched_equal_alone():
    from paper_2603_16623_gb300 import wake as wm
    wakes = [rk4_wake(n=200, steps=300, seed=85), rk4_wake(n=333, steps=250, seed=86),
             W.Wake("ab2", W.edges_uniform(250, 5.0), [W.gaussian_beam(20_000, 1.0, 0.3, 0.6, 1.8, seed=87)],
                    0.01, 280)]
    alone = []
    for wk in wakes:
        g = wm.Wake.from_workload(wk, precision="mixed")
        g.run()
        alone.append((g.ring_state(), g.beam_fields(("ez", "wr"))))
        g.close()
    gs = [wm.Wake.from_workload(wk, precision="mixed") for wk in wakes]
    wm.wake_batch_run(gs)
    for g, (st, bf) in zip(gs, alone):
        r, u = g.ring_state()
        assert np.array_equal(r, st[0]) and np.array_equal(u, st[1])
        f = g.beam_fields(("ez", "wr"))
        assert np.array_equal(f["ez"], bf["ez"]) and np.array_equal(f["wr"], bf["wr"])
        g.close()


def test_rk4_rejects_bad_use():
    from paper_2603_16623_gb300 import wake as wm
    wk = rk4_wake(n=50, steps=20)
    with pytest.raises(wm.WakeError):
        wm.Wake.from_workload(wk, precision="mixed", ions=(1.0, 100.0))
    with pytest.raises(wm.WakeError):
        wm.Wake.from_workload(wk, precision="mixed", rings_per_thread=4)


# ---------------------------------------------------------------------------
# RK4 on a thread-block cluster (wide wakes): the blocks split the sorted
# positions, the scans fold over the cluster, block 0 sorts the state and the
# stage states
# ---------------------------------------------------------------------------
def gpu_run_cl(wk, precision, threads, cluster, dumps=True):
    from paper_2603_16623_gb300 import wake as wm
    g = wm.Wake.from_workload(wk, precision=precision, block_threads=threads, cluster_ctas=cluster,
                              flags=wm.WAKE_DUMP_RING_FIELDS if dumps else 0)
    cfg = g.launch_config()
    st, _, _, _ = g.run()
    out = {"status": st, "progress": g.progress(), "beam": g.beam_fields(), "final": g.ring_state(), "cfg": cfg}
    if dumps:
        out["rings"] = g.ring_dumps()
    g.close()
    return out


@pytest.mark.parametrize("threads,cluster", [(64, 2), (64, 3), (128, 4), (64, 8)])
def test_fp64_rk4_wake_on_a_cluster_matches_oracle(threads, cluster):
    """300 rings over 2-8 blocks (ragged; with 8 blocks of 64 threads at one
    ring each, the last three blocks hold no ring)."""
    wk = rk4_wake()
    ref = oracle_run(wk)
    got = gpu_run_cl(wk, "fp64", threads, cluster)
    assert got["cfg"][0] == threads and got["cfg"][2] == cluster
    assert got["status"] == ref.status == 0
    for k in ("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt", "psi"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k
    assert nerr(got["final"][0], ref.final_r) < FP64_TOL


def test_fp64_rk4_axis_crossings_on_a_cluster_match_oracle():
    """Rings crossing each other and the axis: the state and the stage
    states are re-sorted by block 0 for all three blocks."""
    wk = rk4_wake(steps=450, nb0=5.0, sig_r=0.15, seed=82, edges=W.edges_refined(140, 1.0, 157, 5.0))
    ref = oracle_run(wk)
    assert np.any(np.diff(np.sign(ref.rings["ur"]), axis=0) != 0)
    got = gpu_run_cl(wk, "fp64", 64, 3)
    assert got["status"] == ref.status == 0
    for k in ("r", "ur", "psi", "dpsidz", "bp"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k


def test_mixed_rk4_wake_on_a_cluster_within_tolerance():
    wk = rk4_wake(n=600, steps=600, seed=83)
    ref = oracle_run(wk)
    got = gpu_run_cl(wk, "mixed", 128, 4)
    assert got["status"] == ref.status == 0
    assert nerr(got["rings"]["r"], ref.rings["r"]) < MIXED_TOL
    ok = unambiguous(wk, ref.rings["r"], got["rings"]["r"])
    assert ok.mean() > 0.95
    for k in ("ez", "wr"):
        assert nerr(got["beam"][k][ok], ref.beam[k][ok]) < MIXED_TOL, k


def test_one_step_parity_on_a_strong_rk4_wake_on_a_cluster():
    """The strong wake's slices from the oracle's state, one slice each on a
    cluster of 4 blocks (FP64)."""
    from paper_2603_16623_gb300 import wake as wm
    drv = W.gaussian_beam(60_000, 10.0, 0.15, 0.5, 2.0, seed=84)
    wk = W.Wake("strong_rk4", W.edges_uniform(400, 4.0), [drv], 0.01, 800, integrator="rk4")
    ref = oracle.run_wake(wk, ring_dumps=("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"))
    R = ref.rings
    bad = []
    for n in range(60, ref.slices_run - 1, 120):
        g = wm.Wake.from_workload(wk, precision="fp64", block_threads=64, cluster_ctas=4,
                                  flags=wm.WAKE_DUMP_RING_FIELDS)
        g.set_ring_state(n, R["r"][n], R["ur"][n])
        g.step_slices(1)
        assert g.progress()[:2] == (n + 1, 0)
        d = g.ring_dumps()
        rho, ur = g.ring_state()
        e = {k: nerr(d[k][n], R[k][n]) for k in ("psi", "dpsidr", "dpsidz", "bp", "bb")}
        e["r"] = nerr(rho, R["r"][n + 1])
        e["ur"] = nerr(ur, R["ur"][n + 1])
        g.close()
        bad += [(n, k, v) for k, v in e.items() if not v < max(FP64_TOL, 1e-14 if k == "ur" else 0.0)]
    assert not bad, bad


def test_rk4_cluster_shapes_batches_and_rejections():
    """Automatic blocks per wake (a cluster once a block of 512 threads would
    hold more than 2 rings per thread); a batch mixing one-block and cluster
    shapes gives each wake the bits of its run alone; bad cluster sizes are
    refused."""
    from paper_2603_16623_gb300 import wake as wm
    for rings, blocks in ((1024, 1), (1025, 2), (3000, 3), (7905, 8), (16384, 8)):
        wk = W.Wake("shape", W.edges_uniform(rings, 5.0), [], 0.01, 10, integrator="rk4")
        g = wm.Wake.from_workload(wk, precision="mixed")
        assert g.launch_config() == (512, -(-rings // (512 * blocks)), blocks), rings
        assert g.launch_config() == wm.wake_gm_launch_shape(rings, "rk4")  # the host-side query agrees
        g.close()
    wakes = [rk4_wake(n=1500, steps=60, seed=88), rk4_wake(n=300, steps=80, seed=89),
             rk4_wake(n=600, steps=70, seed=90)]
    shapes = [0, 0, 3]
    alone = []
    for wk, cl in zip(wakes, shapes):
        g = wm.Wake.from_workload(wk, precision="mixed", cluster_ctas=cl)
        g.run()
        alone.append((g.launch_config(), g.ring_state(), g.beam_fields(("ez", "wr"))))
        g.close()
    assert [c[2] for c, _, _ in alone] == [2, 1, 3]
    gs = [wm.Wake.from_workload(wk, precision="mixed", cluster_ctas=cl) for wk, cl in zip(wakes, shapes)]
    wm.wake_batch_run(gs)
    for g, (_, st, bf) in zip(gs, alone):
        r, u = g.ring_state()
        assert np.array_equal(r, st[0]) and np.array_equal(u, st[1])
        f = g.beam_fields(("ez", "wr"))
        assert np.array_equal(f["ez"], bf["ez"]) and np.array_equal(f["wr"], bf["wr"])
        g.close()
    for bad in (-1, 9):
        with pytest.raises(wm.WakeError):
            wm.Wake.from_workload(rk4_wake(n=50, steps=20), precision="mixed", cluster_ctas=bad)
