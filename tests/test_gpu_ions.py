"""GPU parity of wakes with mobile ions (the two-species march of
march_ions.cuh) against the oracle's two-species march (orc_run_ions):
electrons and ions as ring species on the same cells, each solved on its own
rings and gathered into the other by linear interpolation, B_theta^(p) from
the electrons, ions moving with q/m = Z/M (Sec. II, multiple plasma
species).

Tolerances as for electron-only wakes: 1e-10 norm-wise for FP64, 1e-5 for
the mixed path on ring radii and on E_z, W_r at beam particles whose place
among the rings (of either species) is unambiguous at the run's precision.
Strong wakes are checked slice by slice through the checkpoint API (the
oracle's state at slice n, one GPU slice, compared with the oracle's slice
n and state n + 1)."""
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


def ion_wake(n=300, steps=500, nb0=1.5, ions=(1.0, 100.0), seed=61, edges=None):
    drv = W.gaussian_beam(40_000, nb0, 0.3, 0.6, 1.8, seed=seed)
    e = W.edges_uniform(n, 5.0) if edges is None else edges
    return W.Wake(f"ions{seed}", e, [drv], 0.01, steps, ions=ions)


def gpu_run(wk, precision, threads=0, dumps=True):
    from paper_2603_16623_gb300 import wake as wm
    g = wm.Wake.from_workload(wk, precision=precision, block_threads=threads,
                              flags=wm.WAKE_DUMP_RING_FIELDS if dumps else 0)
    assert g.n_rings == 2 * wk.n_rings
    st, _, _, _ = g.run()
    out = {"status": st, "progress": g.progress(), "beam": g.beam_fields(), "final": g.ring_state()}
    if dumps:
        out["rings"] = g.ring_dumps()
    g.close()
    return out


def oracle_run(wk, dumps=True):
    keys = ("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb") if dumps else ()
    return oracle.run_wake(wk, ring_dumps=keys)


@pytest.mark.parametrize("threads", [64, 256])
def test_fp64_ion_wake_matches_oracle(threads):
    wk = ion_wake()
    ref = oracle_run(wk)
    assert ref.status == 0
    # the ions have moved measurably
    n = wk.n_rings
    assert np.max(np.abs(ref.final_r[n:] - ref.rings["r"][0][n:])) > 1e-4
    got = gpu_run(wk, "fp64", threads)
    assert got["status"] == 0
    for k in ("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt", "psi"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k


def test_fp64_light_multiply_charged_ions_on_refined_cells():
    """Z = 2, M = 25 (q/m = 0.08) on refined cells with a ragged ring count."""
    wk = ion_wake(steps=400, nb0=3.0, ions=(2.0, 25.0), seed=62, edges=W.edges_refined(150, 1.0, 133, 5.0))
    ref = oracle_run(wk)
    assert ref.status == 0
    got = gpu_run(wk, "fp64", 128)
    assert got["status"] == 0
    for k in ("r", "ur", "psi", "dpsidr", "dpsidz", "bp"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k


def test_mixed_ion_wake_within_tolerance():
    wk = ion_wake(n=500, steps=600, seed=63)
    ref = oracle_run(wk)
    got = gpu_run(wk, "mixed", 256)
    assert got["status"] == ref.status == 0
    assert nerr(got["rings"]["r"], ref.rings["r"]) < MIXED_TOL
    ok = unambiguous(wk, ref.rings["r"], got["rings"]["r"])
    assert ok.mean() > 0.95
    for k in ("ez", "wr"):
        assert nerr(got["beam"][k][ok], ref.beam[k][ok]) < MIXED_TOL, k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_step_parity_on_a_strong_ion_wake(precision):
    """A dense narrow driver with light ions: rings cross and the ions
    collapse onto the axis; every 50th slice is solved once on the GPU from
    the oracle's state."""
    from paper_2603_16623_gb300 import wake as wm
    drv = W.gaussian_beam(60_000, 12.0, 0.15, 0.5, 2.0, seed=64)
    wk = W.Wake("strong_ions", W.edges_uniform(400, 4.0), [drv], 0.01, 700, ions=(1.0, 20.0))
    ref = oracle.run_wake(wk, ring_dumps=("r", "ur", "frprev", "fuprev", "psi", "dpsidr", "dpsidz", "bp", "bb"))
    R = ref.rings
    n2 = 2 * wk.n_rings
    bad = []
    for n in range(0, ref.slices_run - 1, 50):
        g = wm.Wake.from_workload(wk, precision=precision, flags=wm.WAKE_DUMP_RING_FIELDS)
        g.set_ring_state(n, R["r"][n], R["ur"][n], R["frprev"][n], R["fuprev"][n])
        g.step_slices(1)
        assert g.progress()[:2] == (n + 1, 0)
        d = g.ring_dumps()
        rho, ur = g.ring_state()
        keep = np.ones(n2, dtype=bool)
        if precision == "mixed":
            # rings of one species tied in float may sort either way
            for s in (0, 1):
                idx = np.arange(s * wk.n_rings, (s + 1) * wk.n_rings)
                order = idx[np.argsort(R["r"][n][idx], kind="stable")]
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


def test_ion_wakes_batched_equal_alone():
    from paper_2603_16623_gb300 import wake as wm
    wakes = [ion_wake(n=200, steps=300, seed=65), ion_wake(n=333, steps=250, ions=(1.0, 400.0), seed=66),
             W.Wake("plain", W.edges_uniform(250, 5.0), [W.gaussian_beam(20_000, 1.0, 0.3, 0.6, 1.8, seed=67)],
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


def test_ion_wake_checkpoint_round_trip_resumes_bitwise():
    from paper_2603_16623_gb300 import wake as wm
    wk = ion_wake(n=180, steps=300, seed=68)
    for precision in ("fp64", "mixed"):
        a = wm.Wake.from_workload(wk, precision=precision)
        a.step_slices(110)
        rho, ur, fr, fu = a.ring_state(history=True)
        assert rho.shape == (2 * wk.n_rings,)
        a.step_slices(1000)
        b = wm.Wake.from_workload(wk, precision=precision)
        b.set_ring_state(110, rho, ur, fr, fu)
        b.step_slices(1000)
        ra, rb = a.ring_state(), b.ring_state()
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1]), precision
        a.close()
        b.close()


def test_ion_wake_rejects_bad_arguments():
    from paper_2603_16623_gb300 import wake as wm
    wk = ion_wake(n=50, steps=20)
    for ions in ((-1.0, 10.0), (1.0, 0.0), (1.0, float("nan"))):
        with pytest.raises(wm.WakeError):
            wm.Wake.from_workload(wk, precision="mixed", ions=ions)
    with pytest.raises(wm.WakeError):
        wm.Wake.from_workload(wk, precision="mixed", rings_per_thread=4)
    big = W.Wake("big", W.edges_uniform(4097, 5.0), [], 0.01, 10, ions=(1.0, 100.0))
    with pytest.raises(wm.WakeError):
        wm.Wake.from_workload(big, precision="mixed")


# ---------------------------------------------------------------------------
# radial density profiles (carried by both ring species)
# ---------------------------------------------------------------------------
def profile_wake(ions, n=300, steps=450, seed=70, nb0=1.5):
    e = W.edges_refined(120, 1.5, n - 120, 6.0)
    drv = W.gaussian_beam(40_000, nb0, 0.3, 0.6, 1.8, seed=seed)
    return W.Wake(f"profile{seed}", e, [drv], 0.01, steps, ions=ions, cell_density=W.parabolic_profile(e, 1.0, 3.0))


def test_fp64_parabolic_channel_with_static_ion_rings_matches_oracle():
    wk = profile_wake((1.0, float("inf")))
    ref = oracle_run(wk)
    assert ref.status == 0
    n = wk.n_rings
    assert np.array_equal(ref.final_r[n:], ref.rings["r"][0][n:])  # the ions stand still
    got = gpu_run(wk, "fp64", 256)
    assert got["status"] == 0
    assert np.array_equal(got["final"][0][n:], ref.final_r[n:])
    for k in ("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt", "psi"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k


def test_mixed_parabolic_channel_with_mobile_ions_within_tolerance():
    wk = profile_wake((1.0, 200.0), seed=71)
    ref = oracle_run(wk)
    got = gpu_run(wk, "mixed", 256)
    assert got["status"] == ref.status == 0
    assert nerr(got["rings"]["r"], ref.rings["r"]) < MIXED_TOL
    ok = unambiguous(wk, ref.rings["r"], got["rings"]["r"])
    assert ok.mean() > 0.95
    for k in ("ez", "wr"):
        assert nerr(got["beam"][k][ok], ref.beam[k][ok]) < MIXED_TOL, k


def test_profile_rejects_bad_use():
    from paper_2603_16623_gb300 import wake as wm
    wk = profile_wake((1.0, 100.0), n=160, steps=20)
    with pytest.raises(wm.WakeError):  # a profile needs ion rings
        wm.Wake.from_workload(wk, precision="mixed", ions=None)
    bad = np.array(wk.cell_density)
    bad[7] = -1.0
    with pytest.raises(wm.WakeError):
        wm.Wake.from_workload(wk, precision="mixed", cell_density=bad)


# ---------------------------------------------------------------------------
# the two-species march on a thread-block cluster (wide wakes): its blocks
# split each species' positions, the scans fold over the cluster
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
def test_fp64_ion_wake_on_a_cluster_matches_oracle(threads, cluster):
    """300 cells: 2-3 rings per species and thread over 2-3 blocks (ragged),
    and 8 blocks of which the last three hold no ring."""
    wk = ion_wake()
    ref = oracle_run(wk)
    assert ref.status == 0
    got = gpu_run_cl(wk, "fp64", threads, cluster)
    assert got["cfg"][0] == threads and got["cfg"][2] == cluster
    assert got["status"] == 0
    for k in ("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt", "psi"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k


def test_fp64_ion_cluster_on_refined_cells():
    """Refined cells with a ragged ring count, Z = 2, M = 25, on 3 blocks of
    96 threads."""
    wk = ion_wake(steps=400, nb0=3.0, ions=(2.0, 25.0), seed=62, edges=W.edges_refined(150, 1.0, 133, 5.0))
    ref = oracle_run(wk)
    got = gpu_run_cl(wk, "fp64", 96, 3)
    assert got["status"] == ref.status == 0
    for k in ("r", "ur", "psi", "dpsidr", "dpsidz", "bp"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k


def test_mixed_ion_wake_on_a_cluster_within_tolerance():
    wk = ion_wake(n=500, steps=600, seed=63)
    ref = oracle_run(wk)
    got = gpu_run_cl(wk, "mixed", 128, 4)
    assert got["status"] == ref.status == 0
    assert nerr(got["rings"]["r"], ref.rings["r"]) < MIXED_TOL
    ok = unambiguous(wk, ref.rings["r"], got["rings"]["r"])
    assert ok.mean() > 0.95
    for k in ("ez", "wr"):
        assert nerr(got["beam"][k][ok], ref.beam[k][ok]) < MIXED_TOL, k


def test_ion_cluster_shapes_and_rejections():
    from paper_2603_16623_gb300 import wake as wm
    # automatic: a cluster once a block of 512 threads would hold more than 2
    # rings of each species per thread
    for cells, blocks in ((1024, 1), (1025, 2), (2048, 2), (3000, 3), (4096, 4)):
        wk = W.Wake("shape", W.edges_uniform(cells, 5.0), [], 0.01, 10, ions=(1.0, 100.0))
        g = wm.Wake.from_workload(wk, precision="mixed")
        assert g.launch_config() == (512, -(-2 * cells // (512 * blocks)), blocks), cells
        assert g.launch_config() == wm.wake_gm_launch_shape(cells, "ions")  # the host-side query agrees
        g.close()
    wk = ion_wake(n=50, steps=20)
    for bad in (-1, 9, 16):
        with pytest.raises(wm.WakeError):
            wm.Wake.from_workload(wk, precision="mixed", cluster_ctas=bad)


def test_ion_cluster_static_query_and_budgeted_steps():
    """Fields at query radii between slices, and steps bounded by a time
    budget (the blocks agree on where to stop), resumed to the window's end:
    the same bits as an unbounded run on the same cluster."""
    from paper_2603_16623_gb300 import wake as wm
    wk = ion_wake(n=400, steps=300, seed=69)
    a = wm.Wake.from_workload(wk, precision="fp64", block_threads=64, cluster_ctas=4)
    b = wm.Wake.from_workload(wk, precision="fp64", block_threads=64, cluster_ctas=1)
    for g in (a, b):
        wm.wake_batch_step([g], 120)
    rq = np.linspace(0.0, 6.0, 777)
    fa, fb = a.fields_at_static(rq), b.fields_at_static(rq)
    for k in ("ez", "wr", "bt", "psi"):
        assert nerr(fa[k], fb[k]) < FP64_TOL, k
    a.run()
    ref = (a.ring_state(), a.beam_fields())
    a.close()
    c = wm.Wake.from_workload(wk, precision="fp64", block_threads=64, cluster_ctas=4)
    while c.progress()[0] < wk.n_steps:
        wm.wake_batch_step([c], wk.n_steps, time_budget_ns=200_000)
    assert all(np.array_equal(x, y) for x, y in zip(c.ring_state(), ref[0]))
    fc = c.beam_fields()
    assert all(np.array_equal(fc[k], ref[1][k]) for k in ref[1])
    c.close()
    b.close()


def test_ion_cluster_wakes_batched_equal_alone():
    """A batch mixing one-block and cluster shapes (automatic: 1100 cells
    take 2 blocks) gives each wake the bits of its run alone."""
    from paper_2603_16623_gb300 import wake as wm
    wakes = [ion_wake(n=1100, steps=120, seed=71), ion_wake(n=300, steps=150, seed=72),
             ion_wake(n=1500, steps=100, ions=(1.0, 400.0), seed=73)]
    alone = []
    for wk in wakes:
        g = wm.Wake.from_workload(wk, precision="mixed")
        g.run()
        alone.append((g.launch_config(), g.ring_state(), g.beam_fields(("ez", "wr"))))
        g.close()
    assert [c[2] for c, _, _ in alone] == [2, 1, 2]
    gs = [wm.Wake.from_workload(wk, precision="mixed") for wk in wakes]
    wm.wake_batch_run(gs)
    for g, (_, st, bf) in zip(gs, alone):
        r, u = g.ring_state()
        assert np.array_equal(r, st[0]) and np.array_equal(u, st[1])
        f = g.beam_fields(("ez", "wr"))
        assert np.array_equal(f["ez"], bf["ez"]) and np.array_equal(f["wr"], bf["wr"])
        g.close()


def test_ion_scratch_in_global_memory_when_shared_memory_is_short():
    """A block keeps its rings' own-thread values in shared memory when the
    launch has room; 4096 cells on one block of 512 threads (8 rings of each
    species per thread) leave none, and the kernel keeps them in global
    memory: the results agree with the same wake on 4 blocks (FP64 1e-10)."""
    wk = ion_wake(n=4096, steps=80, ions=(1.0, 1836.0), seed=74)
    one = gpu_run_cl(wk, "fp64", 512, 1, dumps=False)
    four = gpu_run_cl(wk, "fp64", 512, 4, dumps=False)
    assert one["cfg"] == (512, 16, 1) and four["cfg"] == (512, 4, 4)
    assert one["status"] == four["status"] == 0
    assert nerr(one["final"][0], four["final"][0]) < FP64_TOL
    for k in ("ez", "wr", "bt", "psi"):
        assert nerr(one["beam"][k], four["beam"][k]) < FP64_TOL, k
