"""GPU parity of the adaptive beam grids (Sec. IV; the grid path of
march.cuh) against the oracle's grid march (orc_run with grid_nr > 0):
per beam species grid_nr radial cells covering its particles, one node line
per slice, B^(b) at the rings from the grids, beam-particle fields
interpolated from the nodes.  FP64 1e-10 and mixed 1e-5 norm-wise.  The node charges are
summed with atomics on the GPU (order-dependent rounding), so batched and
alone runs agree to rounding, not bitwise."""
import numpy as np
import pytest

import oracle
from paper_2603_16623_gb300 import workloads as W
from test_gpu_parity import FP64_TOL, nerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2603_16623_gb300 import wake
    wake.load()
    yield


def grid_wake(grid_nr=32, n=300, steps=400, seed=91, two_beams=False):
    drv = W.gaussian_beam(30_000, 0.8, 0.35, 0.6, 1.8, seed=seed)
    beams = [drv]
    if two_beams:
        beams.append(W.gaussian_beam(8_000, 0.3, 0.12, 0.2, 3.2, seed=seed + 1))
    return W.Wake(f"grid{seed}", W.edges_uniform(n, 5.0), beams, 0.01, steps, grid_nr=grid_nr)


def gpu_run(wk, threads=0):
    from paper_2603_16623_gb300 import wake as wm
    g = wm.Wake.from_workload(wk, precision="fp64", block_threads=threads, flags=wm.WAKE_DUMP_RING_FIELDS)
    st, _, _, _ = g.run()
    out = {"status": st, "beam": g.beam_fields(), "rings": g.ring_dumps(), "final": g.ring_state()}
    g.close()
    return out


@pytest.mark.parametrize("grid_nr,threads", [(32, 256), (7, 64)])
def test_fp64_grid_wake_matches_oracle(grid_nr, threads):
    wk = grid_wake(grid_nr)
    ref = oracle.run_wake(wk, ring_dumps=("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"))
    assert ref.status == 0
    got = gpu_run(wk, threads)
    assert got["status"] == 0
    for k in ("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt", "psi"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k


def test_fp64_driver_and_witness_grids_match_oracle():
    """Two species with grids of different extents (the witness narrower)."""
    wk = grid_wake(24, steps=420, seed=93, two_beams=True)
    ref = oracle.run_wake(wk, ring_dumps=("r", "bb"))
    assert ref.status == 0
    got = gpu_run(wk, 128)
    assert got["status"] == 0
    assert nerr(got["rings"]["r"], ref.rings["r"]) < FP64_TOL
    assert nerr(got["rings"]["bb"], ref.rings["bb"]) < FP64_TOL
    for k in ("ez", "wr", "bt"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k


def test_grid_wakes_batched_match_alone():
    from paper_2603_16623_gb300 import wake as wm
    wakes = [grid_wake(16, n=200, steps=250, seed=95), grid_wake(40, n=260, steps=300, seed=96, two_beams=True)]
    alone = []
    for wk in wakes:
        g = wm.Wake.from_workload(wk, precision="fp64")
        g.run()
        alone.append((g.ring_state(), g.beam_fields(("ez", "wr"))))
        g.close()
    gs = [wm.Wake.from_workload(wk, precision="fp64") for wk in wakes]
    wm.wake_batch_run(gs)
    for g, (st, bf) in zip(gs, alone):
        r, _ = g.ring_state()
        assert nerr(r, st[0]) < 1e-12
        f = g.beam_fields(("ez", "wr"))
        assert nerr(f["ez"], bf["ez"]) < 1e-12 and nerr(f["wr"], bf["wr"]) < 1e-12
        g.close()


def test_mixed_grid_wake_within_tolerance():
    """The mixed one-CTA march (float-float radii and weights, ln rho from
    the table) with grids, against the oracle at the mixed path's 1e-5; the
    grids decide node membership from the caller's FP64 radii."""
    from paper_2603_16623_gb300 import wake as wm
    wk = grid_wake(32, n=400, steps=500, seed=97, two_beams=True)
    ref = oracle.run_wake(wk, ring_dumps=("r",))
    g = wm.Wake.from_workload(wk, precision="mixed", flags=wm.WAKE_DUMP_RING_R)
    st, _, _, rr = g.run(ring_r=True)
    assert st == ref.status == 0
    assert nerr(rr, ref.rings["r"]) < 1e-5
    f = g.beam_fields(("ez", "wr", "bt"))
    for k in ("ez", "wr", "bt"):
        assert nerr(f[k], ref.beam[k]) < 1e-5, k
    g.close()


def test_grid_rejects_bad_use():
    from paper_2603_16623_gb300 import wake as wm
    wk = grid_wake(8, n=50, steps=20)
    with pytest.raises(wm.WakeError):
        wm.Wake.from_workload(wk, precision="mixed", ions=(1.0, 100.0))
    with pytest.raises(wm.WakeError):
        wm.Wake.from_workload(wk, precision="fp64", grid_nr=2000)
    with pytest.raises(wm.WakeError):
        wm.Wake.from_workload(wk, precision="fp64", integrator="rk4")


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", 1e-5)])
def test_regular_intermediate_grid_matches_oracle(precision, tol):
    """A fixed grid extent of 2.5 for both beams (the regular grid)."""
    from paper_2603_16623_gb300 import wake as wm
    wk = grid_wake(48, n=300, steps=400, seed=98, two_beams=True)
    wk = W.Wake(wk.name, wk.edges, wk.beams, wk.dxi, wk.n_steps, grid_nr=48, grid_rmax=2.5)
    ref = oracle.run_wake(wk, ring_dumps=("r",))
    assert ref.status == 0
    g = wm.Wake.from_workload(wk, precision=precision, flags=wm.WAKE_DUMP_RING_R)
    st, _, _, rr = g.run(ring_r=True)
    assert st == 0
    assert nerr(rr, ref.rings["r"]) < tol
    f = g.beam_fields(("ez", "wr", "bt"))
    for k in ("ez", "wr", "bt"):
        assert nerr(f[k], ref.beam[k]) < tol, k
    g.close()


def test_a_particle_moved_beyond_a_fixed_grid_stops_the_wake():
    """Moving a particle beyond the fixed extent (here by giving it a phase
    space there) stops the next solve with status EINVAL before any slice."""
    from paper_2603_16623_gb300 import wake as wm
    wk = grid_wake(16, n=100, steps=50, seed=99)
    wk = W.Wake(wk.name, wk.edges, wk.beams, wk.dxi, wk.n_steps, grid_nr=16, grid_rmax=3.0)
    g = wm.Wake.from_workload(wk, precision="fp64")
    st, _, _, _ = g.run()
    assert st == 0
    b = wk.beams[0]
    x = b.r.copy()
    x[5] = 3.5
    g.set_beam_phase_space(x, np.zeros(b.n), np.zeros(b.n), np.zeros(b.n), np.full(b.n, 100.0))
    g.reset()
    g.step_slices(10)
    nxt, status, fail = g.progress()
    assert status == wm.WAKE_EINVAL and nxt == 0
    g.close()


# ---------------------------------------------------------------------------
# beam-grid wakes on a thread-block cluster: the blocks split the sorted
# rings, the grid nodes and the slice's particles; block 0 sorts the rings
# and sums the node charges (deposited by every block with atomics)
# ---------------------------------------------------------------------------
def gpu_run_cl(wk, precision, threads, cluster):
    from paper_2603_16623_gb300 import wake as wm
    g = wm.Wake.from_workload(wk, precision=precision, block_threads=threads, cluster_ctas=cluster,
                              flags=wm.WAKE_DUMP_RING_FIELDS)
    cfg = g.launch_config()
    st, _, _, _ = g.run()
    out = {"status": st, "beam": g.beam_fields(), "rings": g.ring_dumps(), "final": g.ring_state(), "cfg": cfg}
    g.close()
    return out


@pytest.mark.parametrize("threads,cluster", [(64, 2), (96, 3), (64, 8)])
def test_fp64_grid_wake_on_a_cluster_matches_oracle(threads, cluster):
    """300 rings over 2, 3 and 8 blocks (with 8 blocks of 64 threads, the
    last three hold no ring), two beams with grids of different extents."""
    wk = grid_wake(24, steps=420, seed=93, two_beams=True)
    ref = oracle.run_wake(wk, ring_dumps=("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"))
    assert ref.status == 0
    got = gpu_run_cl(wk, "fp64", threads, cluster)
    assert got["cfg"][0] == threads and got["cfg"][2] == cluster
    assert got["status"] == 0
    for k in ("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb"):
        assert nerr(got["rings"][k], ref.rings[k]) < FP64_TOL, k
    for k in ("ez", "wr", "bt", "psi"):
        assert nerr(got["beam"][k], ref.beam[k]) < FP64_TOL, k


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", 1e-5)])
def test_regular_and_mixed_grids_on_a_cluster(precision, tol):
    """The regular grid (fixed extent 2.5) on 4 blocks against the oracle."""
    wk = grid_wake(48, n=300, steps=400, seed=98, two_beams=True)
    wk = W.Wake(wk.name, wk.edges, wk.beams, wk.dxi, wk.n_steps, grid_nr=48, grid_rmax=2.5)
    ref = oracle.run_wake(wk, ring_dumps=("r",))
    got = gpu_run_cl(wk, precision, 64, 4)
    assert got["status"] == ref.status == 0
    assert nerr(got["rings"]["r"], ref.rings["r"]) < tol
    for k in ("ez", "wr", "bt"):
        assert nerr(got["beam"][k], ref.beam[k]) < tol, k


def test_grid_cluster_shapes_batches_queries_and_rejections():
    """Automatic blocks per wake (a cluster once a block of 256 threads would
    hold more than 4 rings per thread); a batch mixing one-block and cluster
    grid wakes matches the wakes alone (1e-12: node charges summed with
    atomics); fields at query radii between slices on a cluster match one
    block; bad shapes refused."""
    from paper_2603_16623_gb300 import wake as wm
    for rings, blocks in ((1024, 1), (1025, 2), (3000, 3), (8192, 8)):
        wk = W.Wake("shape", W.edges_uniform(rings, 5.0), [], 0.01, 10, grid_nr=16)
        g = wm.Wake.from_workload(wk, precision="fp64")
        assert g.launch_config() == (256, -(-rings // (256 * blocks)), blocks), rings
        assert g.launch_config() == wm.wake_gm_launch_shape(rings, "grid")  # the host-side query agrees
        g.close()
    wakes = [grid_wake(16, n=1500, steps=150, seed=101), grid_wake(40, n=260, steps=200, seed=96, two_beams=True)]
    alone = []
    for wk in wakes:
        g = wm.Wake.from_workload(wk, precision="fp64")
        g.run()
        alone.append((g.launch_config(), g.ring_state(), g.beam_fields(("ez", "wr"))))
        g.close()
    assert [c[2] for c, _, _ in alone] == [2, 1]
    gs = [wm.Wake.from_workload(wk, precision="fp64") for wk in wakes]
    wm.wake_batch_run(gs)
    for g, (_, st, bf) in zip(gs, alone):
        r, _ = g.ring_state()
        assert nerr(r, st[0]) < 1e-12
        f = g.beam_fields(("ez", "wr"))
        assert nerr(f["ez"], bf["ez"]) < 1e-12 and nerr(f["wr"], bf["wr"]) < 1e-12
        g.close()
    wk = grid_wake(32, n=400, steps=300, seed=102)
    a = wm.Wake.from_workload(wk, precision="fp64", block_threads=64, cluster_ctas=4)
    b = wm.Wake.from_workload(wk, precision="fp64", block_threads=64, cluster_ctas=1)
    for g in (a, b):
        wm.wake_batch_step([g], 150)
    rq = np.linspace(0.0, 6.0, 555)
    fa, fb = a.fields_at_static(rq), b.fields_at_static(rq)
    for k in ("ez", "wr", "bt", "psi"):
        assert nerr(fa[k], fb[k]) < FP64_TOL, k
    a.close()
    b.close()
    for kw in ({"cluster_ctas": 9}, {"cluster_ctas": -1}, {"rings_per_thread": 4}):
        with pytest.raises(wm.WakeError):
            wm.Wake.from_workload(grid_wake(8, n=50, steps=20), precision="mixed", **kw)
