"""The beam push between wake solves on the GPU (wake_push_beam) against
the oracle's Boris push (oracle/beam_push.py): one push in the same fields,
element by element, and a loop of solve -> push -> re-bin -> solve against
the same loop of the oracle."""
import numpy as np
import pytest

import oracle
from oracle import beam_push as bp
from paper_2603_16623_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2603_16623_gb300 import wake
    wake.load()
    yield


def nerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a - b)))


def _phase_space(beam, seed):
    """A beam's full phase space around its (xi, r): random azimuth,
    transverse momenta ~ N(0, 0.5), u_z ~ 1000 +- 10."""
    rng = np.random.Generator(np.random.PCG64(seed))
    phi = rng.uniform(0, 2 * np.pi, beam.n)
    return {"x": beam.r * np.cos(phi), "y": beam.r * np.sin(phi), "xi": beam.xi.copy(),
            "ux": rng.normal(0, 0.5, beam.n), "uy": rng.normal(0, 0.5, beam.n),
            "uz": 1000.0 + rng.normal(0, 10.0, beam.n)}


def _wake(n_rings=300, steps=400, nb0=0.5, seed=31):
    drv = W.gaussian_beam(20_000, nb0, 0.4, 0.8, 2.8, seed=seed)
    return W.Wake(f"push{seed}", W.edges_uniform(n_rings, 5.0), [drv], 0.01, steps)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_push_matches_oracle_in_the_same_fields(precision):
    from paper_2603_16623_gb300 import wake as wm
    wk = _wake()
    g = wm.Wake.from_workload(wk, precision=precision)
    st, _, _, _ = g.run()
    assert st == 0
    ps0 = _phase_space(wk.beams[0], 7)
    g.set_beam_phase_space(ps0["x"], ps0["y"], ps0["ux"], ps0["uy"], ps0["uz"])
    f = g.beam_fields(("ez", "wr", "bt"))
    dt = 0.25
    g.push_beam(dt)
    got = g.beam_phase_space()
    ref = bp.push(ps0, f["ez"].astype(np.float64), f["wr"].astype(np.float64), f["bt"].astype(np.float64),
                  wk.beams[0].q, dt)
    for k in ("x", "y", "xi", "ux", "uy", "uz"):
        # the increments themselves (the state is large next to them).  FP64:
        # a few roundings, except the xi step dt (1 - u_z/gamma), ~1e-7 of
        # xi at gamma ~ 1000, where one rounding of xi (or of the oracle's
        # cancelling 1 - u_z/gamma) is ~4e-9 of it.  Mixed: the increments
        # are taken in FP32 from inputs truncated to 24 bits, ~10 roundings
        # of 2^-24 (6e-8) each at most
        if precision == "fp64":
            tol = 1e-7 if k == "xi" else 1e-9
        else:
            tol = 2e-6
        assert nerr(got[k] - ps0[k], ref[k] - ps0[k]) < tol, k
        # the state: the increment's error scaled to the state, and FP64
        # rounding of the sum
        d = np.max(np.abs(ref[k] - ps0[k])) / np.max(np.abs(ref[k]))
        assert nerr(got[k], ref[k]) < tol * d + 1e-15, k
    assert nerr(got["r"], np.hypot(got["x"], got["y"])) < (1e-15 if precision == "fp64" else 1e-13)
    g.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("mixed", 1e-4)])
def test_solve_push_loop_matches_oracle_loop(precision, tol):
    """Three time steps of: solve the wake of the current beam, push the
    beam in it, bin the moved beam again, against the same loop of the
    oracle.  Mixed wakes carry their fields' norm-wise 1e-5 into every
    step's increments, three steps of it within 1e-4."""
    from paper_2603_16623_gb300 import wake as wm
    wk = _wake(n_rings=200, steps=350, nb0=1.0, seed=33)
    b = wk.beams[0]
    ps = _phase_space(b, 9)
    dt = 2.0
    g = wm.Wake.from_workload(wk, precision=precision)
    g.set_beam_phase_space(ps["x"], ps["y"], ps["ux"], ps["uy"], ps["uz"])
    ref = dict(ps)
    ref["r"] = np.hypot(ps["x"], ps["y"])
    for step in range(3):
        # oracle: the wake of the beam as it is now, then the push
        res = oracle.run_wake(W.Wake(wk.name, wk.edges, [W.Beam(ref["xi"], ref["r"], b.w, b.q)], wk.dxi,
                                     wk.n_steps))
        assert res.status == 0
        ref = bp.push(ref, res.beam["ez"], res.beam["wr"], res.beam["bt"], b.q, dt)
        # GPU
        if step:
            g.reset()
        st, _, _, _ = g.run()
        assert st == 0
        g.push_beam(dt)
    got = g.beam_phase_space()
    for k in ("x", "y", "xi", "ux", "uy", "uz"):
        assert nerr(got[k] - ps[k], ref[k] - ps[k]) < tol, k
    g.close()


def test_push_rejects_bad_use():
    from paper_2603_16623_gb300 import wake as wm
    wk = _wake(n_rings=64, steps=50)
    g = wm.Wake.from_workload(wk, precision="mixed")
    with pytest.raises(wm.WakeError):
        g.push_beam(0.1)        # no phase space yet
    b = wk.beams[0]
    g.set_beam_phase_space(b.r, np.zeros(b.n), np.zeros(b.n), np.zeros(b.n), np.full(b.n, 100.0))
    with pytest.raises(wm.WakeError):
        g.push_beam(-1.0)
    g.close()


def test_two_species_and_batched_push_match_oracle():
    """wake_batch_push_beam over wakes of different sizes, one of them with
    an electron driver and a positron witness (per-species charge), in one
    launch, against the oracle's push of each wake in the same fields.  The
    last wake's witness lies partly behind the window: particles outside see
    no field and drift."""
    from paper_2603_16623_gb300 import wake as wm
    wakes = [_wake(n_rings=120, steps=300, nb0=0.3, seed=41), _wake(n_rings=700, steps=250, nb0=2.0, seed=42)]
    drv = W.gaussian_beam(30_000, 1.0, 0.3, 0.6, 2.0, seed=43, q=-1.0)
    wit = W.gaussian_beam(7_000, 0.2, 0.2, 0.3, 3.3, seed=44, q=+1.0)
    wakes.append(W.Wake("twospecies", W.edges_uniform(400, 5.0), [drv, wit], 0.01, 340))
    gs, ps0s, fields = [], [], []
    for i, wk in enumerate(wakes):
        g = wm.Wake.from_workload(wk, precision="mixed")
        st, _, _, _ = g.run()
        assert st == 0
        xi = np.concatenate([b.xi for b in wk.beams])
        r = np.concatenate([b.r for b in wk.beams])
        beam = W.Beam(xi, r, np.concatenate([b.w for b in wk.beams]), -1.0)
        ps0 = _phase_space(beam, 50 + i)
        g.set_beam_phase_space(ps0["x"], ps0["y"], ps0["ux"], ps0["uy"], ps0["uz"])
        gs.append(g)
        ps0s.append(ps0)
        fields.append(g.beam_fields(("ez", "wr", "bt")))
    assert np.any(np.concatenate([b.xi for b in wakes[2].beams]) > 340 * 0.01)  # some outside the window
    dt = 0.4
    wm.wake_batch_push_beam(gs, dt)
    for g, wk, ps0, f in zip(gs, wakes, ps0s, fields):
        q = np.concatenate([np.full(b.n, b.q) for b in wk.beams])
        ref = bp.push(ps0, f["ez"].astype(np.float64), f["wr"].astype(np.float64), f["bt"].astype(np.float64),
                      q, dt)
        got = g.beam_phase_space()
        for k in ("x", "y", "xi", "ux", "uy", "uz"):
            assert nerr(got[k] - ps0[k], ref[k] - ps0[k]) < 2e-6, (wk.name, k)
        g.close()


def _crowding_beam():
    """Three groups of 1000 particles in slices 18, 19, 20 whose axial
    velocities would slip them all into slice 30 in one push of dt = 0.2
    (where 100 fast particles sit) without fields: the densest slice grows
    from 1000 particles to over 2000."""
    rng = np.random.Generator(np.random.PCG64(77))
    xi, uz = [], []
    for xi0, vz in ((0.20, 0.5), (0.19, 0.45), (0.18, 0.4)):
        xi.append(np.full(1000, xi0))
        uz.append(np.full(1000, vz / np.sqrt(1 - vz * vz)))
    xi.append(np.full(100, 0.30))
    uz.append(np.full(100, 2000.0))
    xi, uz = np.concatenate(xi), np.concatenate(uz)
    r = 0.3 * np.sqrt(-2 * np.log(1 - rng.random(xi.shape[0])))
    beam = W.Beam(xi, r, np.full(xi.shape[0], 2e-4), -1.0)
    return W.Wake("crowd", W.edges_uniform(150, 4.0), [beam], 0.01, 60), uz


@pytest.mark.parametrize("batched", [False, True])
def test_a_push_that_crowds_a_slice_is_binned_again(batched):
    from paper_2603_16623_gb300 import wake as wm
    wk, uz = _crowding_beam()
    n = wk.n_beam
    g = wm.Wake.from_workload(wk, precision="fp64")
    st, _, _, _ = g.run()
    assert st == 0
    g.set_beam_phase_space(wk.beams[0].r, np.zeros(n), np.zeros(n), np.zeros(n), uz)
    if batched:
        wm.wake_batch_push_beam([g], 0.2)
        wm.wake_batch_reset([g])
        wm.wake_batch_run([g])
        st = g.progress()[1]
    else:
        g.push_beam(0.2)
        g.reset()
        st, _, _, _ = g.run()
    assert st == 0
    ps = g.beam_phase_space()
    sl = np.floor(ps["xi"] / wk.dxi + 0.5).astype(int)
    # the fields spread the slow groups over a few slices; the densest now
    # holds more than the 1024 that a sort sized from before the push takes
    assert np.bincount(sl).max() > 1024
    ref = oracle.run_wake(W.Wake(wk.name, wk.edges, [W.Beam(ps["xi"], ps["r"], wk.beams[0].w, -1.0)], wk.dxi,
                                 wk.n_steps))
    got = g.beam_fields(("ez", "wr"))
    for k in ("ez", "wr"):
        assert nerr(got[k], ref.beam[k]) < 1e-10, k
    g.close()
