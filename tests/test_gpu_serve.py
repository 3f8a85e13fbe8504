"""Continuous batching (paper_2603_16623_gb300/serve.py) on the GPU: every
request's result is the same alone and in the mix, however it was split
into steps and whatever shared the device with it."""
import numpy as np
import pytest

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


def _mix():
    """Ten wakes of different sizes (one needs a two-CTA cluster) and windows."""
    out = []
    for k, (n, steps, nb0) in enumerate([(300, 420, 1.0), (900, 260, 4.0), (2600, 180, 2.0), (64, 500, 0.5),
                                         (1500, 333, 8.0), (700, 150, 0.2), (1200, 610, 3.0), (450, 90, 1.5),
                                         (2048, 240, 6.0), (128, 700, 12.0)]):
        drv = W.gaussian_beam(8_000 + 1000 * k, nb0, 0.3, 0.5, 1.6, seed=700 + k)
        out.append(W.Wake(f"s{k}", W.edges_uniform(n, 6.0), [drv], 0.01, steps))
    return out


class _Clock:
    def __init__(self, dt):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def _alone(wk):
    from paper_2603_16623_gb300 import wake as wm
    g = wm.Wake.from_workload(wk, precision="mixed")
    g.step_slices(wk.n_steps)
    nxt, st, _ = g.progress()
    bf = g.beam_fields(("ez", "wr"))
    g.close()
    return nxt, st, bf


def test_served_requests_equal_alone():
    from paper_2603_16623_gb300 import serve
    wakes = _mix()
    ref = [_alone(wk) for wk in wakes]
    reqs = []
    for i, wk in enumerate(wakes):
        arrival = 0.0 if i < 5 else 0.02 * (i - 4)  # a burst, then a trickle
        reqs.append(serve.Request(rid=i, arrival=arrival, edges=wk.edges, beams=wk.beams, dxi=wk.dxi,
                                  n_steps=wk.n_steps, out_ez=np.zeros(wk.n_beam, np.float32),
                                  out_wr=np.zeros(wk.n_beam, np.float32)))
    # a budget of about three wakes forces queueing; short steps make
    # requests join and leave the batch mid-flight
    budget = 3 * max(serve.estimate_device_bytes(w.n_rings, w.n_beam, w.n_steps) for w in wakes)
    srv = serve.WakeServer(budget, step_ns=300_000, clock=_Clock(0.001))
    stats = serve.run_stream(srv, reqs)
    assert len(stats.completed) == len(wakes)
    assert stats.steps > len(wakes)
    assert stats.max_queue >= 2
    for req, wk, (nxt, st, bf) in zip(reqs, wakes, ref):
        assert req.status == st, req.rid
        assert req.slices_done == min(nxt, wk.n_steps), req.rid
        assert np.array_equal(req.out_ez, bf["ez"]), req.rid
        assert np.array_equal(req.out_wr, bf["wr"]), req.rid
    s = stats.summary()
    assert s["requests"] == len(wakes) and s["p99_ms"] >= s["p50_ms"] > 0


def test_batch_step_limits_and_progress():
    from paper_2603_16623_gb300 import wake as wm
    wakes = _mix()[:6]
    gs = [wm.Wake.from_workload(wk, precision="mixed") for wk in wakes]
    wm.wake_batch_step(gs, 7)
    nxt, st = wm.wake_batch_progress(gs)
    assert list(nxt) == [min(7, wk.n_steps) for wk in wakes] and not st.any()
    # a short time budget stops every wake after at least one more slice
    wm.wake_batch_step(gs, 1 << 30, 50_000)
    nxt2, st2 = wm.wake_batch_progress(gs)
    assert all(b > a for a, b in zip(nxt, nxt2))
    wm.wake_batch_step(gs, 1 << 30)
    nxt3, st3 = wm.wake_batch_progress(gs)
    for g, wk, n, s in zip(gs, wakes, nxt3, st3):
        alone = _alone(wk)
        assert (n, s) == alone[:2]
        assert np.array_equal(g.beam_fields(("ez",))["ez"], alone[2]["ez"])
        g.close()


def test_device_bytes_estimate_bounds_the_allocation():
    from paper_2603_16623_gb300 import serve, wake as wm
    for wk in _mix()[:4] + [W.batched_wake(5)]:
        g = wm.Wake.from_workload(wk, precision="mixed", flags=wm.WAKE_INIT_ASYNC)
        got = g.device_bytes()
        est = serve.estimate_device_bytes(wk.n_rings, wk.n_beam, wk.n_steps)
        assert 0 < got <= est, (wk.name, got, est)
        g.close()


def test_pipelined_reset_run_equals_reset_then_run():
    """wake_batch_reset_run gives bitwise the results of wake_batch_reset +
    wake_batch_run, on a batch that mixes one-CTA and cluster wakes, a
    mobile-ion wake and an RK4 wake, run twice in a row."""
    from paper_2603_16623_gb300 import wake as wm
    wakes = _mix()[:6]
    drv = W.gaussian_beam(9_000, 1.0, 0.3, 0.5, 1.6, seed=731)
    wakes.append(W.Wake("ions", W.edges_uniform(300, 5.0), [drv], 0.01, 260, ions=(1.0, 100.0)))
    wakes.append(W.Wake("rk4", W.edges_uniform(280, 5.0), [drv], 0.01, 240, integrator="rk4"))
    a = [wm.Wake.from_workload(wk, precision="mixed") for wk in wakes]
    b = [wm.Wake.from_workload(wk, precision="mixed") for wk in wakes]
    for _ in range(2):
        wm.wake_batch_reset(a)
        wm.wake_batch_run(a)
        wm.wake_batch_reset_run(b)
        na, sa = wm.wake_batch_progress(a)
        nb, sb = wm.wake_batch_progress(b)
        assert list(na) == list(nb) and list(sa) == list(sb)
        for ga, gb in zip(a, b):
            fa, fb = ga.beam_fields(("ez", "wr")), gb.beam_fields(("ez", "wr"))
            assert np.array_equal(fa["ez"], fb["ez"]) and np.array_equal(fa["wr"], fb["wr"])
            assert np.array_equal(ga.ring_state()[0], gb.ring_state()[0])
    for g in a + b:
        g.close()


def test_time_budget_on_the_one_cta_marches():
    """The budgeted batch step also stops the two-species, RK4 and grid
    marches at a slice boundary; run on to the end, they give what they give
    alone (bitwise; the grid's node charges are summed with atomics: to
    float rounding)."""
    from paper_2603_16623_gb300 import wake as wm
    drv = W.gaussian_beam(9_000, 1.0, 0.3, 0.5, 1.6, seed=741)
    wakes = [W.Wake("ions", W.edges_uniform(600, 5.0), [drv], 0.01, 400, ions=(1.0, 100.0)),
             W.Wake("rk4", W.edges_uniform(600, 5.0), [drv], 0.01, 400, integrator="rk4"),
             W.Wake("grid", W.edges_uniform(600, 5.0), [drv], 0.01, 400, grid_nr=32)]
    alone = []
    for wk in wakes:
        g = wm.Wake.from_workload(wk, precision="mixed")
        g.run()
        alone.append((g.ring_state()[0], g.beam_fields(("ez",))["ez"]))
        g.close()
    gs = [wm.Wake.from_workload(wk, precision="mixed") for wk in wakes]
    wm.wake_batch_step(gs, 1 << 30, 50_000)
    nxt, st = wm.wake_batch_progress(gs)
    assert not st.any()
    assert all(0 < k < wk.n_steps for k, wk in zip(nxt, wakes)), list(nxt)
    wm.wake_batch_step(gs, 1 << 30)
    for g, wk, (r, ez) in zip(gs, wakes, alone):
        assert g.progress()[:2] == (wk.n_steps, 0)
        if wk.name == "grid":
            assert np.max(np.abs(g.beam_fields(("ez",))["ez"] - ez)) <= 1e-5 * np.max(np.abs(ez))
        else:
            assert np.array_equal(g.ring_state()[0], r) and np.array_equal(g.beam_fields(("ez",))["ez"], ez)
        g.close()
