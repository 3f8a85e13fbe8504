"""Staging of each slice's beam arrays in shared memory by bulk asynchronous
copies (the on-chip marches of the mixed path): the staged march gives the
same results as the one that reads the beam from global memory, bitwise, on
one CTA and on clusters, with slices that fit the stage and slices denser
than it; and the march's bounded wait for a staged slice, made to run out by
the test flag that never issues that slice's copies, stops the wake with
WAKE_ETIMEOUT before that slice, after which the device and the library
stay usable."""
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


def _wm():
    from paper_2603_16623_gb300 import wake
    return wake


def _cases():
    return [
        # one CTA, every slice fits the stage
        W.Wake("one_cta", W.edges_uniform(700, 6.0), [W.gaussian_beam(60_000, 2.0, 0.3, 0.6, 2.4, seed=11)], 0.01, 500),
        # one CTA of 64 threads (a small stage) with slices denser than it:
        # those read the beam from global memory
        W.Wake("dense", W.edges_uniform(200, 5.0), [W.gaussian_beam(400_000, 5.0, 0.2, 0.3, 1.2, seed=12)], 0.01, 300),
        # clusters of 3 and 5 CTAs, two beams
        W.Wake("cluster3", W.edges_uniform(3000, 6.0),
               [W.gaussian_beam(80_000, 3.0, 0.4, 0.5, 2.0, seed=13),
                W.gaussian_beam(20_000, 0.0, 0.05, 0.2, 4.5, seed=14, total=2.0)], 0.01, 400),
        W.Wake("cluster5", W.edges_uniform(4915, 6.0), [W.gaussian_beam(300_000, 2.0, 1.0, 0.6, 2.4, seed=15)], 0.01,
               300),
    ]


# the dense case keeps one CTA of 64 threads x 4 rings: a small stage
SHAPES = {"dense": {"rings_per_thread": 4, "cluster_ctas": 1}}


def _run(wk, flags):
    wm = _wm()
    g = wm.Wake.from_workload(wk, precision="mixed", flags=flags, **SHAPES.get(wk.name, {}))
    st, _, _, _ = g.run()
    out = {"status": st, "progress": g.progress(), "beam": g.beam_fields(), "state": g.ring_state(history=True),
           "launch": g.launch_config()}
    g.close()
    return out


@pytest.mark.parametrize("case", range(4))
def test_staged_march_equals_global_loads_bitwise(case):
    wm = _wm()
    wk = _cases()[case]
    a = _run(wk, 0)
    b = _run(wk, wm.WAKE_NO_STAGE)
    assert a["status"] == b["status"] == 0 and a["progress"] == b["progress"]
    for k in a["beam"]:
        assert np.array_equal(a["beam"][k], b["beam"][k]), k
    for x, y in zip(a["state"], b["state"]):
        assert np.array_equal(x, y)
    if case >= 2:
        assert a["launch"][2] > 1  # a cluster


def test_staged_batch_equals_global_loads_bitwise():
    wm = _wm()
    wakes = _cases()
    out = []
    for flags in (0, wm.WAKE_NO_STAGE):
        gs = [wm.Wake.from_workload(wk, precision="mixed", flags=flags, **SHAPES.get(wk.name, {})) for wk in wakes]
        wm.wake_batch_run(gs)
        out.append([(g.progress(), g.beam_fields(which=("ez", "wr")), g.ring_state()) for g in gs])
        for g in gs:
            g.close()
    for (pa, ba, sa), (pb, bb, sb) in zip(*out):
        assert pa == pb
        assert all(np.array_equal(ba[k], bb[k]) for k in ba)
        assert all(np.array_equal(x, y) for x, y in zip(sa, sb))


@pytest.mark.parametrize("case", [0, 2])
def test_a_stage_wait_that_runs_out_stops_the_wake_with_etimeout(case):
    """The flag skips the bulk copies of the first beam slice staged after
    the launch's first slice while its mbarrier still expects their bytes:
    the bounded wait gives up (after ~0.25 s), every CTA of the wake stops
    before that slice with status WAKE_ETIMEOUT, no copy is left in flight,
    and the device stays usable."""
    wm = _wm()
    wk = _cases()[case]
    xi = np.concatenate([b.xi for b in wk.beams])
    sl = np.floor(xi / wk.dxi + 0.5).astype(np.int64)
    s_stall = int(sl[sl >= 1].min())  # the first slice after 0 that holds particles
    g = wm.Wake.from_workload(wk, precision="mixed", flags=wm.WAKE_TEST_STALL_STAGE)
    g.step_slices(wk.n_steps)
    assert g.progress() == (s_stall, wm.WAKE_ETIMEOUT, s_stall)
    with pytest.raises(wm.WakeError) as e:
        g.run()
    assert e.value.status == wm.WAKE_ETIMEOUT
    with pytest.raises(wm.WakeError) as e:
        g.fields_at(np.array([0.5]))
    assert e.value.status == wm.WAKE_ETIMEOUT
    g.close()
    # the same wake without the flag: solved whole, as the staged march
    # always gives it
    ref = _run(wk, 0)
    again = _run(wk, 0)
    assert ref["status"] == again["status"] == 0
    assert np.array_equal(ref["beam"]["ez"], again["beam"]["ez"])
