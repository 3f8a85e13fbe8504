"""The launch-shape autotuner's host logic (paper_2603_16623_gb300/
autotune.py) on CPU: candidates come from the library's own shape query
(wake_launch_shape, which needs no device), the choice follows the timings
with the automatic shape kept unless beaten by min_gain, and a table maps
ring counts to shapes the library accepts.  Timings are fakes here; the GPU
test times real launches."""
import math

import pytest

from paper_2603_16623_gb300 import autotune as at
from paper_2603_16623_gb300 import wake as wm


@pytest.fixture(scope="module", autouse=True)
def _lib():
    wm.load()
    yield


@pytest.mark.parametrize("n", [1, 100, 512, 2048, 2049, 4000, 8192, 16385, 40000, 65536])
def test_candidates_are_shapes_the_library_accepts(n):
    cands = at.candidates(n, "mixed", max_candidates=8)
    assert cands[0].automatic
    assert (cands[0].threads, cands[0].ctas) == (wm.wake_launch_shape(n)[0], wm.wake_launch_shape(n)[2])
    assert 1 <= len(cands) <= 8
    shapes = set()
    for c in cands[1:]:
        t, k, cl = wm.wake_launch_shape(n, c.rings_per_thread, c.cluster_ctas)
        assert (t, cl) == (c.threads, c.ctas) and k == c.rings_per_thread
        assert t >= 64 and t <= 512 and 1 <= cl <= 16
        assert t * k * cl >= n and (cl == 1 or t * k * (cl - 1) < n)
        shapes.add((t, k, cl))
    assert len(shapes) == len(cands) - 1
    assert wm.wake_launch_shape(n) not in shapes  # the automatic shape is timed once


def test_candidates_span_the_cluster_sizes():
    cands = at.candidates(6000, "mixed", max_candidates=6)
    ctas = [c.ctas for c in cands[1:]]
    assert ctas == sorted(ctas) and ctas[0] < ctas[-1]
    full = at.candidates(6000, "mixed", max_candidates=100)
    assert cands[1] == full[1] and cands[-1] == full[-1]  # the thinning keeps both ends


def test_global_memory_marches_tune_the_block_size_and_clusters():
    for kind, default in (("fp64", 256), ("ions", 512), ("rk4", 512), ("grid", 256)):
        cands = at.candidates(1000, kind)
        assert cands[0].automatic
        sized = [c for c in cands[1:] if c.block_threads]
        assert sorted(c.block_threads for c in sized) == sorted(t for t in (64, 128, 256, 512) if t != default)
        clustered = [c for c in cands[1:] if not c.block_threads]
        if kind in ("ions", "rk4", "grid"):
            # a block size alone means one block per wake; then clusters of 512 threads
            assert all(c.cluster_ctas == 1 and c.wake_kwargs()["cluster_ctas"] == 1 for c in sized)
            assert [(c.cluster_ctas, c.ctas) for c in clustered] == [(2, 2), (4, 4), (8, 8)]
            assert clustered[1].wake_kwargs() == {"rings_per_thread": 0, "cluster_ctas": 4}
        else:
            assert not clustered and all(c.cluster_ctas == 0 for c in sized)
    with pytest.raises(ValueError):
        at.candidates(5000, "ions")  # more cells than the two-species march takes
    with pytest.raises(ValueError):
        at.candidates(9000, "fp64")


def _fake_rate(favour, gain):
    """Every shape at 1e9 ring-slices/s, the favoured one `gain` faster."""
    def rate(n, c):
        return 1e9 * (1.0 + gain) if favour(c) else 1e9
    return rate


def test_the_fastest_shape_is_chosen_and_the_automatic_one_kept_within_noise():
    n = 4000
    target = at.candidates(n)[2]
    res = at.tune_size(n, "mixed", _fake_rate(lambda c: c == target, 0.10))
    assert res.chosen == target
    assert len(res.rates) == len(at.candidates(n)) and max(r["ring_slices_per_s"] for r in res.rates) == 1.1e9
    res = at.tune_size(n, "mixed", _fake_rate(lambda c: c == target, 0.01), min_gain=0.03)
    assert res.chosen.automatic
    slow_auto = at.tune_size(n, "mixed", lambda n_, c: 0.5e9 if c.automatic else 1e9)
    assert not slow_auto.chosen.automatic


def test_table_maps_ring_counts_to_accepted_shapes():
    # favour 8 rings per thread in as few CTAs as the library allows
    def rate(n, c):
        return 2e9 - 1e7 * c.ctas if c.rings_per_thread == 8 else 1e9
    table = at.tune((1024, 4096, 16384), "mixed", rate)
    assert [e.n_max for e in table.entries] == [1024, 4096, wm.wake_max_rings("mixed")]
    for n in (10, 700, 1024, 1025, 3000, 4096, 5000, 16384, 30000, 65536):
        kw = table.shape_for(n)
        if kw:
            t, k, cl = wm.wake_launch_shape(n, kw["rings_per_thread"], kw["cluster_ctas"])
            assert k == 8 and t <= 512
    # the class tuned at 4096 rings: 8 rings per thread and the rings per CTA it was timed with
    e = table.entry_for(3000)
    assert e.n_max == 4096 and e.rings_per_thread == 8
    kw = table.shape_for(4096)
    assert kw["cluster_ctas"] == math.ceil(4096 / e.rings_per_cta)
    back = at.TuningTable.from_json(table.to_json())
    assert back.entries == table.entries and back.results == table.results
    for n in (700, 3000, 20000):
        assert back.shape_for(n) == table.shape_for(n)


def test_a_stored_shape_that_does_not_fit_falls_back_to_the_automatic_one():
    table = at.TuningTable([at.TableEntry("mixed", 65536, rings_per_thread=4, rings_per_cta=256)])
    assert table.shape_for(500) == {"rings_per_thread": 4, "cluster_ctas": 2}
    assert table.shape_for(5000) == {}        # 20 CTAs: more than a cluster holds
    small = at.TuningTable([at.TableEntry("mixed", 65536, rings_per_thread=4, rings_per_cta=64)])
    assert small.shape_for(500) == {}         # 8 CTAs of 32 threads x 4 rings would leave the last empty
    auto = at.TuningTable([at.TableEntry("mixed", 65536)])
    assert auto.shape_for(3000) == {}
    assert at.TuningTable().shape_for(3000) == {}
    one = at.TuningTable([at.TableEntry("fp64", 8192, block_threads=128)])
    assert one.shape_for(3000, "fp64") == {"block_threads": 128} and one.shape_for(3000, "mixed") == {}
    # mobile ions / RK4: a cluster stored as positions per block, a block size as one block
    ions = at.TuningTable([at.TableEntry("ions", 2048, block_threads=128), at.TableEntry("ions", 4096, rings_per_cta=1000)])
    assert ions.shape_for(1500, "ions") == {"block_threads": 128, "cluster_ctas": 1}
    assert ions.shape_for(3993, "ions") == {"cluster_ctas": 4}
    assert ions.shape_for(3993, "rk4") == {}
    res = at.SizeResult(6000, "rk4", [], at.Candidate(cluster_ctas=4, ctas=4))
    e = at.entry_from(res, 8192)
    assert (e.kind, e.rings_per_cta, e.block_threads) == ("rk4", 1500, 0)
    assert at.TuningTable([e]).shape_for(7905, "rk4") == {"cluster_ctas": 6}


class _FakeHandle:
    closed = 0

    def __init__(self, wake, shape):
        self.n, self.shape = wake.n_rings, dict(shape)

    def close(self):
        _FakeHandle.closed += 1


def _batch_model(fast_class_shape):
    """A batch's step time = its slowest wake's time; a wake of n rings
    takes n microseconds, half that in a shape `fast_class_shape` accepts
    if it has more than 3000 rings, 20 % more in any other explicit
    shape."""
    def run(handles):
        t = 0.0
        for h in handles:
            f = 1.0
            if h.shape:
                f = 0.5 if (h.n > 3000 and fast_class_shape(h.shape)) else 1.2
            t = max(t, 1e-6 * h.n * f)
        return t
    return run


def test_batch_tuning_keeps_what_shortens_the_step():
    from paper_2603_16623_gb300 import workloads as W
    wakes = [W.Wake(f"w{n}", W.edges_uniform(n, 6.0), [], 0.01, 100) for n in (600, 900, 2000, 3500, 3900, 7000)]
    _FakeHandle.closed = 0
    run = _batch_model(lambda s: s.get("rings_per_thread") == 8)
    table = at.tune_batch(wakes, sizes=(1024, 2048, 4096, 8192), make=_FakeHandle, run=run, max_candidates=4)
    by = {e.n_max: e for e in table.entries}
    # the 7000-ring wake sets the step: its class takes an 8-ring shape
    # (3.5 ms); the 3900-ring wake then sets it and its class takes one
    # too; the small classes gain nothing (their wakes never set the step)
    # and stay automatic
    assert by[wm.wake_max_rings("mixed")].rings_per_thread == 8
    assert by[4096].rings_per_thread == 8
    assert by[1024].rings_per_cta == 0 and by[2048].rings_per_cta == 0
    for wk in wakes:
        kw = table.shape_for(wk.n_rings)
        if kw:
            wm.wake_launch_shape(wk.n_rings, **kw)
    # every handle made was closed, and each class's trials are recorded
    assert _FakeHandle.closed >= len(wakes)
    assert {r["class_n_max"] for r in table.results} == {1024, 2048, 4096, wm.wake_max_rings("mixed")}
    assert all(r["tried"][0]["shape"] == "automatic" for r in table.results)


def test_batch_tuning_ignores_gains_below_the_noise():
    from paper_2603_16623_gb300 import workloads as W
    wakes = [W.Wake(f"w{n}", W.edges_uniform(n, 6.0), [], 0.01, 100) for n in (1500, 5000)]

    def run(handles):
        # explicit shapes are 1 % faster: within min_gain
        return max(1e-6 * h.n * (0.99 if h.shape else 1.0) for h in handles)
    table = at.tune_batch(wakes, sizes=(2048, 8192), make=_FakeHandle, run=run, min_gain=0.02)
    assert all(e.rings_per_cta == 0 for e in table.entries)


def test_batch_tuning_takes_only_on_chip_wakes():
    import dataclasses

    from paper_2603_16623_gb300 import workloads as W
    wk = W.Wake("w", W.edges_uniform(1000, 6.0), [], 0.01, 100)
    for bad in (dataclasses.replace(wk, ions=(1.0, 1836.0)), dataclasses.replace(wk, integrator="rk4"),
                dataclasses.replace(wk, grid_nr=16)):
        with pytest.raises(ValueError):
            at.tune_batch([wk, bad], sizes=(2048,), make=_FakeHandle, run=lambda hs: 1.0)
