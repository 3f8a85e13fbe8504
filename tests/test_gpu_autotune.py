"""The launch-shape autotuner on the GPU: it times real batched marches of
each candidate shape, the table it builds gives wakes the shape it chose,
a wake in a tuned shape still matches the oracle, and the serving loop
creates its wakes in the table's shapes (bitwise the result of a wake
created alone in that shape)."""
import numpy as np
import pytest

import oracle
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
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_tuning_times_every_candidate_and_the_table_applies_the_choice():
    from paper_2603_16623_gb300 import autotune as at
    from paper_2603_16623_gb300 import wake as wm
    table = at.tune((1500, 4000), "mixed", max_candidates=3, slices=60, fill=1.0)
    assert len(table.results) == 2
    for res in table.results:
        assert len(res["rates"]) == len(at.candidates(res["n_rings"], "mixed", 3))
        assert all(r["ring_slices_per_s"] > 1e6 for r in res["rates"])
        n = res["n_rings"]
        ch = res["chosen"]
        wk = at.probe_wake(n, 20)
        g = wm.Wake.from_workload(wk, precision="mixed", **table.shape_for(n))
        t, k, cl = g.launch_config()
        assert (t, cl) == (ch["threads"], ch["ctas"])
        g.close()
    fp = at.tune((1000,), "fp64", slices=40, fill=0.5)
    assert len(fp.results[0]["rates"]) == 4 and all(r["ring_slices_per_s"] > 1e5 for r in fp.results[0]["rates"])


def test_a_tuned_shape_matches_the_oracle():
    """A table that forces 8 rings per thread and 768 rings per CTA (not an
    automatic shape) on a 3000-ring wake: ring radii and E_z over 300
    slices within the mixed tolerance."""
    from paper_2603_16623_gb300 import autotune as at
    from paper_2603_16623_gb300 import wake as wm
    table = at.TuningTable([at.TableEntry("mixed", 65536, rings_per_thread=8, rings_per_cta=768)])
    kw = table.shape_for(3000)
    assert kw == {"rings_per_thread": 8, "cluster_ctas": 4}
    drv = W.gaussian_beam(40_000, 1.0, 0.6, 0.6, 2.4, seed=3000)
    wk = W.Wake("tuned", W.edges_uniform(3000, 6.0), [drv], 0.01, 300)
    ref = oracle.run_wake(wk, ring_dumps=("r",))
    g = wm.Wake.from_workload(wk, precision="mixed", flags=wm.WAKE_DUMP_RING_R, **kw)
    assert g.launch_config() == (96, 8, 4)
    st, _, _, _ = g.run()
    assert st == 0
    assert nerr(g.ring_dumps(which=("r",))["r"], ref.rings["r"]) < 1e-5
    assert nerr(g.beam_fields(("ez",))["ez"], ref.beam["ez"]) < 1e-5
    g.close()


def test_the_server_creates_wakes_in_the_table_shapes():
    from paper_2603_16623_gb300 import autotune as at
    from paper_2603_16623_gb300 import serve
    from paper_2603_16623_gb300 import wake as wm
    table = at.TuningTable([at.TableEntry("mixed", 65536, rings_per_thread=8, rings_per_cta=512)])
    wakes = []
    for k, (n, steps) in enumerate(((900, 200), (2600, 150), (1500, 120))):
        drv = W.gaussian_beam(10_000, 2.0, 0.3, 0.5, 1.6, seed=900 + k)
        wakes.append(W.Wake(f"t{k}", W.edges_uniform(n, 6.0), [drv], 0.01, steps))
    alone = []
    for wk in wakes:
        kw = table.shape_for(wk.n_rings)
        assert kw and wm.wake_launch_shape(wk.n_rings, **kw) != wm.wake_launch_shape(wk.n_rings)
        g = wm.Wake.from_workload(wk, precision="mixed", **kw)
        g.step_slices(wk.n_steps)
        alone.append(g.beam_fields(("ez",))["ez"])
        g.close()
    reqs = [serve.Request(rid=i, arrival=0.0, edges=wk.edges, beams=wk.beams, dxi=wk.dxi, n_steps=wk.n_steps,
                          out_ez=np.zeros(wk.n_beam, np.float32)) for i, wk in enumerate(wakes)]
    srv = serve.WakeServer(1 << 34, step_ns=200_000, tuning=table)
    stats = serve.run_stream(srv, reqs)
    assert len(stats.completed) == len(wakes)
    for req, ez in zip(reqs, alone):
        assert req.status == 0
        assert np.array_equal(req.out_ez, ez), req.rid


def test_batch_tuning_on_the_batch_step_time():
    """tune_batch on a small batch of uneven wakes: every class's trials
    are real batched solves, and the table it returns gives shapes the
    library takes for every wake of the batch."""
    from paper_2603_16623_gb300 import autotune as at
    from paper_2603_16623_gb300 import wake as wm
    wakes = []
    for k, (n, nb0) in enumerate(((700, 2.0), (1800, 4.0), (3000, 6.0), (5200, 3.0))):
        drv = W.gaussian_beam(30_000, nb0, 0.4, 0.5, 2.0, seed=1200 + k)
        wakes.append(W.Wake(f"b{k}", W.edges_uniform(n, 6.0), [drv], 0.01, 300))
    table = at.tune_batch(wakes, sizes=(1024, 8192), max_candidates=3, repeats=1)
    assert len(table.results) == 2
    for r in table.results:
        assert len(r["tried"]) >= 2 and all(t["step_s"] > 0 for t in r["tried"])
    for wk in wakes:
        g = wm.Wake.from_workload(wk, precision="mixed", **table.shape_for(wk.n_rings))
        st, _, _, _ = g.run()
        assert st == 0
        g.close()
