"""wake_fields_at_static, the entry point that allocates nothing, against
wake_fields_at on the same wake at the same slice.

Named to be collected last: it must pass alone and after every other GPU
test (the library's static scratch then already holds values of earlier
calls, which no call may return).
"""
import numpy as np
import pytest

from paper_2603_16623_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# the parity tests' tolerances (norm-wise, per field)
TOL = {"fp64": 1e-10, "mixed": 1e-5}
FIELDS = ("ez", "wr", "bt", "psi")


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


def _wake(n_rings, precision, steps=300):
    from paper_2603_16623_gb300 import wake as wm
    drv = W.gaussian_beam(40_000, 1.0, 0.3, 0.5, 1.5, seed=n_rings)
    wk = W.Wake(f"noalloc{n_rings}", W.edges_uniform(n_rings, 6.0), [drv], 0.01, steps)
    return wm.Wake.from_workload(wk, precision=precision)


def _queries(n, seed, r_max=6.5):
    rng = np.random.default_rng(seed)
    return np.concatenate([[0.0, 1e-5], np.sort(rng.uniform(0.0, r_max, n - 2))])


# 700 rings: one CTA; 3000 rings (mixed): a two-CTA thread-block cluster
@pytest.mark.parametrize("precision,n_rings", [("fp64", 700), ("mixed", 700), ("mixed", 3000)])
def test_static_entry_matches_fields_at_on_two_calls_in_a_row(precision, n_rings):
    g = _wake(n_rings, precision)
    g.step_slices(180)
    r1, r2 = _queries(5000, 1), _queries(1234, 2)
    ref1, ref2 = g.fields_at(r1), g.fields_at(r2)
    got1 = g.fields_at_static(r1)
    got2 = g.fields_at_static(r2)
    for k in FIELDS:
        assert nerr(got1[k], ref1[k]) < TOL[precision], ("first call", k)
        assert nerr(got2[k], ref2[k]) < TOL[precision], ("second call", k)
    # the ring state is not advanced by either entry point
    assert g.progress()[0] == 180
    g.close()


def test_static_entry_at_its_size_limit_and_beyond():
    from paper_2603_16623_gb300 import wake as wm
    g = _wake(500, "mixed", steps=100)
    g.step_slices(60)
    r = _queries(wm.WAKE_STATIC_MAX_QUERIES, 3)
    ref = g.fields_at(r)
    got = g.fields_at_static(r)
    for k in FIELDS:
        assert nerr(got[k], ref[k]) < TOL["mixed"], k
    with pytest.raises(wm.WakeError) as ei:
        g.fields_at_static(_queries(wm.WAKE_STATIC_MAX_QUERIES + 1, 4))
    assert ei.value.status == wm.WAKE_EINVAL
    assert "static scratch limit" in str(ei.value)
    # an empty call does only the set-up and succeeds
    out = g.fields_at_static(np.zeros(0))
    assert all(v.shape == (0,) for v in out.values())
    g.close()
