"""The seeded input generators (paper_2603_16623_gb300/workloads.py)
against the input recipe they implement: Gaussian bunch charge by
quadrature, the radial and longitudinal distributions of the drawn beams,
the noise-free sampled slabs, the ring-cell edges of the workloads, and the
parameter ranges of the batched members.  No method arithmetic here: these
are the inputs both the CUDA path and the oracle start from."""
import math

import numpy as np
import pytest

from paper_2603_16623_gb300 import workloads as W


@pytest.mark.parametrize("n_b0,sr,sz", [(0.05, 0.5, 1.0), (10.0, 0.1, 0.5), (3.0, 1.2, 0.3)])
def test_gaussian_charge_is_the_truncated_bunch_integral(n_b0, sr, sz):
    from scipy import integrate
    radial, _ = integrate.quad(lambda r: 2 * math.pi * r * math.exp(-r * r / (2 * sr * sr)), 0, 40 * sr)
    axial, _ = integrate.quad(lambda z: math.exp(-z * z / (2 * sz * sz)), -4 * sz, 4 * sz)
    assert abs(W.gaussian_charge(n_b0, sr, sz) - n_b0 * radial * axial) < 1e-10 * n_b0 * radial * axial


def test_gaussian_beam_is_seeded_round_and_truncated():
    a = W.gaussian_beam(200_000, 2.0, 0.4, 0.7, 3.0, seed=7)
    b = W.gaussian_beam(200_000, 2.0, 0.4, 0.7, 3.0, seed=7)
    assert np.array_equal(a.xi, b.xi) and np.array_equal(a.r, b.r)
    assert np.all(np.abs(a.xi - 3.0) <= 4 * 0.7) and np.all(a.r >= 0)
    # 2-D Gaussian of rms 0.4 per axis: mean radius sigma sqrt(pi/2), mean r^2 = 2 sigma^2
    assert abs(a.r.mean() - 0.4 * math.sqrt(math.pi / 2)) < 3e-3
    assert abs(np.mean(a.r ** 2) - 2 * 0.16) < 3e-3
    # truncated normal in xi: standard deviation sigma_z x 0.9986 (4-sigma truncation)
    assert abs(a.xi.std() - 0.7 * 0.99858) < 3e-3
    assert abs(a.w.sum() - W.gaussian_charge(2.0, 0.4, 0.7)) < 1e-9 * a.w.sum()
    assert a.q == -1.0 and np.all(a.w == a.w[0])


def test_sampled_slab_carries_the_slab_charge_at_radial_quantiles():
    dxi, n_r = 0.01, 128
    b = W.sampled_gaussian_beam(dxi, 500, 1.5, 0.3, 0.4, 2.0, n_r=n_r)
    sl = np.round(b.xi / dxi).astype(int)
    for s in (150, 200, 230):
        m = sl == s
        assert m.sum() == n_r
        expect = 1.5 * math.exp(-0.5 * ((s * dxi - 2.0) / 0.4) ** 2) * 2 * math.pi * 0.09 * dxi
        assert abs(b.w[m].sum() - expect) < 1e-12 * expect
        # the radii are the quantiles (j + 1/2) / n_r of 1 - exp(-r^2 / 2 sigma^2)
        cdf = 1 - np.exp(-np.sort(b.r[m]) ** 2 / (2 * 0.09))
        assert np.allclose(cdf, (np.arange(n_r) + 0.5) / n_r, rtol=0, atol=1e-12)
    assert np.all(np.abs(np.unique(sl) * dxi - 2.0) <= 4 * 0.4 + 1e-12)


def test_workload_edges():
    e = W.blowout_wake().edges
    assert e.shape[0] == 2001 and e[0] == 0.0 and abs(e[-1] - 6.0) < 1e-15
    d = np.diff(e)
    assert np.allclose(d[:288], 0.05 / 288) and np.allclose(d[288:], 5.95 / 1712)
    assert abs(d[288] / d[0] - 20.0) < 0.05   # x20 refinement (20.02 with these integer cell counts)
    g = W.large_wake(n_steps=10, n_drv=10, n_wit=10).edges
    assert g.shape[0] == 65537 and g[0] == 0.0 and abs(g[1] - 1e-5) < 1e-20 and abs(g[-1] - 6.0) < 1e-12
    assert np.all(np.diff(g) > 0)
    assert np.allclose(np.diff(np.log(g[1:])), math.log(6.0 / 1e-5) / 65535)
    lw = W.linear_wake()
    assert lw.n_rings == 200 and lw.edges[-1] == 5.0 and lw.dxi == 0.02 and lw.n_steps == 1000
    assert lw.beams[0].n == 20_000


def test_blowout_witness_carries_0_42_of_the_driver_charge():
    wk = W.blowout_wake(n_drv=20_000, n_wit=5_000)
    drv, wit = wk.beams
    assert abs(wit.w.sum() / drv.w.sum() - 0.42) < 1e-12
    assert abs(np.mean(wit.xi) - 5.0) < 0.02 and abs(np.mean(drv.xi) - 2.0) < 0.02
    assert wk.dxi == 0.005 and wk.n_steps == 4000


def test_batched_members_span_the_stated_ranges():
    ps = [W.batched_params(k) for k in range(256)]
    n = np.array([p.n_rings for p in ps])
    assert n.min() >= 500 and n.max() <= 8000
    # log-uniform: the median near sqrt(500 x 8000) = 2000
    assert 1500 < np.median(n) < 2700
    for p in ps:
        assert 0.05 <= p.n_b0 <= 20 and 0.05 <= p.sigma_r <= 1 and 0.3 <= p.sigma_z <= 2
        assert 50_000 <= p.n_mp <= 500_000 and 1000 <= p.n_steps <= 6000
        assert p.r_max == max(6.0, 6.0 * math.sqrt(p.n_b0) * p.sigma_r)
    wk = W.batched_wake(11)
    p = ps[11]
    assert wk.dxi == 0.01 and abs(np.mean(wk.beams[0].xi) - 4 * p.sigma_z) < 0.05 * p.sigma_z
