"""Pins of the oracle's adaptive beam grids (orc_run with grid_nr > 0,
Sec. IV): per beam species a radial grid of grid_nr cells covering all its
particles, one node line per slice; B^(b) at the nodes from the slice's
enclosed charge, at the rings interpolated (B_N r_N / rho beyond the grid);
the plasma fields evaluated at the nodes and interpolated to the particles.

Against the gridless fields (a9) only smooth quantities converge: between
two rings d_rho psi runs a sawtooth of amplitude ~n d_rho / 2 (the rings'
discreteness), which the grid averages out, so W_r is not compared; E_z is
smooth and converges at second order in the grid spacing."""
import numpy as np
import pytest

import oracle
from paper_2603_16623_gb300 import workloads as W


def _linear_case(grid_nr, n_rings=3000, steps=600):
    drv = W.sampled_gaussian_beam(0.01, steps, 0.05, 0.5, 0.6, 2.4, n_r=512)
    return W.Wake("grid", W.edges_uniform(n_rings, 6.0), [drv], 0.01, steps, grid_nr=grid_nr)


def test_grid_ez_converges_at_second_order_in_the_grid_spacing():
    ref = oracle.run_wake(_linear_case(0), beam_fields=("ez",))
    errs = []
    for nr in (4, 8, 16):
        g = oracle.run_wake(_linear_case(nr), beam_fields=("ez",))
        assert g.status == 0
        errs.append(np.max(np.abs(g.beam["ez"] - ref.beam["ez"])) / np.max(np.abs(ref.beam["ez"])))
    q = [a / b for a, b in zip(errs, errs[1:])]
    assert all(3.5 < x < 4.5 for x in q), (errs, q)


def test_beam_field_beyond_the_grid_is_the_enclosed_charge():
    """At slice 0 the rings sit at their cell centres in both runs: beyond
    the grid's extent B_N r_N / rho is the field of all the slice's charge;
    inside it the grid's interpolation differs from the exact count."""
    drv = W.gaussian_beam(20_000, 1.0, 0.3, 0.3, 0.0, seed=11)
    e = W.edges_uniform(400, 5.0)
    a = oracle.run_wake(W.Wake("a", e, [drv], 0.01, 3), ring_dumps=("r", "bb"), beam_fields=())
    b = oracle.run_wake(W.Wake("b", e, [drv], 0.01, 3, grid_nr=16), ring_dumps=("r", "bb"), beam_fields=())
    R = np.max(drv.r) * (1 + 1 / 16)
    r0 = a.rings["r"][0]
    out = r0 >= R
    assert out.sum() > 100 and (~out).sum() > 10
    assert np.max(np.abs(b.rings["bb"][0][out] - a.rings["bb"][0][out]) / np.abs(a.rings["bb"][0][out])) < 1e-13
    assert np.max(np.abs(b.rings["bb"][0][~out] - a.rings["bb"][0][~out])) > 1e-6


def test_a_beam_split_into_two_identical_species_gives_the_same_fields():
    drv = W.gaussian_beam(8_000, 1.0, 0.3, 0.5, 1.5, seed=12)
    half = W.Beam(drv.xi, drv.r, 0.5 * drv.w, drv.q)
    e = W.edges_uniform(300, 5.0)
    one = oracle.run_wake(W.Wake("one", e, [drv], 0.01, 400, grid_nr=24), ring_dumps=("r",))
    two = oracle.run_wake(W.Wake("two", e, [half, half], 0.01, 400, grid_nr=24), ring_dumps=("r",))
    n = drv.n
    for k in ("ez", "wr", "bt", "psi"):
        f2 = two.beam[k]
        assert np.allclose(f2[:n], f2[n:], rtol=0, atol=0), k          # both halves alike
        den = np.max(np.abs(one.beam[k]))
        assert np.max(np.abs(f2[:n] - one.beam[k])) < 1e-12 * den, k
    assert np.max(np.abs(two.rings["r"] - one.rings["r"])) < 1e-12


def test_regular_grid_of_the_adaptive_extent_equals_the_adaptive_grid():
    """A fixed extent equal to the adaptive one (one species) gives the same
    wake bitwise: the extent is the only difference between the two."""
    drv = W.gaussian_beam(8_000, 1.0, 0.3, 0.5, 1.5, seed=13)
    e = W.edges_uniform(300, 5.0)
    ada = oracle.run_wake(W.Wake("a", e, [drv], 0.01, 300, grid_nr=20), ring_dumps=("r",))
    R = float(np.max(drv.r) * (1 + 1 / 20))
    reg = oracle.run_wake(W.Wake("r", e, [drv], 0.01, 300, grid_nr=20, grid_rmax=R), ring_dumps=("r",))
    assert np.array_equal(ada.rings["r"], reg.rings["r"]) and np.array_equal(ada.beam["ez"], reg.beam["ez"])


def test_regular_grid_ez_converges_at_second_order():
    """The regular intermediate grid over [0, 3] (the beam within it)."""
    ref = oracle.run_wake(_linear_case(0), beam_fields=("ez",))
    errs = []
    for nr in (8, 16, 32):
        wk = _linear_case(nr)
        g = oracle.run_wake(W.Wake(wk.name, wk.edges, wk.beams, wk.dxi, wk.n_steps, grid_nr=nr, grid_rmax=3.0),
                            beam_fields=("ez",))
        assert g.status == 0
        errs.append(np.max(np.abs(g.beam["ez"] - ref.beam["ez"])) / np.max(np.abs(ref.beam["ez"])))
    q = [a / b for a, b in zip(errs, errs[1:])]
    assert all(3.5 < x < 4.5 for x in q), (errs, q)


def test_regular_grid_refuses_a_beam_beyond_it():
    drv = W.gaussian_beam(2_000, 1.0, 0.5, 0.5, 0.6, seed=14)
    wk = W.Wake("out", W.edges_uniform(100, 5.0), [drv], 0.01, 100, grid_nr=8, grid_rmax=0.5)
    with pytest.raises(RuntimeError):
        oracle.run_wake(wk)


def test_grid_beam_field_converges_to_the_closed_form_on_each_species_grid():
    """With a negligible plasma (density 1e-9: B^(p) ~ 1e-9 of B^(b)) the
    B_theta a beam particle gathers through its species' grid is the beam
    field alone, and for a noise-free Gaussian slab (8192 radial quantile
    samples per slice) it converges at second order in the grid spacing to
    the closed form q N_slab (1 - exp(-r^2 / 2 sigma_r^2)) / (2 pi dxi r)
    (Gauss's law for the smooth slab).  A wide driver and a narrow witness
    (sigma_r 0.5 and 0.01, in separate xi ranges) each converge on their own
    grid; the witness could not on the driver's."""
    import math
    dxi, steps, n_r = 0.01, 400, 8192
    pars = [(0.5, 0.5, 0.15, 1.5), (20.0, 0.01, 0.15, 3.0)]   # n_b0, sigma_r, sigma_z, xi_c
    beams = [W.sampled_gaussian_beam(dxi, steps, *p, n_r=n_r) for p in pars]
    closed = []
    for b, (n_b0, sr, sz, xc) in zip(beams, pars):
        slab = n_b0 * np.exp(-0.5 * ((b.xi - xc) / sz) ** 2) * 2 * math.pi * sr ** 2 * dxi
        closed.append(b.q * slab * (1 - np.exp(-b.r ** 2 / (2 * sr ** 2))) / (2 * math.pi * dxi * b.r))
    n0 = beams[0].n
    errs = {"driver": [], "witness": []}
    for nr in (8, 16, 32, 64):
        g = oracle.run_wake(W.Wake("slab", W.edges_uniform(300, 5.0), beams, dxi, steps, density=1e-9, grid_nr=nr),
                            beam_fields=("bt",))
        assert g.status == 0
        for name, got, ref in (("driver", g.beam["bt"][:n0], closed[0]), ("witness", g.beam["bt"][n0:], closed[1])):
            errs[name].append(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    for name, e in errs.items():
        q = [a / b for a, b in zip(e, e[1:])]
        assert all(x > 3.3 for x in q) and e[-1] < 1e-3, (name, e, q)
