"""Pins of the oracle's mobile ions (orc_run_ions): ions as a second ring
species, each species solved on its own rings and gathered into the other by
linear interpolation (Sec. II, multiple plasma species), B_theta^(p) from the
electrons only, ions moving with q/m = Z/M.  Each pin comes from physics or
from a limit, not from the oracle's own formulas:

- an unperturbed two-species plasma has no field anywhere and stays put;
- infinitely heavy ions reproduce the immobile ion column, converging at
  second order in the ring spacing (linear interpolation of the uniform
  column's linear d_rho psi is exact; its quadratic psi is not), and so do
  the fields on the beam particles and the B^(p) at the ion rings;
- the Lorentz force integrated along the ion trajectories gives the
  algebraic u_z of the ions' own cold-plasma constant (q/m = Z/M);
- the model depends on Z and M only through Z/M (neutrality fixes the ion
  charge density), and the ions' weak response scales as Z/M;
- a dense electron beam pulls the ions inside it towards the axis."""
import numpy as np
import pytest

import oracle
from paper_2603_16623_gb300 import workloads as W


def _drv(nb0, sig_r=0.4, seed=3):
    return W.gaussian_beam(20_000, nb0, sig_r, 0.6, 1.6, seed=seed)


@pytest.mark.parametrize("ions", [(1.0, 1836.0), (2.0, 50.0)])
def test_unperturbed_two_species_plasma_has_no_field(ions):
    e = W.edges_refined(40, 0.5, 60, 4.0)
    res = oracle.run(e, [], [], [], 0.05, 60, ions=ions,
                     ring_dumps=("r", "psi", "dpsidr", "dpsidz", "bp"))
    assert res.status == 0 and res.slices_run == 60
    for k in ("psi", "dpsidr", "dpsidz", "bp"):
        assert np.max(np.abs(res.rings[k])) == 0.0, k
    assert np.array_equal(res.final_r, res.rings["r"][0])


def test_heavy_ions_converge_to_the_immobile_column_at_second_order():
    drv = _drv(0.5)
    errs = []
    for n in (50, 100, 200, 400):
        mob = oracle.run_wake(W.Wake("m", W.edges_uniform(n, 5.0), [drv], 0.02, 200, ions=(1.0, 1e12)),
                              ring_dumps=("r", "dpsidr"), beam_fields=())
        col = oracle.run_wake(W.Wake("c", W.edges_uniform(n, 5.0), [drv], 0.02, 200),
                              ring_dumps=("r", "dpsidr"), beam_fields=())
        assert mob.status == col.status == 0
        # the ions have not moved
        assert np.max(np.abs(mob.final_r[n:] - mob.rings["r"][0][n:])) < 1e-11
        errs.append(np.max(np.abs(mob.rings["r"][:, :n] - col.rings["r"])))
    ratios = [a / b for a, b in zip(errs, errs[1:])]
    assert all(q > 3.5 for q in ratios), (errs, ratios)
    assert errs[-1] < 5e-5


@pytest.mark.parametrize("q,r_max", [(-1.0, 5.0), (+1.0, 2.0)])
def test_heavy_ions_give_the_column_fields_on_beam_particles_and_ion_rings(q, r_max):
    """With infinitely heavy ions, what the beam particles see (the exact
    sums of both species) and the B^(p) the ion rings see (the electrons'
    field interpolated) converge to the immobile column's, the latter taken
    from the column's own slice solve at the ion radii: psi on the beam at
    second order in the ring spacing, the rest at first (a particle or an
    ion ring between rings sees a staircase of enclosed charge and B^(p)
    jumps across each electron ring).  Errors relative to the column's
    largest value, over three halvings of the spacing (first order: 8x).
    A positron driver in a narrow column draws the outermost electrons in,
    so that the outermost ion rings take B^(p) from beyond the last
    electron ring."""
    drv = W.gaussian_beam(20_000, 0.5, 0.4, 0.6, 1.6, seed=3, q=q)
    dxi, steps = 0.02, 200
    sl = np.floor(drv.xi / dxi + 0.5)
    errs = {k: [] for k in ("ion_bp", "ez", "bt", "wr", "psi")}
    for n in (50, 100, 200, 400):
        edges = W.edges_uniform(n, r_max)
        mob = oracle.run_wake(W.Wake("m", edges, [drv], dxi, steps, ions=(1.0, 1e12)), ring_dumps=("r", "bp"),
                              beam_fields=("ez", "wr", "bt", "psi"))
        col = oracle.run_wake(W.Wake("c", edges, [drv], dxi, steps), ring_dumps=("r", "ur"),
                              beam_fields=("ez", "wr", "bt", "psi"))
        assert mob.status == col.status == 0
        _, _, w, wh = oracle.ring_init(edges)
        e = scale = 0.0
        for s in range(10, steps, 20):
            m = sl == s
            sf = oracle.slice_fields(col.rings["r"][s], col.rings["ur"][s], w, wh, 1.0, r_max, drv.r[m],
                                     drv.q * drv.w[m], dxi, rq=mob.rings["r"][s, n:])
            e = max(e, np.max(np.abs(mob.rings["bp"][s, n:] - sf["q_bp"])))
            scale = max(scale, np.max(np.abs(sf["q_bp"])))
        errs["ion_bp"].append(e / scale)
        if q > 0:
            beyond = np.max(mob.rings["r"][:, n:], axis=1) > np.max(mob.rings["r"][:, :n], axis=1)
            assert beyond.sum() > steps // 2
        for k in ("ez", "bt", "wr", "psi"):
            errs[k].append(np.max(np.abs(mob.beam[k] - col.beam[k])) / np.max(np.abs(col.beam[k])))
    gain = {k: v[0] / v[-1] for k, v in errs.items()}
    assert gain["psi"] > 40 and errs["psi"][-1] < 1e-3, errs
    for k, (g, last) in {"ion_bp": (5, 0.02), "ez": (5, 0.01), "bt": (5, 0.01), "wr": (4, 0.2)}.items():
        assert gain[k] > g and errs[k][-1] < last, (k, errs[k])
        assert all(a > b for a, b in zip(errs[k], errs[k][1:])), (k, errs[k])


def _lorentz_residual(n, dxi, M):
    drv = _drv(6.0, sig_r=0.3)
    wk = W.Wake("l", W.edges_uniform(n, 4.0), [drv], dxi, int(round(6.0 / dxi)), ions=(1.0, M))
    res = oracle.run_wake(wk, beam_fields=(),
                          ring_dumps=("ur", "psibar", "uz", "gamma", "dpsidz", "bp", "bb"))
    assert res.status == 0
    R = res.rings
    ions = slice(n, 2 * n)
    qm = 1.0 / M
    # du_z/dxi = (q/m)(gamma E_z + u_r B_theta)/psibar with E_z = -d_zeta psi
    f = qm * (R["gamma"][:, ions] * (-R["dpsidz"][:, ions])
              + R["ur"][:, ions] * (R["bp"][:, ions] + R["bb"][:, ions])) / R["psibar"][:, ions]
    uz = R["uz"][0][None, ions] + np.concatenate(
        [np.zeros((1, n)), np.cumsum(0.5 * (f[1:] + f[:-1]) * dxi, axis=0)])
    return np.max(np.abs(uz - R["uz"][:, ions])), np.max(np.abs(R["uz"][:, ions]))


def test_ion_lorentz_force_integration_matches_algebraic_uz():
    """The interpolated fields are consistent with the interpolated psi only
    to O(d rho), so the residual falls as both the ring spacing and d xi
    are refined."""
    errs = []
    for n, dxi in ((100, 0.02), (200, 0.01), (400, 0.005)):
        e, scale = _lorentz_residual(n, dxi, 20.0)
        errs.append(e / scale)
    assert errs[0] / errs[1] > 2.0 and errs[1] / errs[2] > 2.0, errs
    assert errs[-1] < 5e-4, errs


def test_model_depends_on_ion_charge_and_mass_only_through_z_over_m():
    drv = _drv(3.0, sig_r=0.3)
    a = oracle.run_wake(W.Wake("a", W.edges_uniform(120, 4.0), [drv], 0.01, 400, ions=(1.0, 25.0)),
                        ring_dumps=("r", "ur"))
    b = oracle.run_wake(W.Wake("b", W.edges_uniform(120, 4.0), [drv], 0.01, 400, ions=(2.0, 50.0)),
                        ring_dumps=("r", "ur"))
    assert a.status == b.status == 0
    assert np.array_equal(a.rings["r"], b.rings["r"]) and np.array_equal(a.beam["ez"], b.beam["ez"])


def test_weak_ion_response_scales_with_z_over_m():
    drv = _drv(2.0, sig_r=0.3)
    disp = []
    for M in (4000.0, 8000.0):
        res = oracle.run_wake(W.Wake("s", W.edges_uniform(150, 4.0), [drv], 0.01, 500, ions=(1.0, M)),
                              ring_dumps=("r",), beam_fields=())
        assert res.status == 0
        disp.append(res.final_r[150:] - res.rings["r"][0][150:])
    # displacement ~ (Z/M) x (a fixed electron wake) + O((Z/M)^2)
    ratio = np.max(np.abs(disp[0])) / np.max(np.abs(disp[1]))
    assert abs(ratio - 2.0) < 0.02, ratio
    assert np.max(np.abs(disp[0] - 2.0 * disp[1])) < 0.02 * np.max(np.abs(disp[0]))


def test_dense_electron_beam_pulls_ions_inward():
    """Inside a dense electron driver the beam's own radial field points
    to the axis (for positive ions: E_r < 0 inside a negative column) and
    outweighs the ion channel's field: the ions within it gain u_r < 0."""
    drv = _drv(20.0, sig_r=0.15)
    n = 200
    res = oracle.run_wake(W.Wake("p", W.edges_uniform(n, 3.0), [drv], 0.01, 300, ions=(1.0, 100.0)),
                          ring_dumps=("r", "ur"), beam_fields=())
    assert res.status == 0
    r0 = res.rings["r"][0][n:]
    inside = r0 < 0.2
    ur_ions = res.final_ur[n:]
    assert inside.sum() > 5
    assert np.all(ur_ions[inside] < 0.0)
    assert np.all(res.final_r[n:][inside] < r0[inside])


# --------------------------------------------------------------------------
# radial density profiles (Sec. II: arbitrary profiles, carried by the rings
# of both species; ion rings of infinite mass stand still)
# --------------------------------------------------------------------------
def test_unperturbed_profiled_plasma_has_no_field():
    e = W.edges_refined(50, 1.0, 70, 6.0)
    prof = W.parabolic_profile(e, 1.0, 3.0)
    for ions in ((1.0, float("inf")), (1.0, 1836.0)):
        res = oracle.run(e, [], [], [], 0.05, 40, ions=ions, cell_density=prof,
                         ring_dumps=("r", "psi", "dpsidr", "dpsidz", "bp"))
        assert res.status == 0
        for k in ("psi", "dpsidr", "dpsidz", "bp"):
            assert np.max(np.abs(res.rings[k])) == 0.0, k
        assert np.array_equal(res.final_r, res.rings["r"][0])


def test_uniform_profile_equals_the_scalar_density():
    drv = _drv(1.0)
    e = W.edges_uniform(120, 4.0)
    a = oracle.run_wake(W.Wake("a", e, [drv], 0.01, 300, density=2.5, ions=(1.0, 100.0)), ring_dumps=("r",))
    b = oracle.run_wake(W.Wake("b", e, [drv], 0.01, 300, density=1.0, ions=(1.0, 100.0),
                               cell_density=np.full(120, 2.5)), ring_dumps=("r",))
    assert np.array_equal(a.rings["r"], b.rings["r"]) and np.array_equal(a.beam["ez"], b.beam["ez"])


def test_rings_oscillate_at_the_local_plasma_frequency():
    """A weak, wide, short driver kicks the rings of a parabolic channel
    n = 1 + r^2/16 (static ion rings); afterwards each ring oscillates at
    the local plasma frequency sqrt(n(rho)) (its displacement delta moves
    the enclosed ion charge by n rho delta: E_r = n delta)."""
    n = 200
    e = W.edges_uniform(n, 8.0)
    c = 0.5 * (e[1:] + e[:-1])
    prof = 1.0 + 4.0 * c * c / 64.0
    drv = W.gaussian_beam(40_000, 0.002, 6.0, 0.3, 1.0, seed=5)
    res = oracle.run_wake(W.Wake("osc", e, [drv], 0.01, 3000, ions=(1.0, float("inf")), cell_density=prof),
                          ring_dumps=("r",), beam_fields=())
    assert res.status == 0
    r = res.rings["r"]
    omegas, local = [], []
    for j in range(10, n - 10, 30):
        d = r[300:, j] - r[0, j]
        d = d - d.mean()
        f = np.abs(np.fft.rfft(d * np.hanning(d.shape[0])))
        k = int(np.argmax(f[1:])) + 1
        kk = k + 0.5 * (f[k - 1] - f[k + 1]) / (f[k - 1] - 2 * f[k] + f[k + 1])
        omegas.append(2 * np.pi * kk / (d.shape[0] * 0.01))
        local.append(np.sqrt(prof[j]))
    omegas, local = np.array(omegas), np.array(local)
    assert np.all(np.abs(omegas / local - 1.0) < 0.05), (omegas, local)
    assert np.all(np.diff(omegas) > 0)
