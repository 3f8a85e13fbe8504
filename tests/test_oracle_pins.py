"""Pins of the FP64 oracle to facts other than its own formulas.

Each test checks the oracle against something the paper or the mathematics
fixes independently of how the oracle computes it: the ODE and boundary
conditions that define psi (Eq. phi_b_eq_1 integrated, Eq. dpsi_dr/psi),
finite differences of psi along the ring motion (Eq. dpsi_dzeta), the jump
conditions behind Eq. ai_bi solved by dense elimination, Ampere's law
(Eq. maxwell_qsa_4), Lorentz-force integration of u_z against the constant of
motion (Eqs. cold_plasma_constant, plasma_particle_motion_3), the linear
closed form, and convergence orders.  A dropped term, wrong sign, wrong index
or transposed operand in the oracle fails at least one of these.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_16623_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _random_state(n=40, seed=11, r_max=3.0, u_scale=0.3, density=1.0):
    edges, rho, ur = W.random_ring_state(n, seed, r_max=r_max, u_scale=u_scale)
    _, _, w, wh = oracle.ring_init(edges, density)
    return edges, rho, ur, w, wh


def _nerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _between_ring_points(rho, n_per_gap=3, rmin=1e-3):
    rs = np.sort(rho)
    pts = []
    for lo, hi in zip(rs[:-1], rs[1:]):
        for f in np.linspace(0.2, 0.8, n_per_gap):
            pts.append(lo + f * (hi - lo))
    pts.append(0.5 * rs[0])
    return np.array([p for p in pts if p > rmin])


# --------------------------------------------------------------------------
# psi and d_rho psi: the ODE, jumps and boundary conditions that define them
# --------------------------------------------------------------------------
@pytest.mark.parametrize("density", [1.0, 2.5])
def test_psi_solves_poisson_with_ring_jumps(density):
    """Between rings (1/rho) d(rho d psi)/drho = -n (ion column) or 0 outside
    it; rho d psi/drho jumps by w_j at ring j; psi and d psi/drho vanish
    outside the neutral column; rho d psi/drho -> 0 on the axis."""
    edges, rho, ur, w, wh = _random_state(density=density)
    r_max = edges[-1]
    x = _between_ring_points(rho)
    h = 1e-6 * np.minimum(1.0, x)
    sf = oracle.slice_fields(rho, ur, w, wh, density, r_max, rq=np.concatenate([x - h, x, x + h]))
    m = x.shape[0]
    psi_m, psi_0, psi_p = sf["q_psi"][:m], sf["q_psi"][m:2 * m], sf["q_psi"][2 * m:]
    dpr_m, dpr_0, dpr_p = sf["q_dpsidr"][:m], sf["q_dpsidr"][m:2 * m], sf["q_dpsidr"][2 * m:]
    # d psi / d rho by central difference
    fd = (psi_p - psi_m) / (2 * h)
    assert np.max(np.abs(fd - dpr_0)) < 1e-6 * max(1.0, np.max(np.abs(dpr_0)))
    # Poisson operator between rings
    lap = ((x + h) * dpr_p - (x - h) * dpr_m) / (2 * h * x)
    src = np.where(x < r_max, -density, 0.0)
    assert np.max(np.abs(lap - src)) < 1e-5 * density
    # jumps of rho d psi/drho across each ring equal its weight
    eps = 1e-9
    sj = oracle.slice_fields(rho, ur, w, wh, density, r_max,
                             rq=np.concatenate([rho * (1 - eps), rho * (1 + eps)]))
    n = rho.shape[0]
    jump = rho * (1 + eps) * sj["q_dpsidr"][n:] - rho * (1 - eps) * sj["q_dpsidr"][:n]
    # ion charge in the shell [rho(1-eps), rho(1+eps)] inside the column
    ion_jump = np.where(rho < r_max, 2.0 * density * rho ** 2 * eps, 0.0)
    assert np.allclose(jump + ion_jump, w, rtol=1e-6, atol=1e-10)
    # outside everything: neutral, psi and its gradient vanish
    far = np.array([1.01, 2.0, 10.0]) * max(r_max, rho.max())
    sf_far = oracle.slice_fields(rho, ur, w, wh, density, r_max, rq=far)
    assert np.max(np.abs(sf_far["q_psi"])) < 1e-12 * density * r_max ** 2
    assert np.max(np.abs(sf_far["q_dpsidr"])) < 1e-12 * density * r_max
    # regular on the axis
    near = np.array([1e-9, 1e-7])
    sf_ax = oracle.slice_fields(rho, ur, w, wh, density, r_max, rq=near)
    assert np.all(np.abs(near * sf_ax["q_dpsidr"]) < 1e-12)


def test_psi_is_minus_integral_of_gauss_field():
    """psi(rho) = -int_rho^inf d psi/drho, with d psi/drho from Gauss's law
    (enclosed electron minus ion charge over rho), by adaptive quadrature."""
    from scipy import integrate
    edges, rho, ur, w, wh = _random_state(n=12, seed=5)
    r_max = edges[-1]

    def gauss(x):
        return (np.sum(w[rho < x]) - 0.5 * min(x, r_max) ** 2) / x

    top = max(r_max, rho.max())
    brk = sorted(set(list(rho) + [r_max]))
    x = np.array([0.3, 0.9, 1.7, 2.4])
    sf = oracle.slice_fields(rho, ur, w, wh, 1.0, r_max, rq=x)
    for xi, psi in zip(x, sf["q_psi"]):
        pts = [p for p in brk if xi < p < top]
        val, _ = integrate.quad(gauss, xi, top, points=pts or None, limit=400,
                                epsabs=1e-13, epsrel=1e-12)
        assert abs(-val - psi) < 1e-10


@pytest.mark.parametrize("edges", [W.edges_uniform(200, 5.0),
                                   W.edges_refined(288, 0.05, 1712, 6.0),
                                   W.edges_geometric(3000, 1e-5, 6.0)],
                         ids=["uniform", "refined", "geometric"])
def test_unperturbed_plasma_has_no_radial_field_at_rings(edges):
    """A uniform neutral plasma at rest: the self weight makes the enclosed
    electron charge at each ring equal the ion charge, so d psi/drho = 0 at
    every ring (Gauss), for any spacing; d psi/dzeta = 0 (no motion)."""
    rho0, _, w, wh = oracle.ring_init(edges)
    sf = oracle.slice_fields(rho0, np.zeros_like(rho0), w, wh, 1.0, edges[-1])
    scale = edges[-1]
    assert np.max(np.abs(sf["dpsidr"])) < 5e-13 * scale
    assert np.max(np.abs(sf["dpsidz"])) == 0.0
    # total electron charge equals the ion column's
    assert abs(w.sum() - 0.5 * edges[-1] ** 2) < 1e-12 * edges[-1] ** 2


def test_unperturbed_offset_is_second_order_in_ring_spacing():
    """Discrete rings against a continuous ion column leave psi = O(drho^2)
    at the rings, which drives an O(drho^2) response of the plasma at rest:
    halving the spacing cuts every spurious field by ~4."""
    res = []
    for n in (100, 200, 400):
        edges = W.edges_uniform(n, 5.0)
        steps = 500
        pxi = np.arange(steps) * 0.02
        out = oracle.run(edges, pxi, np.zeros(steps), np.zeros(steps), 0.02, steps,
                         beam_fields=("ez",), ring_dumps=("r", "psi"))
        r = out.rings["r"]
        res.append((np.abs(out.rings["psi"][0]).max(), np.abs(out.beam["ez"]).max(),
                    np.abs(r - r[0]).max()))
    res = np.array(res)
    ratio = res[:-1] / res[1:]
    assert np.all(ratio > 3.3) and np.all(ratio < 4.7), ratio


# --------------------------------------------------------------------------
# d_zeta psi: finite difference along the ring motion
# --------------------------------------------------------------------------
def test_dzeta_psi_matches_finite_difference_of_psi():
    """Moving every ring by d rho/d zeta = -u/psibar (Eq. plasma_particle_motion_2)
    and differencing psi at fixed rho reproduces d psi/d zeta (pins the sign
    reading of Eq. dpsi_dzeta)."""
    edges, rho, ur, w, wh = _random_state(n=40, seed=3)
    x = _between_ring_points(rho, n_per_gap=2)
    sf = oracle.slice_fields(rho, ur, w, wh, 1.0, edges[-1], rq=x)
    errs = []
    for eps in (1e-4, 1e-5):
        moved = rho + eps * ur / sf["psibar"]          # zeta -> zeta - eps
        sfm = oracle.slice_fields(moved, ur, w, wh, 1.0, edges[-1], rq=x)
        fd = (sf["q_psi"] - sfm["q_psi"]) / eps
        errs.append(np.max(np.abs(fd - sf["q_dpsidz"])))
    scale = np.max(np.abs(sf["q_dpsidz"]))
    assert errs[1] < 2e-5 * scale
    assert errs[0] / errs[1] > 5.0     # first-order convergence of the difference


def test_fields_at_ring_blend_one_sided_limits_with_self_weight():
    """At ring i each discontinuous field is the one-sided limit from below
    plus what_i/w_i of its jump (the self-weight rule); psi is continuous."""
    edges, rho, ur, w, wh = _random_state(n=30, seed=9)
    eps = 1e-10
    sf = oracle.slice_fields(rho, ur, w, wh, 1.0, edges[-1],
                             rq=np.concatenate([rho * (1 - eps), rho * (1 + eps)]))
    n = rho.shape[0]
    f = wh / w
    for key, qkey in (("dpsidr", "q_dpsidr"), ("dpsidz", "q_dpsidz")):
        lo, hi = sf[qkey][:n], sf[qkey][n:]
        blend = lo + f * (hi - lo)
        assert np.allclose(sf[key], blend, rtol=1e-6, atol=1e-7), key
    assert np.allclose(sf["psi"], sf["q_psi"][:n], atol=1e-8)
    # B^(p) at the ring is the mean of its one-sided limits
    lo, hi = sf["q_bp"][:n], sf["q_bp"][n:]
    assert np.allclose(sf["bp"], 0.5 * (lo + hi), rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("n,seed", [(8, 31), (24, 32), (64, 33)])
def test_direct_pairwise_summation_of_ring_contributions(n, seed):
    """O(N^2) superposition, no sorting and no prefix sums: every field at a
    point is the sum over rings of that ring's own contribution (Sec. II,
    Eqs. dpsi_dr, psi, dpsi_dzeta) plus the uniform ion column.  Ring j adds
    w_j ln max(rho, rho_j) to psi, w_j / rho to d_rho psi where it lies below
    rho, and t_j = w_j u_j / (rho_j psibar_j) to -d_zeta psi where it lies
    above; at ring i itself, ring i counts with what_i below and w_i - what_i
    above.  The beam term is the Gauss count of the charge strictly inside."""
    edges, rho, ur, w, wh = _random_state(n=n, seed=seed, u_scale=0.5)
    rmax = edges[-1]
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    br = rng.uniform(0.0, rmax, 3 * n)
    bq = -rng.uniform(0.2, 1.0, 3 * n)
    dxi = 0.03
    rq = np.concatenate([rng.uniform(1e-3, 1.2 * rmax, 2 * n), [1.5 * rmax]])
    sf = oracle.slice_fields(rho, ur, w, wh, 1.0, rmax, br, bq, dxi, rq=rq)

    def psi_ion(r):  # uniform column of radius rmax, density 1, neutralising sum w
        if r <= rmax:
            return -0.5 * rmax ** 2 * math.log(rmax) + 0.25 * (rmax ** 2 - r ** 2)
        return -0.5 * rmax ** 2 * math.log(r)

    def enclosed_ions(r):
        return 0.5 * min(r, rmax) ** 2

    def psi_at(r):
        total = psi_ion(r)
        for j in range(n):
            total += w[j] * math.log(max(r, rho[j]))
        return total

    psib = [1.0 + psi_at(rho[j]) for j in range(n)]
    t = [w[j] * ur[j] / (rho[j] * psib[j]) for j in range(n)]

    def fields(r, at_ring=None):
        below = 0.0
        above_t = 0.0
        for j in range(n):
            if j == at_ring:
                below += wh[j]
                above_t += (w[j] - wh[j]) / w[j] * t[j]
            elif rho[j] < r:
                below += w[j]
            elif rho[j] > r:
                above_t += t[j]
        q = sum(bq[k] for k in range(br.shape[0]) if br[k] < r)
        return (psi_at(r), (below - enclosed_ions(r)) / r, -above_t, q / (2 * math.pi * dxi * r))

    ref_ring = np.array([fields(rho[i], i) for i in range(n)])
    for col, key in enumerate(("psi", "dpsidr", "dpsidz", "bb")):
        assert _nerr(sf[key], ref_ring[:, col]) < 1e-13, key
    ref_q = np.array([fields(r) for r in rq])
    for col, key in enumerate(("q_psi", "q_dpsidr", "q_dpsidz", "q_bb")):
        assert _nerr(sf[key], ref_q[:, col]) < 1e-13, key


def test_quasistatic_invariant_gamma_minus_uz():
    """gamma - u_z = 1 + psi = psibar at every ring (Eq. cold_plasma_constant)."""
    edges, rho, ur, w, wh = _random_state(n=60, seed=21, u_scale=2.0)
    sf = oracle.slice_fields(rho, ur, w, wh, 1.0, edges[-1])
    assert np.allclose(sf["gamma"] - sf["uz"], 1.0 + sf["psi"], rtol=0, atol=1e-12)
    assert np.allclose(sf["psibar"], 1.0 + sf["psi"], rtol=0, atol=0)


# --------------------------------------------------------------------------
# B_theta^(p): closed form, dense elimination, jump conditions, Ampere
# --------------------------------------------------------------------------
def test_bp_one_ring_closed_form():
    g = json.load(open(os.path.join(GOLDEN, "one_ring_bp.json")))
    a, b = oracle.bp_shooting(g["rho"], g["A"], g["B"], g["C"])
    assert np.allclose(a, g["a"], rtol=1e-14, atol=1e-16)
    assert np.allclose(b, g["b"], rtol=1e-14, atol=1e-16)


def _jump_system(rho, A, B, C):
    """Dense 2N+2 system: b_0 = 0, a_N = 0, and at ring i (1-based)
    [rho B] = C_i rho_i and [2a] = A_i (mean of one-sided B) + B_i, with the
    unknowns ordered (a_0, b_0, a_1, b_1, ..., a_N, b_N)."""
    n = rho.shape[0]
    M = np.zeros((2 * n + 2, 2 * n + 2))
    v = np.zeros(2 * n + 2)
    M[0, 1] = 1.0
    M[1, 2 * n] = 1.0
    for i in range(1, n + 1):
        r = rho[i - 1]
        ia, ib, ja, jb = 2 * (i - 1), 2 * (i - 1) + 1, 2 * i, 2 * i + 1
        row = 2 * i
        M[row, ja] += r * r; M[row, jb] += 1.0
        M[row, ia] -= r * r; M[row, ib] -= 1.0
        v[row] = C[i - 1] * r
        row += 1
        M[row, ja] += 2.0; M[row, ia] -= 2.0
        for col, coef in ((ia, r), (ib, 1.0 / r), (ja, r), (jb, 1.0 / r)):
            M[row, col] -= 0.5 * A[i - 1] * coef
        v[row] = B[i - 1]
    sol = np.linalg.solve(M, v)
    return sol[0::2], sol[1::2]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bp_shooting_matches_dense_jump_solve(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 30
    rho = np.sort(rng.uniform(0.05, 3.0, n))
    A = rng.uniform(0.0, 0.2, n)
    B = rng.normal(0.0, 0.1, n)
    C = rng.normal(0.0, 0.05, n)
    a, b = oracle.bp_shooting(rho, A, B, C)
    ad, bd = _jump_system(rho, A, B, C)
    scale = max(np.abs(ad).max(), np.abs(bd).max())
    assert np.max(np.abs(a - ad)) < 1e-10 * scale
    assert np.max(np.abs(b - bd)) < 1e-10 * scale


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bp_banded_solve_matches_dense_jump_solve(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 30
    rho = np.sort(rng.uniform(0.05, 3.0, n))
    A = rng.uniform(0.0, 0.2, n)
    B = rng.normal(0.0, 0.1, n)
    C = rng.normal(0.0, 0.05, n)
    a, b = oracle.bp_solve(rho, A, B, C)
    ad, bd = _jump_system(rho, A, B, C)
    scale = max(np.abs(ad).max(), np.abs(bd).max())
    assert np.max(np.abs(a - ad)) < 1e-12 * scale
    assert np.max(np.abs(b - bd)) < 1e-12 * scale
    g = json.load(open(os.path.join(GOLDEN, "one_ring_bp.json")))
    a1, b1 = oracle.bp_solve(g["rho"], g["A"], g["B"], g["C"])
    assert np.allclose(a1, g["a"], rtol=1e-14, atol=1e-16) and np.allclose(b1, g["b"], rtol=1e-14, atol=1e-16)


def test_shooting_loses_digits_on_wide_columns_banded_solve_does_not():
    """Uniform column of 120 rings out to rho_max = 30 at rest-like
    coefficients (A = w/rho): the homogeneous solution grows ~e^30, so the
    App. A shooting error is ~1e-16 x 1e13 while the banded solve keeps the
    dense solve's accuracy."""
    edges = W.edges_uniform(120, 30.0)
    rho0, _, w, _ = oracle.ring_init(edges)
    A = w / rho0
    rng = np.random.Generator(np.random.PCG64(4))
    B = 1e-3 * rng.normal(size=rho0.shape[0]) * np.exp(-rho0)
    C = np.zeros_like(rho0)
    ad, bd = _jump_system(rho0, A, B, C)
    scale = np.max(np.abs(ad * rho0.max()))
    a_b, b_b = oracle.bp_solve(rho0, A, B, C)
    a_s, b_s = oracle.bp_shooting(rho0, A, B, C)
    err_band = np.max(np.abs(a_b - ad)) / scale
    err_shoot = np.max(np.abs(a_s - ad)) / scale
    assert err_band < 1e-10
    assert err_shoot > 1e3 * err_band


def test_slice_bp_satisfies_jump_and_boundary_conditions():
    edges, rho, ur, w, wh = _random_state(n=50, seed=4, u_scale=0.5)
    sf = oracle.slice_fields(rho, ur, w, wh, 1.0, edges[-1])
    order = sf["order"]
    r = rho[order]
    A, B, C = sf["A"][order], sf["B"][order], sf["C"][order]
    a, b = sf["a"], sf["b"]
    scale = np.abs(a).max() + np.abs(b).max()
    assert abs(b[0]) == 0.0 and abs(a[-1]) < 1e-10 * scale
    rb = (a[1:] - a[:-1]) * r ** 2 + (b[1:] - b[:-1])
    assert np.allclose(rb, C * r, atol=1e-10 * scale)
    bl = a[:-1] * r + b[:-1] / r
    br = a[1:] * r + b[1:] / r
    assert np.allclose(2 * (a[1:] - a[:-1]), A * 0.5 * (bl + br) + B, atol=1e-10 * scale)


def _nonlinear_wake(dxi, span, n_b0=0.5, sigma_r=0.3, n_rings=400, n_r=64):
    """Noise-free driver.  B^(b) at a ring is a step function of its radius
    (the enclosed count of discrete beam radii), so a ring crossing a beam
    radius costs a first-order error; convergence tests use many radii."""
    steps = int(round(span / dxi))
    drv = W.sampled_gaussian_beam(dxi, steps, n_b0, sigma_r, 0.6, 2.4, n_r=n_r)
    return W.Wake("pin", W.edges_uniform(n_rings, 5.0), [drv], dxi, steps)


def test_ampere_law_for_plasma_field_converges_second_order():
    """rho B^(p)(rho) = -sum_{rho_i<rho} w_i u_z,i/psibar_i + d/dzeta int_0^rho rho' d_zeta psi
    (Eq. maxwell_qsa_4 with the beam term removed), the zeta derivative taken
    by central differences across slices behind the driver."""
    rq = np.linspace(0.05, 4.5, 37)
    errs = []
    for dxi in (0.02, 0.01, 0.005):
        wk = _nonlinear_wake(dxi, 9.0)
        _, _, w, wh = oracle.ring_init(wk.edges)
        res = oracle.run_wake(wk, beam_fields=(), ring_dumps=("r", "ur", "psibar", "uz"))
        assert res.status == 0
        n = int(round(8.0 / dxi))
        R = res.rings
        sf = oracle.slice_fields(R["r"][n], R["ur"][n], w, wh, 1.0, 5.0, rq=rq)

        def zint(k):
            t = w * R["ur"][k] / (R["r"][k] * R["psibar"][k])
            return -np.sum(t[None, :] * np.minimum(rq[:, None], R["r"][k][None, :]) ** 2 / 2, axis=1)

        jz = np.array([-np.sum((w * R["uz"][n] / R["psibar"][n])[R["r"][n] < x]) for x in rq])
        rhs = jz - (zint(n + 1) - zint(n - 1)) / (2 * dxi)
        lhs = rq * sf["q_bp"]
        errs.append(np.max(np.abs(lhs - rhs)) / np.max(np.abs(lhs)))
    assert errs[-1] < 5e-4, errs
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def test_lorentz_force_integration_matches_algebraic_uz():
    """du_z/dxi = -(gamma E_z + u_r B_theta)/psibar along each ring (Lorentz
    force with d xi/dt = psibar/gamma) reproduces the algebraic u_z of
    Eq. plasma_particle_motion_3, converging at second order."""
    errs = []
    for dxi in (0.02, 0.01, 0.005):
        wk = _nonlinear_wake(dxi, 12.0)
        res = oracle.run_wake(wk, beam_fields=(),
                              ring_dumps=("ur", "psibar", "uz", "gamma", "dpsidz", "bp", "bb"))
        R = res.rings
        f = -(R["gamma"] * (-R["dpsidz"]) + R["ur"] * (R["bp"] + R["bb"])) / R["psibar"]
        uz = R["uz"][0][None, :] + np.concatenate(
            [np.zeros((1, f.shape[1])), np.cumsum(0.5 * (f[1:] + f[:-1]) * dxi, axis=0)])
        errs.append(np.max(np.abs(uz - R["uz"])))
    scale = np.max(np.abs(R["uz"]))
    assert errs[-1] < 5e-5 * scale / 0.08, errs
    assert errs[0] / errs[1] > 2.8 and errs[1] / errs[2] > 2.8, errs


# --------------------------------------------------------------------------
# the integrator
# --------------------------------------------------------------------------
def test_adams_bashforth_is_second_order():
    """Ring radii at xi = 8 against a dxi/8 reference: error drops ~4x per
    halving of dxi (Euler start, AB2 after)."""
    def radii(dxi):
        wk = _nonlinear_wake(dxi, 8.0, n_r=4096)
        res = oracle.run_wake(wk, beam_fields=())
        return res.final_r
    ref = radii(0.0025)
    errs = [np.max(np.abs(radii(d) - ref)) for d in (0.04, 0.02, 0.01)]
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3, errs


# --------------------------------------------------------------------------
# the whole wake against linear theory
# --------------------------------------------------------------------------
def _axis_ez(n_b0, n_rings, dxi, sigma_r=0.5, sigma_z=1.0, span=20.0, xi_d=4.0):
    steps = int(round(span / dxi))
    pxi = np.arange(steps) * dxi
    beams_xi, beams_r, beams_qw = [pxi], [np.zeros(steps)], [np.zeros(steps)]
    if n_b0 > 0:
        drv = W.sampled_gaussian_beam(dxi, steps, n_b0, sigma_r, sigma_z, xi_d, n_r=256)
        beams_xi.insert(0, drv.xi)
        beams_r.insert(0, drv.r)
        beams_qw.insert(0, drv.q * drv.w)
    res = oracle.run(W.edges_uniform(n_rings, 5.0), np.concatenate(beams_xi),
                     np.concatenate(beams_r), np.concatenate(beams_qw), dxi, steps,
                     beam_fields=("ez",))
    return pxi, res.beam["ez"][-steps:]


def _fit(pxi, ez, xi_d=4.0, lo=9.0, hi=19.9):
    m = (pxi > lo) & (pxi < hi)
    Amat = np.stack([np.cos(pxi[m] - xi_d), np.sin(pxi[m] - xi_d)], 1)
    c, *_ = np.linalg.lstsq(Amat, ez[m], rcond=None)
    return math.hypot(*c), math.atan2(c[1], c[0])


def test_linear_wake_matches_closed_form():
    """E_z on axis behind a weak Gaussian driver (sigma_r = 0.5, sigma_z = 1)
    against the closed form of linear theory (golden linear_wake.json), with
    the O(drho^2) response of the undriven column subtracted.

    - Linear regime, n_b0 = 0.005: amplitude within 0.5 % and phase within
      0.005 rad (well inside 2 % / 0.02 rad), at 400 rings / dxi = 0.01 and
      at 800 rings / dxi = 0.005; the amplitude deviation shrinks under that
      refinement (measured 1.0e-3 -> 8e-5).
    - n_b0 = 0.05: amplitude within 2 % (measured 0.6 %), phase within
      0.03 rad (measured 0.024 rad): 0.02 rad is not reachable there, the
      phase offset being the model's own second-order response, which no
      refinement removes (it moves by < 1 % between the two resolutions).
    - That deviation is the nonlinear response: with E(n) the wake of peak
      density n, D(n) = E(n) - (n / 0.005) E(0.005) on one grid grows as
      n (n - 0.005) (rms ratio D(0.05) / D(0.025) = 4.5 expected, measured
      4.54), and the phase offset grows in proportion to n_b0 (ratio 2.1
      between 0.05 and 0.025)."""
    g = json.load(open(os.path.join(GOLDEN, "linear_wake.json")))["cases"]
    amp_per_nb = g[0]["Ez_axis_amplitude"] / g[0]["n_b0"]  # the closed form is linear in n_b0
    assert g[0]["n_b0"] == 0.05 and g[1]["n_b0"] == 0.005
    assert abs(g[1]["Ez_axis_amplitude"] - 0.1 * g[0]["Ez_axis_amplitude"]) < 1e-15
    dev = {}
    for n_rings, dxi in ((400, 0.01), (800, 0.005)):
        pxi, base = _axis_ez(0.0, n_rings, dxi)
        ez = {nb: _axis_ez(nb, n_rings, dxi)[1] - base for nb in (0.005, 0.025, 0.05)}
        fits = {nb: _fit(pxi, e) for nb, e in ez.items()}
        dev[n_rings] = {nb: (amp / (amp_per_nb * nb) - 1.0, ph) for nb, (amp, ph) in fits.items()}
        d_small, ph_small = dev[n_rings][0.005]
        d_big, ph_big = dev[n_rings][0.05]
        assert abs(d_small) < 0.005 and abs(ph_small) < 0.005, (n_rings, dev[n_rings])
        assert abs(d_big) < 0.02 and abs(ph_big) < 0.03, (n_rings, dev[n_rings])
        m = (pxi > 9.0) & (pxi < 19.9)
        rms = {nb: np.sqrt(np.mean((ez[nb][m] - (nb / 0.005) * ez[0.005][m]) ** 2)) for nb in (0.025, 0.05)}
        assert 4.0 < rms[0.05] / rms[0.025] < 5.0, rms
        assert 1.8 < ph_big / dev[n_rings][0.025][1] < 2.4, dev[n_rings]
    # refinement: the linear-regime amplitude error shrinks, the nonlinear
    # phase offset stays
    assert abs(dev[800][0.005][0]) < 0.5 * abs(dev[400][0.005][0]), dev
    assert abs(dev[800][0.05][1] - dev[400][0.05][1]) < 0.05 * abs(dev[400][0.05][1]), dev


# --------------------------------------------------------------------------
# beam source and binning
# --------------------------------------------------------------------------
def test_beam_field_is_gauss_count_and_excludes_self():
    rng = np.random.Generator(np.random.PCG64(8))
    m = 300
    br = rng.uniform(0.0, 2.0, m)
    bq = -rng.uniform(0.5, 1.5, m)
    edges, rho, ur, w, wh = _random_state(n=20, seed=8)
    dxi = 0.05
    sf = oracle.slice_fields(rho, ur, w, wh, 1.0, edges[-1], br, bq, dxi, rq=br)
    for k in range(0, m, 7):
        Q = bq[br < br[k]].sum()
        assert abs(sf["q_bb"][k] - Q / (2 * math.pi * dxi * br[k])) < 1e-12 * max(1, abs(Q))
    for i in range(rho.shape[0]):
        Q = bq[br < rho[i]].sum()
        assert abs(sf["bb"][i] - Q / (2 * math.pi * dxi * rho[i])) < 1e-12 * max(1, abs(Q))


def test_nearest_slice_binning():
    """A particle belongs to slice floor(xi/dxi + 1/2) (beam-grid spacing =
    solver step, Sec. III); particles whose slice lies outside the window get
    zero fields.  One charged particle in slice 1 makes the beam field of that
    slice large, so the probes show which slice they landed in."""
    dxi, steps = 0.1, 5
    edges = W.edges_uniform(10, 1.0)
    probes = {0.0499: 0, 0.0501: 1, 0.1: 1, 0.1499: 1, 0.1501: 2, -0.0499: 0,
              -0.0501: None, 0.4499: 4, 0.4501: None}
    xi = np.array([0.1] + list(probes))
    r = np.array([0.25] + [0.5] * len(probes))
    qw = np.array([-1.0] + [0.0] * len(probes))
    res = oracle.run(edges, xi, r, qw, dxi, steps, beam_fields=("bt", "psi"))
    bt, psi = res.beam["bt"][1:], res.beam["psi"][1:]
    in_one = [k for k, sl in enumerate(probes.values()) if sl == 1]
    for k, sl in enumerate(probes.values()):
        if sl is None:
            assert bt[k] == 0.0 and psi[k] == 0.0
        elif sl == 1:
            # beam field -1/(2 pi dxi r) partly shielded by the plasma response
            assert bt[k] == bt[in_one[0]] and bt[k] < -1.0
        else:
            assert abs(bt[k]) < 0.1 and psi[k] != 0.0


def test_charge_conservation_and_neutrality_through_a_run():
    wk = _nonlinear_wake(0.02, 10.0, n_b0=2.0)
    _, _, w, wh = oracle.ring_init(wk.edges)
    res = oracle.run_wake(wk, beam_fields=(), ring_dumps=("r", "ur"))
    assert res.status == 0
    assert abs(w.sum() - 12.5) < 1e-12
    for n in (100, 300, 499):
        r, u = res.rings["r"][n], res.rings["ur"][n]
        far = np.array([1.001, 3.0]) * max(5.0, r.max())
        sf = oracle.slice_fields(r, u, w, wh, 1.0, 5.0, rq=far)
        assert np.max(np.abs(sf["q_psi"])) < 1e-11
        assert np.max(np.abs(sf["q_dpsidr"])) < 1e-12
        assert np.all(r >= 0.0)


def test_fields_on_the_axis_are_the_limits_from_outside():
    """At r = 0 exactly (a beam particle on the axis) the plasma fields are
    the limits r -> 0+ of the off-axis sums: psi and E_z of all rings
    outside, no radial field, no B^(p); the beam field is zero (no charge
    strictly inside r = 0, though a particle sits on the axis)."""
    edges, rho, ur, w, wh = _random_state(n=25, seed=5)
    br = np.array([0.0, 0.3, 0.9])
    bq = np.array([-1e-3, -2e-3, -1e-3])
    sf = oracle.slice_fields(rho, ur, w, wh, 1.0, edges[-1], br, bq, 0.05, rq=np.array([0.0, 1e-12]))
    assert abs(sf["q_psi"][0] - sf["q_psi"][1]) < 1e-10
    assert abs(sf["q_ez"][0] - sf["q_ez"][1]) < 1e-12 * max(1.0, abs(sf["q_ez"][1]))
    assert sf["q_ez"][0] != 0.0
    for k in ("q_wr", "q_bp"):
        assert sf[k][0] == 0.0 and abs(sf[k][1]) < 1e-9, k
    assert sf["q_bb"][0] == 0.0 and sf["q_bt"][0] == 0.0


def test_the_wake_stops_at_the_first_slice_where_psibar_reaches_zero():
    """c11: a strong driver drives psibar through zero behind the first
    bubble; the march stops there with ENONFINITE (the failing slice's
    fields are kept, nothing after it), psibar having stayed positive and
    every field finite before."""
    wk = W.batched_wake(3)
    res = oracle.run_wake(W.Wake(wk.name, wk.edges, wk.beams, wk.dxi, 1700), beam_fields=(),
                          ring_dumps=("psibar", "psi", "dpsidr", "dpsidz", "bp"))
    f = res.fail_slice
    assert res.status == 4 and 0 < f < 1700 and res.slices_run == f + 1
    R = res.rings
    assert np.min(R["psibar"][:f]) > 0.0
    assert all(np.all(np.isfinite(R[k][:f])) for k in ("psi", "dpsidr", "dpsidz", "bp"))
    bad = (R["psibar"][f] <= 0.0) | ~np.isfinite(R["psi"][f]) | ~np.isfinite(R["bp"][f])
    assert bad.any()
    assert np.all(R["psibar"][f + 1:] == 0.0)  # slices after the stop are never solved


def test_rings_at_equal_radii_keep_their_previous_order():
    """c10: the radius sort is stable with respect to the previous order (at
    a slice's start, ring id order): of rings at exactly the same radius the
    earlier one counts as below the later ones, so the later ring's partial
    sums include the earlier one's weight and not the other way round."""
    edges, rho, ur, w, wh = _random_state(n=30, seed=21)
    rho = rho.copy()
    rho[[4, 17, 25]] = rho[9]        # four rings at one radius
    rho[[2, 28]] = rho[13]           # two at another
    sf = oracle.slice_fields(rho, ur, w, wh, 1.0, edges[-1])
    order = list(sf["order"])
    assert order == sorted(range(30), key=lambda i: (rho[i], i))
    # the tied group's d_rho psi steps by each earlier member's weight
    grp = [4, 9, 17, 25]
    for a, b in zip(grp, grp[1:]):
        jump = (sf["dpsidr"][b] - sf["dpsidr"][a]) * rho[a]
        assert abs(jump - (w[a] + wh[b] - wh[a])) < 1e-12


def test_axis_crossing_reflects_and_stays_finite():
    """A strong narrow driver throws rings through the axis; they come back at
    rho >= 0 and the march completes."""
    dxi = 0.01
    drv = W.sampled_gaussian_beam(dxi, 800, 5.0, 0.15, 0.5, 2.0, n_r=64)
    wk = W.Wake("axis", W.edges_uniform(300, 5.0), [drv], dxi, 800)
    res = oracle.run_wake(wk, beam_fields=(), ring_dumps=("r", "ur"))
    assert res.status == 0
    r = res.rings["r"]
    assert np.all(r >= 0.0) and np.all(np.isfinite(r))
    crossed = np.any(np.diff(np.sign(res.rings["ur"]), axis=0) != 0, axis=0)
    assert crossed.any()


def test_ab2_stays_second_order_through_axis_crossings():
    """A light ring oscillating through the axis five times in the ion
    column's focusing field (tests/axis_orbit.py): the AB2 march converges
    to the independently integrated signed orbit at second order, which
    needs the reflection to negate rho, u_r and the ring's AB2 history
    (without the history flip each crossing errs by O(dxi): first order)."""
    import axis_orbit
    r_ref, u_ref, crossings = axis_orbit.reference()
    assert crossings >= 4
    errs = []
    for dxi in (0.02, 0.01, 0.005):
        r, u, rmin = axis_orbit.march(dxi, "ab2")
        assert rmin > 1e-5  # the self-weight layer at the axis is never sampled
        errs.append(max(np.max(np.abs(r - r_ref)), np.max(np.abs(u - u_ref))))
    q = [a / b for a, b in zip(errs, errs[1:])]
    assert all(3.6 < x < 4.4 for x in q), (errs, q)
    assert errs[-1] < 2e-5, errs
