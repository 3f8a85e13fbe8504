"""Pins of the oracle's beam push (oracle/beam_push.py) to properties of
the Boris method and of motion in simple fields that do not come from its
own formulas: exact kicks in a pure electric field, exact norm conservation
and the known rotation angle 2 atan(|q B| dt / 2 m gamma) in a pure magnetic
field, the Larmor circle, the E x B drift, second-order convergence of a
betatron oscillation in an ion channel to its closed form, the co-moving
drift of xi, and the Cartesian form of the axisymmetric fields."""
import math

import numpy as np

from oracle import beam_push as bp


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_pure_electric_field_is_an_exact_kick():
    rng = _rng(1)
    u = rng.normal(size=(3, 50))
    E = rng.normal(size=(3, 50))
    h = 0.37
    un = bp.boris_step(u, E, np.zeros((3, 50)), h)
    assert np.allclose(un, u + 2 * h * E, rtol=0, atol=1e-14)


def test_pure_magnetic_field_rotates_by_the_boris_angle():
    rng = _rng(2)
    u = rng.normal(size=(3, 40)) * 3.0
    bz = 2.5
    B = np.zeros((3, 40))
    B[2] = bz
    h = -0.11  # electrons, dt = 0.22
    un = bp.boris_step(u, np.zeros((3, 40)), B, h)
    # |u| and u_z are conserved
    assert np.allclose(np.linalg.norm(un, axis=0), np.linalg.norm(u, axis=0), rtol=1e-14)
    assert np.allclose(un[2], u[2], rtol=0, atol=1e-14)
    # the transverse momentum turns by 2 atan(|h B| / gamma)
    g = np.sqrt(1 + np.sum(u * u, axis=0))
    ang = np.arctan2(un[1], un[0]) - np.arctan2(u[1], u[0])
    ang = (ang + np.pi) % (2 * np.pi) - np.pi
    expect = -np.sign(h * bz) * 2 * np.arctan(np.abs(h * bz) / g)
    assert np.allclose(ang, expect, rtol=0, atol=1e-12)


def test_larmor_circle():
    """A positron (q = +1) in B_z: radius gamma v_perp / B = u_perp / B."""
    u = np.array([[0.8], [0.0], [0.3]])
    B = np.array([[0.0], [0.0], [1.7]])
    dt = 0.005
    x = np.zeros((3, 1))
    xs = []
    for _ in range(4000):
        u = bp.boris_step(u, np.zeros((3, 1)), B, 0.5 * dt)
        g = math.sqrt(1 + float(np.sum(u * u)))
        x = x + dt * u / g
        xs.append(x[:2, 0].copy())
    xs = np.array(xs)  # about four turns
    centre = 0.5 * (xs.max(axis=0) + xs.min(axis=0))
    radius = np.linalg.norm(xs - centre, axis=1)
    assert abs(radius.mean() - 0.8 / 1.7) < 1e-4
    assert radius.std() < 1e-4


def test_e_cross_b_drift():
    """Crossed E_y, B_z with E < B: the guiding centre drifts at E x B / B^2
    along x."""
    Ey, Bz = 0.2, 1.0
    u = np.zeros((3, 1))
    x = np.zeros((3, 1))
    E = np.array([[0.0], [Ey], [0.0]])
    B = np.array([[0.0], [0.0], [Bz]])
    dt = 0.01
    n = 20000
    for _ in range(n):
        u = bp.boris_step(u, E, B, 0.5 * dt)
        g = math.sqrt(1 + float(np.sum(u * u)))
        x = x + dt * u / g
    vd = x[0, 0] / (n * dt)
    assert abs(vd - Ey / Bz) < 5e-3


def test_betatron_oscillation_converges_at_second_order():
    """An ultra-relativistic electron in an ion channel (W_r = r/2, no
    B_theta, no E_z) oscillates as x0 cos(t / sqrt(2 gamma)); the Boris
    error at a fixed time falls ~4x per halving of dt."""
    gamma = 200.0
    x0 = 0.05
    T = 0.5 * 2 * math.pi * math.sqrt(2 * gamma)
    errs = []
    for n in (200, 400, 800):
        dt = T / n
        st = {"x": np.array([x0]), "y": np.array([0.0]), "xi": np.array([0.0]),
              "ux": np.array([0.0]), "uy": np.array([0.0]), "uz": np.array([math.sqrt(gamma ** 2 - 1)])}
        # start the momentum half a step back (leapfrog)
        st["ux"] = st["ux"] + 0.5 * dt * 0.5 * x0
        for _ in range(n):
            r = np.hypot(st["x"], st["y"])
            st = bp.push(st, np.zeros(1), 0.5 * r, np.zeros(1), -1.0, dt)
        wb = 1.0 / math.sqrt(2 * gamma)
        errs.append(abs(st["x"][0] - x0 * math.cos(wb * T)))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
    assert errs[-1] < 1e-4 * x0


def test_free_drift_of_xi():
    rng = _rng(5)
    n = 30
    st = {k: rng.normal(size=n) for k in ("x", "y", "xi", "ux", "uy")}
    st["uz"] = rng.uniform(1, 50, n)
    dt = 0.7
    out = bp.push(st, np.zeros(n), np.zeros(n), np.zeros(n), -1.0, dt)
    g = np.sqrt(1 + st["ux"] ** 2 + st["uy"] ** 2 + st["uz"] ** 2)
    assert np.allclose(out["xi"], st["xi"] + dt * (1 - st["uz"] / g), rtol=0, atol=1e-14)
    assert np.allclose(out["x"], st["x"] + dt * st["ux"] / g, rtol=0, atol=1e-14)


def test_cartesian_fields_are_radial_and_azimuthal():
    rng = _rng(6)
    x, y = rng.normal(size=20), rng.normal(size=20)
    ez, wr, bt = rng.normal(size=20), rng.normal(size=20), rng.normal(size=20)
    E, B = bp.cartesian_fields(x, y, ez, wr, bt)
    r = np.hypot(x, y)
    assert np.allclose((E[0] * x + E[1] * y) / r, wr + bt)       # E_r
    assert np.allclose(E[0] * y - E[1] * x, 0.0, atol=1e-14)      # no E_theta
    assert np.allclose((B[1] * x - B[0] * y) / r, bt)             # B_theta
    assert np.allclose(B[0] * x + B[1] * y, 0.0, atol=1e-14)      # no B_r
    assert np.allclose(E[2], ez) and np.allclose(B[2], 0.0)
    E0, B0 = bp.cartesian_fields([0.0], [0.0], [1.5], [2.0], [3.0])
    assert np.allclose(E0[:, 0], [0, 0, 1.5]) and np.allclose(B0[:, 0], 0.0)


def test_rotation_between_the_half_kicks_uses_the_half_kicked_gamma():
    """With E and B together the Boris step is kick - rotate - kick: the
    momentum after the first half kick, u- = u + hE, and the one before
    the second, u+ = u_new - hE, have the same norm and the same component
    along B, and the part across B turns by 2 atan(|h B| / gamma(u-))
    (the rotation is taken at the half-kicked momentum's gamma)."""
    rng = _rng(7)
    n = 40
    u = rng.normal(size=(3, n)) * 2.0
    E = rng.normal(size=(3, n))
    B = rng.normal(size=(3, n)) * 1.5
    h = 0.09
    un = bp.boris_step(u, E, B, h)
    um, up = u + h * E, un - h * E
    assert np.allclose(np.linalg.norm(up, axis=0), np.linalg.norm(um, axis=0), rtol=1e-14)
    b = B / np.linalg.norm(B, axis=0)
    assert np.allclose(np.sum(up * b, axis=0), np.sum(um * b, axis=0), rtol=0, atol=1e-13)
    pm = um - np.sum(um * b, axis=0) * b
    pp = up - np.sum(up * b, axis=0) * b
    cosang = np.sum(pm * pp, axis=0) / (np.linalg.norm(pm, axis=0) * np.linalg.norm(pp, axis=0))
    gm = np.sqrt(1 + np.sum(um * um, axis=0))
    expect = 2 * np.arctan(h * np.linalg.norm(B, axis=0) / gm)
    assert np.allclose(np.arccos(np.clip(cosang, -1, 1)), expect, rtol=0, atol=1e-7)
