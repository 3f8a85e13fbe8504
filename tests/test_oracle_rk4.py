"""Pins of the oracle's RK4 ring integrator (orc_run, integrator "rk4"):
classical fourth-order Runge-Kutta over each slice, the beam source at the
half step the mean of slices n and n+1.

Order of convergence needs a right-hand side that is smooth in rho and xi:
B^(b) at a ring jumps where the ring crosses a beam particle's radius and
the fields jump where rings cross each other, and nearest-slice sampling of
a source that switches on misplaces the switch by O(dxi).  The pins use a
thin shell of beam charge at rho = 2 whose line density ramps linearly from
xi = 0 (the half-step mean of two slices is then exact), weak enough that
no ring crosses another or the shell."""
import numpy as np

import oracle
from paper_2603_16623_gb300 import workloads as W


def _shell_ramp_wake(dxi, integrator, span=5.0, q0=0.01, radius=2.0):
    steps = int(round(span / dxi)) + 1
    xi = np.arange(steps) * dxi
    beam = W.Beam(xi, np.full(steps, radius), q0 * xi * dxi, -1.0)
    return W.Wake("shell", W.edges_uniform(300, 5.0), [beam], dxi, steps, integrator=integrator)


def _radii_at(dxi, integrator, at=4.0):
    res = oracle.run_wake(_shell_ramp_wake(dxi, integrator), ring_dumps=("r",), beam_fields=())
    assert res.status == 0
    r = res.rings["r"]
    assert np.all(np.diff(r, axis=1) > 0)  # no ring crossing
    return r[int(round(at / dxi))]


def test_rk4_is_fourth_order_and_ab2_second():
    ref = _radii_at(0.00125, "rk4")
    e4 = [np.max(np.abs(_radii_at(d, "rk4") - ref)) for d in (0.08, 0.04, 0.02)]
    e2 = [np.max(np.abs(_radii_at(d, "ab2") - ref)) for d in (0.04, 0.02, 0.01)]
    q4 = [a / b for a, b in zip(e4, e4[1:])]
    q2 = [a / b for a, b in zip(e2, e2[1:])]
    assert all(q > 12.0 for q in q4), (e4, q4)
    assert all(3.5 < q < 4.5 for q in q2), (e2, q2)


def test_rk4_and_ab2_agree_on_a_wake():
    """Both integrators solve the same equations: on a moderate wake their
    ring radii differ by the AB2 error only (second order in dxi)."""
    diffs = []
    for dxi in (0.01, 0.005):
        steps = int(round(6.0 / dxi))
        drv = W.sampled_gaussian_beam(dxi, steps, 0.5, 0.4, 0.6, 2.4, n_r=256)
        a = oracle.run_wake(W.Wake("a", W.edges_uniform(300, 5.0), [drv], dxi, steps), beam_fields=())
        b = oracle.run_wake(W.Wake("b", W.edges_uniform(300, 5.0), [drv], dxi, steps, integrator="rk4"),
                            beam_fields=())
        assert a.status == b.status == 0
        diffs.append(np.max(np.abs(a.final_r - b.final_r)))
    assert diffs[1] < 1e-3 and diffs[0] / diffs[1] > 2.5, diffs


def test_rk4_axis_crossing_is_mirrored():
    """Rings driven through the axis by a dense narrow driver come back on
    the other side: finite, non-negative radii and a finite window."""
    drv = W.gaussian_beam(40_000, 8.0, 0.1, 0.5, 1.8, seed=9)
    res = oracle.run_wake(W.Wake("axis", W.edges_uniform(200, 4.0), [drv], 0.01, 500, integrator="rk4"),
                          ring_dumps=("r", "ur"))
    assert res.status == 0
    assert np.all(res.rings["r"] >= 0.0) and np.all(np.isfinite(res.rings["ur"]))
    assert np.any(np.diff(np.sign(res.rings["ur"]), axis=0) != 0)


def test_rk4_linear_wake_matches_closed_form():
    """The linear closed form of E_z on axis behind a weak Gaussian driver
    (golden linear_wake.json, n_b0 = 0.005) holds for the RK4 march too:
    amplitude within 1 %, phase within 0.01 rad after subtracting the
    undriven column's O(drho^2) response; the sampled driver enters every
    stage (half-step sources the mean of two slices)."""
    import json
    import math
    import os
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "linear_wake.json")
    case = json.load(open(golden))["cases"][1]
    assert case["n_b0"] == 0.005
    dxi, steps, xi_d = 0.01, 2000, 4.0
    pxi = np.arange(steps) * dxi

    def axis_ez(n_b0):
        xs, rs, qs = [pxi], [np.zeros(steps)], [np.zeros(steps)]
        if n_b0 > 0:
            drv = W.sampled_gaussian_beam(dxi, steps, n_b0, case["sigma_r"], case["sigma_z"], xi_d, n_r=256)
            xs.insert(0, drv.xi)
            rs.insert(0, drv.r)
            qs.insert(0, drv.q * drv.w)
        res = oracle.run(W.edges_uniform(400, 5.0), np.concatenate(xs), np.concatenate(rs), np.concatenate(qs),
                         dxi, steps, beam_fields=("ez",), integrator="rk4")
        assert res.status == 0
        return res.beam["ez"][-steps:]

    ez = axis_ez(case["n_b0"]) - axis_ez(0.0)
    m = (pxi > 9.0) & (pxi < 19.9)
    A = np.stack([np.cos(pxi[m] - xi_d), np.sin(pxi[m] - xi_d)], 1)
    c, *_ = np.linalg.lstsq(A, ez[m], rcond=None)
    amp, ph = math.hypot(*c), math.atan2(c[1], c[0])
    assert abs(amp / case["Ez_axis_amplitude"] - 1.0) < 0.01, amp
    assert abs(ph) < 0.01, ph


def test_rk4_stays_fourth_order_through_axis_crossings():
    """The light ring of tests/axis_orbit.py, oscillating through the axis
    five times: the RK4 march converges to the independently integrated
    signed orbit at fourth order, which needs each stage state below the
    axis to be evaluated mirrored and its derivative mirrored back."""
    import axis_orbit
    r_ref, u_ref, crossings = axis_orbit.reference()
    assert crossings >= 4
    errs = []
    for dxi in (0.16, 0.08, 0.04):
        r, u, rmin = axis_orbit.march(dxi, "rk4")
        assert rmin > 1e-5
        errs.append(max(np.max(np.abs(r - r_ref)), np.max(np.abs(u - u_ref))))
    q = [a / b for a, b in zip(errs, errs[1:])]
    assert all(q_ > 12.0 for q_ in q), (errs, q)
    assert errs[-1] < 1e-7, errs
