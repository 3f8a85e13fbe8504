"""A ring that passes through the axis, for the pins of the two readings
the paper leaves open there: a ring pushed below the axis reappears at
-rho with u_r and its AB2 history negated, and an RK4 stage state below
the axis is evaluated mirrored (its derivative mirrored back).

Ring 0 fills the cell [0, 1e-5], so its weight (5e-11) and self weight
(1.25e-11) are negligible; it starts at rho = 0.15 moving inward
(u_r = -0.15) and oscillates through the axis in the focusing field of the
ion column (Sec. II, the Baxevanis-Stupakov limit), five times over
xi = 20, always below ring 1 (cell [1e-5, 0.8], ring at 0.4).  The other
rings start at rest at their cell centres and drift slowly and smoothly
(the discrete psi offset of the wide second cell gives them a small
B_theta^(p)); no two rings cross.

Read as a signed radius, the orbit of ring 0 is smooth through the axis:
the ring equations (Eqs. plasma_particle_motion_1,2 with the fields of
Eqs. dpsi_dr..b_theta) are odd under (rho, u_r) -> (-rho, -u_r).  The
reference below integrates that signed orbit with an adaptive Runge-Kutta
method of order 8 (scipy's DOP853, rtol 1e-12), independent of the
oracle's integrators and of its axis handling: the other rings take their
slice fields from the oracle's slice function (without ring 0, whose
charge moves their fields by ~1e-10), and ring 0 is a massless test ring
driven by the off-ring fields at |rho_0| (its own self-weight barrier
~w_0 / rho, which turns a continuous ring back within ~1e-11 of the axis,
is the part of the model that a discrete step jumps over; the oracle's
steps never come within 5e-5 of the axis here, where it is below 1e-6 of
the focusing force).  A march that reflects correctly converges to this
orbit at the integrator's order; one that mishandles a crossing commits an
O(dxi) error there and converges at first order at best.
"""
import numpy as np

import oracle

EDGES = np.concatenate([[0.0, 1e-5], np.linspace(0.8, 5.0, 85)])
SPAN = 20.0
R0, U0 = 0.15, -0.15


def initial_state():
    rho0, _, _, _ = oracle.ring_init(EDGES)
    r, u = rho0.copy(), np.zeros(rho0.shape[0])
    r[0], u[0] = R0, U0
    return r, u


def reference():
    """(rho, u_r) by ring id at xi = SPAN from the signed test-ring orbit,
    and the number of axis crossings of ring 0 on the way."""
    from scipy.integrate import solve_ivp
    _, _, w, wh = oracle.ring_init(EDGES)
    n = w.shape[0]
    rho_max = EDGES[-1]

    def rhs(_x, y):
        r, u = y[:n], y[n:]
        sf = oracle.slice_fields(r[1:], u[1:], w[1:], wh[1:], 1.0, rho_max, rq=np.array([abs(r[0])]))
        f = np.empty(2 * n)
        pb = sf["psibar"]
        f[1:n] = u[1:] / pb
        f[n + 1:] = sf["gamma"] * sf["dpsidr"] / pb - (sf["bp"] + sf["bb"])
        # ring 0 at the signed radius r[0]: the fields at |r[0]|, the radial
        # force odd in the signed radius
        pb0 = 1.0 + sf["q_psi"][0]
        g0 = (1.0 + u[0] ** 2 + pb0 ** 2) / (2.0 * pb0)
        sgn = -1.0 if r[0] < 0.0 else 1.0
        f[0] = u[0] / pb0
        f[n] = sgn * (g0 * sf["q_dpsidr"][0] / pb0 - (sf["q_bp"][0] + sf["q_bb"][0]))
        return f

    r, u = initial_state()
    sol = solve_ivp(rhs, (0.0, SPAN), np.concatenate([r, u]), method="DOP853", rtol=1e-12, atol=1e-14)
    assert sol.status == 0, sol.message
    y = sol.y[:, -1].copy()
    if y[0] < 0.0:  # the same ring, seen at +rho moving the other way
        y[0], y[n] = -y[0], -y[n]
    crossings = int(np.count_nonzero(np.diff(np.sign(sol.y[0])) != 0))
    return y[:n], y[n:], crossings


def march(dxi, integrator):
    """The oracle's march of the same state: final (rho, u_r) by id and the
    smallest radius ring 0 was seen at."""
    r, u = initial_state()
    steps = int(round(SPAN / dxi))
    res = oracle.run(EDGES, np.zeros(0), np.zeros(0), np.zeros(0), dxi, steps, beam_fields=(),
                     ring_dumps=("r",), init_state=(r, u), integrator=integrator)
    assert res.status == 0 and res.slices_run == steps
    return res.final_r, res.final_ur, float(res.rings["r"][:, 0].min())
