"""Writes the closed-form fixtures in this folder.

The paper prints no worked numerical example, so every fixture here is a
closed form derived from the paper's equations (the derivation is stored in
the fixture).  This script uses only the standard library and scipy; it
calls neither the oracle nor the CUDA library.

    python tests/golden/make_golden.py
"""
import json
import math
import os
from fractions import Fraction

from scipy import integrate, special

HERE = os.path.dirname(os.path.abspath(__file__))


def one_ring_bp():
    # One ring at rho1 with coefficients A, B, C.  Region 0 (0, rho1):
    # B = a0 rho (b0 = 0); region 1 (rho1, inf): B = b1 / rho (a1 = 0).
    # Integrating d/drho[(1/rho) d/drho(rho B)] = A delta Bbar + B delta + C d/drho delta
    # across the ring: [rho B] = C rho1 and [2a] = A Bbar + B, Bbar the mean of
    # the one-sided values.  Hence
    #   a0 = -(2B + A C) / (2 (2 + A rho1)),  b1 = a0 rho1^2 + C rho1.
    rho1, A, B, C = Fraction(4, 5), Fraction(3, 10), Fraction(-1, 5), Fraction(1, 20)
    a0 = -(2 * B + A * C) / (2 * (2 + A * rho1))
    b1 = a0 * rho1 ** 2 + C * rho1
    return {
        "citation": "Eq. ai_bi with b_0 = 0, a_N = 0 (Sec. II) and its App. A solution, N = 1",
        "derivation": "jump conditions [rho B] = C rho1, [2a] = A Bbar + B at the ring; "
                      "a0 = -(2B + AC)/(2(2 + A rho1)), b1 = a0 rho1^2 + C rho1",
        "rho": [float(rho1)], "A": [float(A)], "B": [float(B)], "C": [float(C)],
        "a": [float(a0), 0.0], "b": [0.0, float(b1)],
        "exact": {"a0": str(a0), "b1": str(b1)},
    }


def linear_wake(sigma_r, sigma_z, n_b0):
    # Linearised cold fluid in the quasistatic limit (Sec. II equations with
    # q = -1, m = 1, gamma - u_z = 1 + psi to first order):
    #   (d^2/dxi^2 + 1) dn = -n_b,  (grad_perp^2 - 1) psi = dn,  E_z = d psi / d xi.
    # Behind a Gaussian driver n_b = n_b0 exp(-r^2/2sr^2 - (xi-xi_d)^2/2sz^2):
    #   E_z(xi, 0) = n_b0 sqrt(2 pi) sz exp(-sz^2/2) F(0) cos(xi - xi_d),
    #   F(0) = int_0^inf r K0(r) exp(-r^2/2sr^2) dr = (sr^2/2) exp(sr^2/2) E1(sr^2/2).
    x = 0.5 * sigma_r ** 2
    f_closed = x * math.exp(x) * special.exp1(x)
    f_quad, _ = integrate.quad(lambda r: r * special.k0(r) * math.exp(-r * r / (2 * sigma_r ** 2)),
                               0.0, math.inf, epsabs=1e-14, epsrel=1e-13, limit=400)
    amp = n_b0 * math.sqrt(2 * math.pi) * sigma_z * math.exp(-0.5 * sigma_z ** 2) * f_closed
    return {"sigma_r": sigma_r, "sigma_z": sigma_z, "n_b0": n_b0,
            "F0_closed": f_closed, "F0_quadrature": f_quad, "Ez_axis_amplitude": amp}


def main():
    with open(os.path.join(HERE, "one_ring_bp.json"), "w") as f:
        json.dump(one_ring_bp(), f, indent=1)
    lin = {
        "citation": "linearised Sec. II model (Eqs. maxwell_qsa, lorentz_gauge, phi_b_eq_1, "
                    "cold_plasma_constant); E_z = -d psi/d zeta with zeta = -xi",
        "derivation": "(d_xi^2+1) dn = -n_b, (grad_perp^2-1) psi = dn, Green's function "
                      "-K0/(2 pi); E_z(xi,0) = n_b0 sqrt(2pi) sz e^{-sz^2/2} F(0) cos(xi-xi_d) "
                      "far behind the driver",
        "cases": [linear_wake(0.5, 1.0, 0.05), linear_wake(0.5, 1.0, 0.005),
                  linear_wake(0.3, 0.6, 0.005)],
    }
    with open(os.path.join(HERE, "linear_wake.json"), "w") as f:
        json.dump(lin, f, indent=1)


if __name__ == "__main__":
    main()
