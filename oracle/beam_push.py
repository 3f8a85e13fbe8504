"""FP64 numpy oracle of the beam push in the wake fields.

TEST INFRASTRUCTURE ONLY: used by tests/ (and nothing in the product).

Between two wake solves the beam macroparticles move over a time step dt in
the fields the wake gave at their positions; the paper's code integrates
this motion with the Boris method or fourth-order Runge-Kutta (Sec. V,
"Integration into Wake-T").  This is the Boris method, written from its
definition, in the paper's normalised units (time 1/omega_p, lengths 1/k_p,
momenta u = p / (m c), fields in m c omega_p / e):

  u-  = u + h E                      h = q dt / (2 m)
  t   = h B / gamma(u-),   s = 2 t / (1 + |t|^2)
  u'  = u- + u- x t
  u+  = u- + u' x s                  (rotation about B, |u+| = |u-|)
  u_new = u+ + h E
  x_new = x + dt u_new / gamma(u_new)
  xi_new = xi + dt (1 - u_z,new / gamma(u_new))   (xi = c t - z)

The axisymmetric wake fields at a particle at (x, y), r = |(x, y)|: E_z, and
E_r = W_r + B_theta (W_r = E_r - B_theta is what the wake reports), B_theta;
in Cartesian components E = (E_r x/r, E_r y/r, E_z), B = (-B_theta y/r,
B_theta x/r, 0), and E = (0, 0, E_z), B = 0 on the axis.
"""
from __future__ import annotations

from typing import Dict

import numpy as np


def boris_step(u: np.ndarray, E: np.ndarray, B: np.ndarray, h) -> np.ndarray:
    """One Boris momentum update.  u, E, B: arrays of shape (3, n);
    h = q dt / (2 m) (scalar or (n,))."""
    um = u + h * E
    gm = np.sqrt(1.0 + np.sum(um * um, axis=0))
    t = h * B / gm
    s = 2.0 * t / (1.0 + np.sum(t * t, axis=0))
    up = um + np.cross(um, t, axis=0)
    upl = um + np.cross(up, s, axis=0)
    return upl + h * E


def cartesian_fields(x, y, ez, wr, bt):
    """(E, B) of shape (3, n) from the wake's E_z, W_r, B_theta at (x, y)."""
    x, y, ez, wr, bt = (np.asarray(a, dtype=np.float64) for a in (x, y, ez, wr, bt))
    r = np.hypot(x, y)
    on_axis = r == 0.0
    rs = np.where(on_axis, 1.0, r)
    c = np.where(on_axis, 0.0, x / rs)
    s = np.where(on_axis, 0.0, y / rs)
    er = wr + bt
    E = np.stack([er * c, er * s, ez])
    B = np.stack([-bt * s, bt * c, np.zeros_like(bt)])
    return E, B


def push(state: Dict[str, np.ndarray], ez, wr, bt, q, dt: float) -> Dict[str, np.ndarray]:
    """One time step of every particle: state holds x, y, xi, ux, uy, uz
    (float64 arrays); q the charge per particle or scalar (mass 1: electrons
    or positrons).  Returns the new state (r = |(x, y)| added)."""
    E, B = cartesian_fields(state["x"], state["y"], ez, wr, bt)
    u = np.stack([state["ux"], state["uy"], state["uz"]]).astype(np.float64)
    h = 0.5 * np.asarray(q, dtype=np.float64) * dt
    un = boris_step(u, E, B, h)
    g = np.sqrt(1.0 + np.sum(un * un, axis=0))
    out = {"x": state["x"] + dt * un[0] / g, "y": state["y"] + dt * un[1] / g,
           "xi": state["xi"] + dt * (1.0 - un[2] / g), "ux": un[0], "uy": un[1], "uz": un[2]}
    out["r"] = np.hypot(out["x"], out["y"])
    return out
