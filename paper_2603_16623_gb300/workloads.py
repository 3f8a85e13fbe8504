"""Seeded synthetic inputs for the gridless quasistatic wake solver.

This module only *draws* inputs: ring-cell edges of the plasma column and
macroparticle beams (xi, r, weight, charge sign).  It holds none of the
method's arithmetic (no ring weights, no slice binning, no fields); both the
CUDA path and the CPU oracle turn these arrays into their own state.

Units are the paper's normalised plasma units (Sec. II): lengths in k_p^-1,
densities in n0, beam weights in n0 k_p^-3 (number of real particles a
macroparticle stands for).  xi = -zeta grows towards the back of the window;
the driver sits near the front (xi = 0 is the head of the window).

Workloads (the paper prints no datasets; these stand in for its physical
setups, with the shapes of Sec. IV-V):
  * linear  : 200 uniform rings on (0,5], weak Gaussian driver n_b0=0.05
  * blowout : 2000 rings on (0,6], x20 refinement inside r<0.05, strong driver
              n_b0=10 plus a narrow witness 3 k_p^-1 behind (collider-like)
  * batched : 256 independent wakes, log-uniform ring counts in [500, 8000]
  * large   : 65,536 log-spaced rings down to r=1e-5, 2M + 2M particles
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Tuple

import numpy as np

TRUNC_SIGMAS = 4.0  # Gaussian beams are truncated at +-4 sigma_z in xi


@dataclass
class Beam:
    xi: np.ndarray      # float64 [n] longitudinal position (xi = -zeta)
    r: np.ndarray       # float64 [n] radius, >= 0
    w: np.ndarray       # float64 [n] weight (real particles, n0 k_p^-3 units), > 0
    q: float = -1.0     # charge sign of the species (-1: electrons)

    @property
    def n(self) -> int:
        return int(self.xi.shape[0])


@dataclass
class Wake:
    """One independent wake problem: plasma column, beams and the xi grid."""
    name: str
    edges: np.ndarray           # float64 [n_rings+1], edges[0]=0, increasing
    beams: List[Beam]
    dxi: float
    n_steps: int
    density: float = 1.0
    # mobile ions (charge Z, mass M in electron masses; M = inf: ion rings
    # that never move) as a second ring species on the same edges; None: an
    # immobile ion column
    ions: Optional[Tuple[float, float]] = None
    # radial density profile: density per cell (uniform within a cell), in
    # place of the uniform `density`; needs ion rings (`ions`)
    cell_density: Optional[np.ndarray] = None
    # ring integrator: "ab2" (Sec. III) or "rk4"
    integrator: str = "ab2"
    # beam-plasma coupling: 0 = gridless (fields at each beam particle);
    # > 0 = adaptive beam grids of this many radial cells per beam (Sec. IV)
    grid_nr: int = 0
    # > 0: the grids' fixed extent (a regular intermediate grid over [0,
    # grid_rmax] that every beam particle lies in); 0: adaptive
    grid_rmax: float = 0.0

    @property
    def n_rings(self) -> int:
        return int(self.edges.shape[0] - 1)

    @property
    def n_beam(self) -> int:
        return sum(b.n for b in self.beams)

    @property
    def ring_slices(self) -> int:
        return self.n_rings * self.n_steps


# ----------------------------------------------------------------------------
# ring-cell edges
# ----------------------------------------------------------------------------
def parabolic_profile(edges: np.ndarray, n0: float = 1.0, w0: float = 2.0) -> np.ndarray:
    """Density per cell of the parabolic channel n0 (1 + 4 r^2 / w0^4) (the
    paper's guiding profile with k_p = 1), sampled at the cell centres."""
    c = 0.5 * (edges[1:] + edges[:-1])
    return n0 * (1.0 + 4.0 * c * c / w0 ** 4)


def edges_uniform(n_rings: int, r_max: float) -> np.ndarray:
    return np.linspace(0.0, r_max, n_rings + 1, dtype=np.float64)


def edges_refined(n_inner: int, r_inner: float, n_outer: int, r_max: float) -> np.ndarray:
    """n_inner equal cells on (0, r_inner], then n_outer equal cells up to r_max."""
    inner = np.linspace(0.0, r_inner, n_inner + 1)
    outer = np.linspace(r_inner, r_max, n_outer + 1)[1:]
    return np.concatenate([inner, outer]).astype(np.float64)


def edges_geometric(n_rings: int, r_min: float, r_max: float) -> np.ndarray:
    """edges 0, then n_rings geometric edges from r_min to r_max."""
    geo = np.geomspace(r_min, r_max, n_rings)
    return np.concatenate([[0.0], geo]).astype(np.float64)


# ----------------------------------------------------------------------------
# beams
# ----------------------------------------------------------------------------
def gaussian_charge(n_b0: float, sigma_r: float, sigma_z: float) -> float:
    """Real particles in a Gaussian bunch of peak density n_b0, truncated at
    +-TRUNC_SIGMAS sigma_z (n0 k_p^-3 units)."""
    full = n_b0 * (2.0 * math.pi) ** 1.5 * sigma_r ** 2 * sigma_z
    return full * math.erf(TRUNC_SIGMAS / math.sqrt(2.0))


def gaussian_beam(n_mp: int, n_b0: float, sigma_r: float, sigma_z: float,
                  xi_c: float, seed: int, q: float = -1.0,
                  total: float | None = None) -> Beam:
    """Cold Gaussian bunch: r from a 2-D Gaussian of rms sigma_r per axis,
    xi from N(xi_c, sigma_z) truncated to +-4 sigma_z, equal weights."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = 1.0 - rng.random(n_mp)                     # (0, 1]
    r = sigma_r * np.sqrt(-2.0 * np.log(u))
    xi = np.empty(n_mp)
    filled = 0
    while filled < n_mp:
        z = rng.standard_normal(2 * (n_mp - filled) + 16)
        z = z[np.abs(z) <= TRUNC_SIGMAS][: n_mp - filled]
        xi[filled:filled + z.shape[0]] = xi_c + sigma_z * z
        filled += z.shape[0]
    n_real = gaussian_charge(n_b0, sigma_r, sigma_z) if total is None else total
    w = np.full(n_mp, n_real / n_mp)
    return Beam(xi=xi, r=r, w=w, q=q)


def sampled_gaussian_beam(dxi: float, n_steps: int, n_b0: float, sigma_r: float,
                          sigma_z: float, xi_c: float, n_r: int = 64,
                          q: float = -1.0) -> Beam:
    """Noise-free Gaussian bunch for convergence studies: at every slice
    centre xi_n = n dxi within +-4 sigma_z of xi_c, n_r particles at the
    radial quantiles of the 2-D Gaussian, each carrying 1/n_r of the slab's
    real particles n_b0 exp(-(xi_n-xi_c)^2 / 2 sigma_z^2) 2 pi sigma_r^2 dxi."""
    n = np.arange(n_steps)
    xi_n = n * dxi
    keep = np.abs(xi_n - xi_c) <= TRUNC_SIGMAS * sigma_z
    xi_n = xi_n[keep]
    quant = (np.arange(n_r) + 0.5) / n_r
    r_j = sigma_r * np.sqrt(-2.0 * np.log(1.0 - quant))
    slab = n_b0 * np.exp(-0.5 * ((xi_n - xi_c) / sigma_z) ** 2) * 2.0 * math.pi * sigma_r ** 2 * dxi
    xi = np.repeat(xi_n, n_r)
    r = np.tile(r_j, xi_n.shape[0])
    w = np.repeat(slab / n_r, n_r)
    return Beam(xi=xi, r=r, w=w, q=q)


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------
def linear_wake(n_b0: float = 0.05, n_mp: int = 20_000, seed: int = 1,
                n_rings: int = 200, dxi: float = 0.02, n_steps: int = 1000) -> Wake:
    """200 uniform rings on (0,5]; driver sigma_r=0.5, sigma_z=1, centre xi=4."""
    drv = gaussian_beam(n_mp, n_b0, 0.5, 1.0, 4.0, seed)
    return Wake("linear", edges_uniform(n_rings, 5.0), [drv], dxi, n_steps)


def blowout_wake(n_drv: int = 200_000, n_wit: int = 50_000,
                 dxi: float = 0.005, n_steps: int = 4000) -> Wake:
    """2000 rings on (0,6]: 288 cells of 0.05/288 inside 0.05 (x20 refined),
    then 1712 cells of 5.95/1712.  Driver sigma_r=0.1, sigma_z=0.5, n_b0=10 at
    xi=2; witness sigma_r=1e-3, sigma_z=0.25 at xi=5 carrying 0.42 of the
    driver charge (the 833 pC : 2 nC ratio of the collider stage in Sec. V)."""
    edges = edges_refined(288, 0.05, 1712, 6.0)
    drv = gaussian_beam(n_drv, 10.0, 0.1, 0.5, 2.0, seed=2)
    q_drv = gaussian_charge(10.0, 0.1, 0.5)
    wit = gaussian_beam(n_wit, 0.0, 1e-3, 0.25, 5.0, seed=3, total=0.42 * q_drv)
    return Wake("blowout", edges, [drv, wit], dxi, n_steps)


@dataclass(frozen=True)
class BatchedParams:
    """The drawn parameters of one batched-workload member (no arrays)."""
    n_rings: int
    n_b0: float
    sigma_r: float
    sigma_z: float
    n_mp: int
    n_steps: int
    r_max: float


def batched_params(k: int) -> BatchedParams:
    """Member k's parameters, seed 3000+k: ring count log-uniform in [500,
    8000], n_b0 ~ U[0.05, 20], sigma_r ~ U[0.05, 1], sigma_z ~ U[0.3, 2],
    50k-500k macroparticles, 1000-6000 steps of 0.01; uniform spacing out to
    max(6, 3 x (2 sqrt(n_b0) sigma_r)).  Cheap: a request stream can be
    planned (sizes, work) without drawing any beam."""
    rng = np.random.Generator(np.random.PCG64(3000 + k))
    n_rings = int(math.floor(math.exp(rng.uniform(math.log(500), math.log(8000)))))
    n_b0 = rng.uniform(0.05, 20.0)
    sigma_r = rng.uniform(0.05, 1.0)
    sigma_z = rng.uniform(0.3, 2.0)
    n_mp = int(rng.integers(50_000, 500_001))
    n_steps = int(rng.integers(1000, 6001))
    r_max = max(6.0, 3.0 * 2.0 * math.sqrt(n_b0) * sigma_r)
    return BatchedParams(n_rings, n_b0, sigma_r, sigma_z, n_mp, n_steps, r_max)


def batched_wake(k: int) -> Wake:
    """Member k (0..255) of the batched workload (parameters from
    batched_params(k)); the driver's particles drawn with seed 10000+k."""
    p = batched_params(k)
    drv = gaussian_beam(p.n_mp, p.n_b0, p.sigma_r, p.sigma_z, TRUNC_SIGMAS * p.sigma_z,
                        seed=10_000 + k)
    return Wake(f"batched[{k}]", edges_uniform(p.n_rings, p.r_max), [drv], 0.01, p.n_steps)


def batched_workload(n_wakes: int = 256) -> List[Wake]:
    return [batched_wake(k) for k in range(n_wakes)]


def large_wake(n_rings: int = 65_536, n_drv: int = 2_000_000, n_wit: int = 2_000_000,
               dxi: float = 0.002, n_steps: int = 8000) -> Wake:
    """65,536 rings: edge 0, then geometric edges from 1e-5 to 6.  Driver as
    in the blowout wake; witness sigma_r=1e-4.  Seed 5."""
    edges = edges_geometric(n_rings, 1e-5, 6.0)
    drv = gaussian_beam(n_drv, 10.0, 0.1, 0.5, 2.0, seed=5)
    q_drv = gaussian_charge(10.0, 0.1, 0.5)
    wit = gaussian_beam(n_wit, 0.0, 1e-4, 0.25, 5.0, seed=6, total=0.42 * q_drv)
    return Wake("large", edges, [drv, wit], dxi, n_steps)


def random_ring_state(n_rings: int, seed: int, r_max: float = 3.0,
                      u_scale: float = 0.3, jitter: float = 0.15):
    """A perturbed plasma column for unit tests of the per-slice field
    evaluation: random cell edges on (0, r_max], ring radii at the cell
    centres moved by a relative Gaussian jitter (so radius order changes),
    Gaussian radial momenta.  Returns (edges, rho, u_r), rho by ring id."""
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = np.sort(rng.uniform(0.0, r_max, n_rings + 1))
    edges[0] = 0.0
    edges[-1] = r_max
    centre = 0.5 * (edges[1:] + edges[:-1])
    rho = np.abs(centre * (1.0 + jitter * rng.standard_normal(n_rings)))
    ur = u_scale * rng.standard_normal(n_rings)
    return edges, rho, ur
