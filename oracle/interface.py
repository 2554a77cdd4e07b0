"""Interface measures used by the paper's dynamic validation (Section V.E).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``interfacial_tension`` -- Eq. eqMCsigma: for a flat interface normal to x,
  sigma = integral over x of sum_ij kappa_ij (d rho~_i / dx)(d rho~_j / dx), with
  kappa_ij = sqrt(kappa_i kappa_j) (Eq. eqkappa).  On a lattice profile the
  derivative is the central difference of Eq. eq1stder and the integral a sum over
  nodes (unit spacing).  A periodic slab has two interfaces; ``n_interfaces``
  divides by their number.
* ``lamb_period`` -- Eq. eqPeriod: the period of mode n of a droplet oscillating
  under surface tension, T_a = 2 pi [n (n^2 - 1) sigma / (rho_L R_e^3)]^(-1/2), with
  R_e = sqrt(R_max R_min) = R_0 sqrt(h) for the ellipse of Eq. eqInit2D.
* ``crossing_radius`` -- the droplet radius of Section V.E: the distance from the
  centre to where the density profile along an axis crosses (rho_V + rho_L) / 2,
  located by linear interpolation between the two nodes around the crossing.

Pins (tests/test_oracle_interface.py): the tanh profile of Eq. eqInit has the closed
form integral 8 b^2 / (3 W) per interface for amplitude b and width W (the central
difference converges to it at second order); the period formula against
hand-evaluated numbers; the crossing radius of a sampled tanh profile.
"""
import numpy as np


def interfacial_tension(rt_profile: np.ndarray, kappa, n_interfaces: int = 1) -> float:
    """Eq. eqMCsigma on a periodic 1-D molar-density profile rt_profile[N][nx]."""
    rt = np.asarray(rt_profile, dtype=np.float64)
    d = 0.5 * (np.roll(rt, -1, axis=1) - np.roll(rt, 1, axis=1))
    k = np.sqrt(np.outer(kappa, kappa))
    return float(np.einsum("ij,ix,jx->", k, d, d)) / n_interfaces


def lamb_period(sigma: float, rho_L: float, R_e: float, n: int = 2) -> float:
    """Eq. eqPeriod."""
    return 2.0 * np.pi / np.sqrt(n * (n * n - 1) * sigma / (rho_L * R_e ** 3))


def crossing_radius(profile: np.ndarray, centre: float, level: float) -> float:
    """Distance from `centre` (a node index) outwards (increasing index) to the first
    crossing of `level` by a profile that is above it at the centre; NaN if none."""
    p = np.asarray(profile, dtype=np.float64)
    i0 = int(round(centre))
    for k in range(i0, len(p) - 1):
        if p[k] >= level > p[k + 1]:
            return k + (p[k] - level) / (p[k] - p[k + 1]) - centre
    return float("nan")
