"""Phase-equilibrium oracle: PT flash, pure-component coexistence, slab-state pressure.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper compares every equilibrated lattice with "a flash calculation ... using
the relevant EOS" (Sections V.A-V.C) but prints no flash algorithm.  This module is
the standard textbook procedure, written independently of the lattice code:

* bulk-phase molar volumes are real roots of the cubic EOS at (p, x)
  (``eos.volume_roots``): liquid = smallest, vapour = largest;
* fugacity coefficients use the textbook phi-forms of Appendix C
  (Eqs. eqfugvdW / eqfugSRK / eqfugPR), valid because bulk pressures are positive;
* Wilson K-values start the iteration; Rachford-Rice gives the vapour mole
  fraction beta (negative flash allowed, so beta may leave [0, 1]);
* successive substitution K_i <- phi_i^L / phi_i^V until max |d ln K| < 1e-12
  (fugacity equality, the iso-fugacity criterion of Section V.D).

``pure_coexistence`` is the N = 1 case: the saturation pressure at which the
liquid and vapour roots have equal fugacity, which is the Maxwell equal-area
construction (pinned by quadrature in tests/test_oracle_flash.py).

``slab_state`` picks the pressure at which a feed z splits into phases occupying
a prescribed vapour volume fraction S_V (Section V.B uses S_V = 0.5 for every
run); the paper leaves open how that pressure is found, the reading used here is
bisection on p of S_V(p) - S_V.

Pins: fugacity equality and material balance to round-off; pure limit equals the
Maxwell pair; physical-unit C2/n-C5 at 387.70 K against the fugacities printed in
Table tabFug (tests/golden/tabFug_c2c5_387K.json).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq

from .eos import Mixture, ln_phi_textbook, pressure_from_volume, volume_roots, lnf_density_form


def phase_volume(mix: Mixture, p: float, x: np.ndarray, phase: str) -> float:
    roots = volume_roots(mix, p, x)
    if roots.size == 0:
        raise ArithmeticError("no physical volume root")
    return float(roots[0] if phase == "liquid" else roots[-1])


def wilson_K(mix: Mixture, p: float) -> np.ndarray:
    """Wilson's correlation, only a starting guess for the K-values."""
    return (mix.Pc / p) * np.exp(5.373 * (1.0 + mix.omega) * (1.0 - mix.Tc / mix.T))


def rachford_rice(z: np.ndarray, K: np.ndarray) -> float:
    """Root beta of sum_i z_i (K_i - 1) / (1 + beta (K_i - 1)) = 0 inside the window
    where every 1 + beta (K_i - 1) > 0 (negative flash allowed)."""
    Km1 = K - 1.0
    if np.all(Km1 > 0) or np.all(Km1 < 0):
        raise ArithmeticError("Rachford-Rice has no root: all K on one side of 1")
    lo = 1.0 / (1.0 - K.max())
    hi = 1.0 / (1.0 - K.min())
    span = hi - lo
    f = lambda beta: float(np.sum(z * Km1 / (1.0 + beta * Km1)))
    eps = 1e-14 * max(1.0, abs(span))
    return brentq(f, lo + eps, hi - eps, xtol=1e-17, rtol=1e-15, maxiter=500)


def flash(mix: Mixture, p: float, z, K0=None, tol: float = 1e-12, maxiter: int = 20000) -> dict:
    """Two-phase PT flash by successive substitution.  Returns a dict with beta, x, y,
    liquid/vapour molar volumes vL, vV and molar densities rtL = x / vL, rtV = y / vV."""
    z = np.asarray(z, dtype=np.float64)
    z = z / z.sum()
    K = wilson_K(mix, p) if K0 is None else np.asarray(K0, dtype=np.float64).copy()
    converged = False
    last_step = np.inf
    for it in range(maxiter):
        beta = rachford_rice(z, K)
        x = z / (1.0 + beta * (K - 1.0))
        y = K * x
        x = x / x.sum()
        y = y / y.sum()
        vL = phase_volume(mix, p, x, "liquid")
        vV = phase_volume(mix, p, y, "vapor")
        lnK_new = ln_phi_textbook(mix, vL, x) - ln_phi_textbook(mix, vV, y)
        step = np.max(np.abs(lnK_new - np.log(K)))
        K = np.exp(lnK_new)
        if step < tol:
            converged = True
            break
        # stagnation at round-off: the update no longer shrinks
        if step < 1e3 * tol and it > 0 and step >= last_step:
            converged = True
            break
        last_step = step
        if np.max(np.abs(np.log(K))) < 1e-6:
            raise ArithmeticError("flash collapsed to the trivial solution")
    beta = rachford_rice(z, K)
    x = z / (1.0 + beta * (K - 1.0))
    y = K * x
    x = x / x.sum()
    y = y / y.sum()
    vL = phase_volume(mix, p, x, "liquid")
    vV = phase_volume(mix, p, y, "vapor")
    return dict(p=p, beta=beta, x=x, y=y, vL=vL, vV=vV, rtL=x / vL, rtV=y / vV, K=K,
                iterations=it + 1, converged=converged)


def vapour_volume_fraction(res: dict) -> float:
    """S_V = beta vV / (beta vV + (1 - beta) vL) (the saturation of Eq. eqInit)."""
    b = res["beta"]
    return b * res["vV"] / (b * res["vV"] + (1.0 - b) * res["vL"])


def pure_coexistence(mix: Mixture, tol: float = 1e-14) -> dict:
    """Saturation state of a single component (N = 1): the pressure where the liquid
    and vapour roots of the EOS have equal ln f (equivalently equal chemical potential,
    the Maxwell construction).  Returns p_sat, vL, vV, rtL, rtV."""
    assert mix.n == 1
    x = np.array([1.0])
    # bracket: pressures between the two spinodals have three real roots
    vs = np.geomspace(mix.b[0] * 1.0001, mix.b[0] * 1e4, 200001)
    ps = pressure_from_volume(mix, vs, x)
    dp = np.diff(ps)
    ext = np.where(np.sign(dp[1:]) != np.sign(dp[:-1]))[0] + 1
    if ext.size < 2:
        raise ArithmeticError("supercritical: no van der Waals loop")
    p_min, p_max = ps[ext[0]], ps[ext[1]]
    lo = max(p_min, 0.0) + 1e-12 * abs(p_max)
    hi = p_max * (1 - 1e-12)

    def g(p):
        vL = phase_volume(mix, p, x, "liquid")
        vV = phase_volume(mix, p, x, "vapor")
        return float(ln_phi_textbook(mix, vL, x)[0] - ln_phi_textbook(mix, vV, x)[0])

    if lo <= 0.0 or g(lo) * g(hi) > 0:
        lo = max(p_min, hi * 1e-12)
    psat = brentq(g, lo, hi, xtol=1e-300, rtol=max(tol, 1e-15), maxiter=500)
    vL = phase_volume(mix, psat, x, "liquid")
    vV = phase_volume(mix, psat, x, "vapor")
    return dict(p=psat, vL=vL, vV=vV, rtL=1.0 / vL, rtV=1.0 / vV)


def slab_state(mix: Mixture, z, S_V: float = 0.5, p_lo: float = None, p_hi: float = None,
               n_scan: int = 80) -> dict:
    """Pressure at which feed z, flashed at the mixture temperature, gives vapour volume
    fraction S_V, and the flash result there (reading of Section V.B's "S_V = 0.5")."""
    z = np.asarray(z, dtype=np.float64)
    z = z / z.sum()
    psat_w = mix.Pc * np.exp(5.373 * (1.0 + mix.omega) * (1.0 - mix.Tc / mix.T))
    if p_lo is None:
        p_lo = 0.2 / np.sum(z / psat_w)
    if p_hi is None:
        p_hi = 5.0 * np.sum(z * psat_w)
    grid = np.geomspace(p_lo, p_hi, n_scan)

    def split(r):
        # beta vV (1 - S_V) - S_V (1 - beta) vL: zero exactly at the requested volume
        # fraction, and monotone through beta = 0 (unlike S_V itself under negative flash)
        return r["beta"] * r["vV"] * (1.0 - S_V) - S_V * (1.0 - r["beta"]) * r["vL"]

    prev = None
    K = None
    bracket = None
    for p in grid:
        try:
            r = flash(mix, p, z, K0=K, maxiter=400)
            if not r["converged"]:
                raise ArithmeticError("scan flash did not converge")
            s = split(r)
            K = r["K"]
        except (ArithmeticError, ValueError):
            prev = None
            K = None
            continue
        if prev is not None and prev[1] * s <= 0:
            bracket = (prev[0], p, prev[2])
            break
        prev = (p, s, r["K"])
    if bracket is None:
        raise ArithmeticError("could not bracket the slab-state pressure")
    a, b, Kb = bracket
    Kc = [Kb]

    def h(p):
        r = flash(mix, p, z, K0=Kc[0])
        Kc[0] = r["K"]
        return split(r)

    p_star = brentq(h, a, b, xtol=1e-300, rtol=1e-15, maxiter=300)
    r = flash(mix, p_star, z, K0=Kc[0])
    r["S_V"] = vapour_volume_fraction(r)
    return r


def bubble_point_from_liquid(mix: Mixture, xL, p0: float, y0=None, tol: float = 1e-13,
                             maxiter: int = 20000) -> dict:
    """Given the liquid composition xL at the mixture temperature, find the pressure p and
    the incipient vapour composition y with f_i^L = f_i^V for all i (bubble-point problem).
    Used to compare a ternary lattice's vapour with the state in equilibrium with its
    own bulk liquid.  Fixed-point iteration y_i <- K_i x_i, p <- p * sum_i K_i x_i."""
    xL = np.asarray(xL, dtype=np.float64)
    xL = xL / xL.sum()
    p = float(p0)
    y = (wilson_K(mix, p) * xL) if y0 is None else np.asarray(y0, dtype=np.float64)
    y = y / y.sum()
    for it in range(maxiter):
        vL = phase_volume(mix, p, xL, "liquid")
        vV = phase_volume(mix, p, y, "vapor")
        K = np.exp(ln_phi_textbook(mix, vL, xL) - ln_phi_textbook(mix, vV, y))
        s = float(np.sum(K * xL))
        y_new = K * xL / s
        p_new = p * s
        done = abs(s - 1.0) < tol and np.max(np.abs(y_new - y)) < tol
        y, p = y_new, p_new
        if done:
            break
    vL = phase_volume(mix, p, xL, "liquid")
    vV = phase_volume(mix, p, y, "vapor")
    return dict(p=p, x=xL, y=y, vL=vL, vV=vV, rtL=xL / vL, rtV=y / vV, iterations=it + 1)


def lnf_at(mix: Mixture, rt) -> np.ndarray:
    """ln f_i of a bulk state given by its molar densities (density form, Eq. eqfugupdatePR)."""
    return lnf_density_form(mix, np.asarray(rt, dtype=np.float64))
