"""Plain FP64 lattice Boltzmann step of the fugacity-based method (the oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

One call of ``step`` performs the nine-step procedure of Section III.B
(Implementation) on a periodic D2Q9 lattice, in that order, with whole-grid numpy
array operations and nothing fused or reordered:

 1. rho_i = sum_a g_{a,i};  rho = sum_i rho_i;  the first moment sum_a g_{a,i} e_a
 2. molar densities rho~_i = rho_i / M_i, rho~ = sum_i rho~_i, x_i = rho~_i / rho~
 3. mixing rules b_m, (a alpha)_m                    (Appendix C)
 4. pressure p from the EOS                           (Eq. eqPREOS / eqSRKEOS / eqvdwEOS)
 5. ln f_i, density-explicit form                     (Eq. eqfugupdatePR / SRK / VDW)
 6. mu_{I,i} = -sum_j sqrt(kappa_i kappa_j) lap(rho~_j)   (Eqs. eqChemPotI2, eqkappa, eq2ndder)
 7. F_i = -rho~_i RT grad ln f_i - rho~_i grad mu_{I,i}    (Eqs. eqforceFugLBM / eqforcefinal, eq1stder)
    then u = (1/rho) sum_i [sum_a g_{a,i} e_a + F_i / 2]  (the velocity of step 1)
 8. well-balanced equilibrium with rho_0 = 0 (Eq. eqLBEMCb) and forcing term (Eq. eqLBEMCfinal3)
 9. collision (Eq. eqLBEMCa) then streaming g_{a,i}(r + e_a) <- g*_{a,i}(r), periodic.

Readings where the paper is silent or ambiguous (each one is listed in the design
document of this repository):

* Step 1 computes u from the distributions "and body forces ... from the previous
  time step", before steps 6-7 compute this step's force.  Default
  ``velocity_force="lagged"`` takes that literally: u uses the total force
  sum_i F_i stored by the previous step (zero before the first step), while the
  forcing term F_{a,i} of step 8 uses this step's F_i.  ``"current"`` uses this
  step's force in u instead.  Both share every equilibrium state (u = 0, F = 0);
  the lagged form is the one that stays stable at the paper's kappa and density
  ratios (a linearised 1-D analysis of the tau = 1 update shows the current form
  losing stability once kappa rho~ exceeds about (1 - c^2) / 4).
* The paper's derivatives are 1-D central differences per axis (Eqs. eq1stder,
  eq2ndder): ``stencil="central"``.  ``stencil="isotropic"`` uses the D2Q9
  weighted stencils  grad h = (1/c_s^2) sum_a w_a e_a h(r + e_a)  and
  lap h = (2/c_s^2) sum_a w_a [h(r + e_a) - h(r)], which equal the central ones on
  any field that is uniform along y (every flat-slab case).
* The (1 - 1/(2 tau)) prefactor multiplies the whole F_{a,i} of Eq. eqLBEMCfinal3.
* rho_0 and rho_{0,i} of Eq. eqLBEMCb are one constant, 0.
* ``formulation="standard"`` is the variant Section VI (Discussion) allows: the
  standard LBE of Eq. eqLBE per component (equilibrium rho_i w_a [1 + ...], i.e.
  Eq. eqLBEMCb with rho_{0,i} = rho_i; forcing term of Eq. eqLBEfinal3, i.e.
  Eq. eqLBEMCfinal3 without its grad rho_i part) with the force of Eq. eqForceGen,
  which adds c_s^2 grad rho_i (mass density) to Eq. eqforcefinal.  Its flat-interface
  equilibria deviate slightly from the flash, as the paper says.
* The direction order below is a convention of this code, not of the paper.

Parity: the step-by-step transient is "parity unpinned" beyond the invariants
tests/test_oracle_lbm.py checks (exact mass conservation, an exactly stationary
uniform state, the moment identities of Eqs. eqLBEMCb and eqLBEMCfinal3 in exact
rational arithmetic, the single-component Maxwell limit, and flat-interface
equilibria against the flash oracle); nothing in the paper fixes transient values.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .eos import Mixture, lnf_density_form, mixing, molar_state, pressure

# D2Q9 velocities and weights; c_s^2 = 1/3, D = 2.
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
CS2 = 1.0 / 3.0
DIM = 2


class NonPhysicalState(ArithmeticError):
    """A node left the domain of the EOS: rho_i <= 0, rho~ b_m >= 1 or a non-finite value."""

    def __init__(self, what: str, comp: int, y: int, x: int):
        super().__init__(f"{what} at component {comp}, node (x={x}, y={y})")
        self.comp, self.y, self.x = comp, y, x


@dataclass
class Lattice:
    tau: float
    stencil: str = "isotropic"     # or "central"
    velocity_force: str = "lagged"  # or "current"
    rho0: float = 0.0
    formulation: str = "well_balanced"  # or "standard" (Eq. eqLBE with Eq. eqForceGen)


def neighbour(h: np.ndarray, dx: int, dy: int) -> np.ndarray:
    """h(r + (dx, dy)) on the periodic grid (last two axes are y, x)."""
    return np.roll(h, shift=(-dy, -dx), axis=(-2, -1))


def gradient(h: np.ndarray, stencil: str):
    """First derivatives (d/dx, d/dy) of a field: Eq. eq1stder, or the isotropic variant."""
    if stencil == "central":
        gx = (neighbour(h, 1, 0) - neighbour(h, -1, 0)) / 2.0
        gy = (neighbour(h, 0, 1) - neighbour(h, 0, -1)) / 2.0
        return gx, gy
    gx = np.zeros_like(h)
    gy = np.zeros_like(h)
    for a in range(1, 9):
        hn = neighbour(h, E[a, 0], E[a, 1])
        gx += W[a] * E[a, 0] * hn
        gy += W[a] * E[a, 1] * hn
    return gx / CS2, gy / CS2


def laplacian(h: np.ndarray, stencil: str) -> np.ndarray:
    """Laplacian of a field: Eq. eq2ndder along each axis, or the isotropic variant."""
    if stencil == "central":
        return (neighbour(h, 1, 0) + neighbour(h, -1, 0) + neighbour(h, 0, 1) + neighbour(h, 0, -1)
                - 4.0 * h)
    out = np.zeros_like(h)
    for a in range(1, 9):
        out += W[a] * (neighbour(h, E[a, 0], E[a, 1]) - h)
    return 2.0 * out / CS2


def equilibrium(rho_i: np.ndarray, ux: np.ndarray, uy: np.ndarray, rho0: float = 0.0,
                standard: bool = False) -> np.ndarray:
    """Well-balanced equilibrium of Eq. eqLBEMCb for every component and direction
    (standard=True: the equilibrium of Eq. eqLBE, rho_i w_a [1 + S]).

    rho_i has shape (N, ny, nx); the result has shape (N, 9, ny, nx).
    """
    n = rho_i.shape[0]
    geq = np.empty((n, 9) + rho_i.shape[1:], dtype=np.float64)
    usq = ux * ux + uy * uy
    for a in range(9):
        eu = E[a, 0] * ux + E[a, 1] * uy
        S = eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - usq / (2.0 * CS2)
        if standard:
            geq[:, a] = W[a] * rho_i * (1.0 + S)
        elif a == 0:
            geq[:, 0] = rho_i - (1.0 - W[0]) * rho0 + W[0] * rho_i * S
        else:
            geq[:, a] = W[a] * rho0 + W[a] * rho_i * S
    return geq


def forcing_term(Fx, Fy, grx, gry, ux, uy) -> np.ndarray:
    """Well-balanced multicomponent forcing term F_{a,i} of Eq. eqLBEMCfinal3.

    Fx, Fy: component body forces (N, ny, nx); grx, gry: gradients of the component
    mass densities rho_i; ux, uy: barycentric velocity.
    """
    n = Fx.shape[0]
    out = np.empty((n, 9) + Fx.shape[1:], dtype=np.float64)
    for a in range(9):
        ex, ey = E[a]
        eu = ex * ux + ey * uy
        e2 = ex * ex + ey * ey
        # F_i . w_a [ (e_a - u)/c_s^2 + (u.e_a) e_a / c_s^4 ]
        tF = ((ex - ux) * Fx + (ey - uy) * Fy) / CS2 + eu * (ex * Fx + ey * Fy) / (CS2 * CS2)
        # grad rho_i . w_a [ -u + (u.e_a) e_a / c_s^2 + (e_a^2/c_s^2 - D) u / 2 ]
        c = 0.5 * (e2 / CS2 - DIM)
        tG = (-ux * grx - uy * gry) + eu * (ex * grx + ey * gry) / CS2 + c * (ux * grx + uy * gry)
        out[:, a] = W[a] * (tF + tG)
    return out


def check_physical(mix: Mixture, rho: np.ndarray, rt: np.ndarray) -> None:
    """Raise NonPhysicalState at the first node outside the EOS domain (rho_i > 0, rho~ b_m < 1)."""
    bad = ~(rho > 0.0)
    if bad.any():
        i, y, x = np.argwhere(bad)[0]
        raise NonPhysicalState("non-positive or non-finite density", int(i), int(y), int(x))
    _, x_frac, _ = molar_state(mix, rt)
    bm, _, _ = mixing(mix, x_frac)
    packed = bm * np.sum(rt, axis=0)
    bad = ~(packed < 1.0)
    if bad.any():
        y, x = np.argwhere(bad)[0]
        raise NonPhysicalState("packing fraction rho~ b_m >= 1", 0, int(y), int(x))


def macroscopic(g: np.ndarray, mix: Mixture, lat: Lattice, F_prev: np.ndarray = None) -> dict:
    """Steps 1-7 of Section III.B at every node.  g has shape (N, 9, ny, nx) and holds the
    distributions after streaming; F_prev (2, ny, nx) is the total body force sum_i F_i of
    the previous step (used in u under the "lagged" reading; None means zero).
    Returns the densities, ln f, forces and velocity."""
    # step 1
    rho = g.sum(axis=1)
    jx = np.tensordot(E[:, 0].astype(np.float64), g, axes=(0, 1))
    jy = np.tensordot(E[:, 1].astype(np.float64), g, axes=(0, 1))
    rho_tot = rho.sum(axis=0)
    # step 2
    M = mix.M.reshape(-1, 1, 1)
    rt = rho / M
    check_physical(mix, rho, rt)
    # steps 3-5
    p = pressure(mix, rt)
    lnf = lnf_density_form(mix, rt)
    # step 6: interface chemical potential mu_I,i = -sum_j kappa_ij lap(rho~_j)
    kappa_ij = np.sqrt(np.outer(mix.kappa, mix.kappa))
    lap_rt = np.stack([laplacian(rt[j], lat.stencil) for j in range(mix.n)])
    muI = -np.tensordot(kappa_ij, lap_rt, axes=(1, 0))
    # step 7: F_i = -rho~_i RT grad ln f_i - rho~_i grad mu_I,i (+ c_s^2 grad rho_i in the
    # standard formulation, Eq. eqForceGen)
    Fx = np.empty_like(rho)
    Fy = np.empty_like(rho)
    grx = np.empty_like(rho)
    gry = np.empty_like(rho)
    for i in range(mix.n):
        glx, gly = gradient(lnf[i], lat.stencil)
        gmx, gmy = gradient(muI[i], lat.stencil)
        grx[i], gry[i] = gradient(rho[i], lat.stencil)
        Fx[i] = -rt[i] * mix.RT * glx - rt[i] * gmx
        Fy[i] = -rt[i] * mix.RT * gly - rt[i] * gmy
        if lat.formulation == "standard":
            Fx[i] = Fx[i] + CS2 * grx[i]
            Fy[i] = Fy[i] + CS2 * gry[i]
    # velocity of step 1: u = (1/rho) sum_i [sum_a g_{a,i} e_a + F_i / 2]
    if lat.velocity_force == "current":
        Fu_x, Fu_y = Fx.sum(axis=0), Fy.sum(axis=0)
    elif F_prev is None:
        Fu_x = Fu_y = np.zeros_like(rho_tot)
    else:
        Fu_x, Fu_y = F_prev[0], F_prev[1]
    ux = (jx.sum(axis=0) + 0.5 * Fu_x) / rho_tot
    uy = (jy.sum(axis=0) + 0.5 * Fu_y) / rho_tot
    F_tot = np.stack([Fx.sum(axis=0), Fy.sum(axis=0)])
    return dict(rho=rho, rt=rt, p=p, lnf=lnf, muI=muI, Fx=Fx, Fy=Fy, grx=grx, gry=gry, ux=ux, uy=uy, F_tot=F_tot)


def step(g: np.ndarray, mix: Mixture, lat: Lattice, F_prev: np.ndarray = None,
         return_macro: bool = False):
    """One full time step (steps 1-9).

    Returns (g_new, F_tot): the new post-streaming distributions and the total body force
    sum_i F_i of this step (shape (2, ny, nx)), which the next step's velocity uses under
    the "lagged" reading.  With return_macro, also the dict of ``macroscopic``."""
    m = macroscopic(g, mix, lat, F_prev)
    # step 8
    if lat.formulation == "standard":
        # Eq. eqLBE per component: rho_{0,i} = rho_i, forcing without the grad rho_i part
        geq = equilibrium(m["rho"], m["ux"], m["uy"], standard=True)
        zero = np.zeros_like(m["rho"])
        Fa = forcing_term(m["Fx"], m["Fy"], zero, zero, m["ux"], m["uy"])
    else:
        geq = equilibrium(m["rho"], m["ux"], m["uy"], lat.rho0)
        Fa = forcing_term(m["Fx"], m["Fy"], m["grx"], m["gry"], m["ux"], m["uy"])
    # step 9: collision (Eq. eqLBEMCa), then streaming to r + e_a
    gstar = g - (g - geq) / lat.tau + (1.0 - 1.0 / (2.0 * lat.tau)) * Fa
    out = np.empty_like(g)
    for a in range(9):
        out[:, a] = np.roll(gstar[:, a], shift=(E[a, 1], E[a, 0]), axis=(-2, -1))
    if return_macro:
        return out, m["F_tot"], m
    return out, m["F_tot"]


def init_at_rest(rho: np.ndarray, rho0: float = 0.0, formulation: str = "well_balanced"):
    """State of a fluid at rest: g = g^eq(rho_i, u = 0) of Eq. eqLBEMCb (Eq. eqLBE in the
    standard formulation: rho_i w_a) and a zero stored force (there is no previous step
    whose force the first velocity could use)."""
    rho = np.asarray(rho, dtype=np.float64)
    z = np.zeros(rho.shape[1:], dtype=np.float64)
    geq = equilibrium(rho, z, z, rho0, standard=formulation == "standard")
    return geq, np.zeros((2,) + rho.shape[1:], dtype=np.float64)


def run(g: np.ndarray, F_prev: np.ndarray, mix: Mixture, lat: Lattice, nsteps: int):
    for _ in range(nsteps):
        g, F_prev = step(g, mix, lat, F_prev)
    return g, F_prev


def moments(g: np.ndarray, F_prev: np.ndarray, mix: Mixture, lat: Lattice) -> dict:
    """Densities, velocity of step 1 (with the half force) and ln f of the current state."""
    m = macroscopic(g, mix, lat, F_prev)
    return dict(rho=m["rho"], ux=m["ux"], uy=m["uy"], lnf=m["lnf"])


def component_mass(g: np.ndarray) -> np.ndarray:
    """sum over the lattice of rho_i, per component."""
    return g.sum(axis=(1, 2, 3))


def phase_measure(rho: np.ndarray) -> np.ndarray:
    """Phase measure of a state: lambda_i = mean over the nodes of ln rho_i, per component
    (rho has shape (N, ny, nx)).  Its change between two states, max_i |d lambda_i|, is the
    volume-averaged relative change of each component's density: it follows the phases
    (densities, compositions, volumes) but not a rigid motion of the field, since a sum of a
    smooth function of the densities over a periodic lattice does not change when the field
    moves.  A convergence measure of this build (the paper runs fixed step counts)."""
    return np.log(rho).reshape(rho.shape[0], -1).mean(axis=1)


def residual(rho_now: np.ndarray, rho_before: np.ndarray) -> float:
    """Convergence measure: ||rho(t) - rho(t - D)||_2 / ||rho(t)||_2 over all nodes and
    components (the paper runs fixed step counts; this criterion is this build's)."""
    return float(np.sqrt(np.sum((rho_now - rho_before) ** 2)) / np.sqrt(np.sum(rho_now ** 2)))
