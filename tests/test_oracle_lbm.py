"""Pins of the lattice Boltzmann oracle (oracle/lbm.py).

* Moments of the well-balanced equilibrium (Eq. eqLBEMCb): density rho_i, momentum
  rho_i u and momentum flux rho_i u u (no c_s^2 rho I term, which is the point of
  the well-balanced form with rho_0 = 0).
* Moments of the forcing term (Eq. eqLBEMCfinal3): zero mass, momentum F_i, and the
  second moment u F + F u + c_s^2 (u grad rho + grad rho u + (u . grad rho) I) that
  follows from the D2Q9 isotropy identities.
* Exact per-component mass conservation over many steps; an exactly stationary
  uniform state; mirror and transpose symmetry of one step (catches wrong signs,
  swapped indices and mis-assigned directions); the isotropic stencils equal the
  central ones on y-uniform fields.
* Newton's law of the forced collision: with u = (j + F/2) / rho, BGK relaxation plus the
  (1 - 1/(2 tau)) F_{a,i} of Eq. eqLBEMCa leaves j + F at every node, for any tau (fixes
  the 1/2 in u and the prefactor, which no equilibrium depends on).
* The single-component limit settles on the Maxwell pair of the PR EOS.
* The standard formulation of Section VI (Eq. eqLBE, force of Eq. eqForceGen): its
  equilibrium carries c_s^2 rho_i I, Guo's forcing term has the plain moments, mass is
  conserved, a uniform state is invariant, and a flat slab settles slightly off the
  Maxwell pair (close enough to catch a wrong sign of the c_s^2 grad rho_i term).
"""
import numpy as np
import pytest

from oracle import lbm
from oracle.eos import Mixture, OMEGA
from oracle.flash import pure_coexistence, slab_state
from paper_2212_10680_gb300 import inputs

CS2 = 1.0 / 3.0


def lattice_units():
    oa, ob = OMEGA["pr"]
    Tc1 = (2 / 49) / (2 / 21) * ob / oa
    return Tc1, ob * Tc1 / (2 / 21)


def binary_mixture(Tr=0.8):
    Tc1, Pc1 = lattice_units()
    return Mixture("pr", 1.0, Tr * Tc1, Tc=[Tc1, 1.5 * Tc1], Pc=[Pc1, 0.9 * Pc1], omega=[0.011, 0.2],
                   kappa=[0.1, 0.15])


def test_d2q9_isotropy():
    E, W = lbm.E.astype(float), lbm.W
    assert np.isclose(W.sum(), 1.0)
    assert np.allclose(np.einsum("a,ai->i", W, E), 0)
    assert np.allclose(np.einsum("a,ai,aj->ij", W, E, E), CS2 * np.eye(2))
    assert np.allclose(np.einsum("a,ai,aj,ak->ijk", W, E, E, E), 0)
    d = np.eye(2)
    iso4 = CS2**2 * (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
                     + np.einsum("il,jk->ijkl", d, d))
    assert np.allclose(np.einsum("a,ai,aj,ak,al->ijkl", W, E, E, E, E), iso4)


@pytest.mark.parametrize("rho0", [0.0, 0.7])
def test_equilibrium_moments(rho0):
    rng = np.random.default_rng(0)
    rho = rng.uniform(0.1, 3.0, (2, 3, 4))
    ux = rng.uniform(-0.1, 0.1, (3, 4))
    uy = rng.uniform(-0.1, 0.1, (3, 4))
    geq = lbm.equilibrium(rho, ux, uy, rho0)
    E = lbm.E.astype(float)
    assert np.allclose(geq.sum(axis=1), rho, rtol=1e-14, atol=1e-14)
    assert np.allclose(np.tensordot(E[:, 0], geq, axes=(0, 1)), rho * ux, atol=1e-15)
    assert np.allclose(np.tensordot(E[:, 1], geq, axes=(0, 1)), rho * uy, atol=1e-15)
    Pxx = np.tensordot(E[:, 0] * E[:, 0], geq, axes=(0, 1))
    Pxy = np.tensordot(E[:, 0] * E[:, 1], geq, axes=(0, 1))
    Pyy = np.tensordot(E[:, 1] * E[:, 1], geq, axes=(0, 1))
    assert np.allclose(Pxx, rho * ux * ux + rho0 * CS2, atol=1e-14)
    assert np.allclose(Pxy, rho * ux * uy, atol=1e-14)
    assert np.allclose(Pyy, rho * uy * uy + rho0 * CS2, atol=1e-14)


def test_forcing_term_moments():
    rng = np.random.default_rng(1)
    shape = (3, 5, 4)
    Fx, Fy, gx, gy = (rng.normal(size=shape) for _ in range(4))
    ux = rng.uniform(-0.1, 0.1, shape[1:])
    uy = rng.uniform(-0.1, 0.1, shape[1:])
    Fa = lbm.forcing_term(Fx, Fy, gx, gy, ux, uy)
    E = lbm.E.astype(float)
    assert np.allclose(Fa.sum(axis=1), 0.0, atol=1e-14)
    assert np.allclose(np.tensordot(E[:, 0], Fa, axes=(0, 1)), Fx, atol=1e-14)
    assert np.allclose(np.tensordot(E[:, 1], Fa, axes=(0, 1)), Fy, atol=1e-14)
    ug = ux * gx + uy * gy
    Sxx = np.tensordot(E[:, 0] ** 2, Fa, axes=(0, 1))
    Sxy = np.tensordot(E[:, 0] * E[:, 1], Fa, axes=(0, 1))
    Syy = np.tensordot(E[:, 1] ** 2, Fa, axes=(0, 1))
    assert np.allclose(Sxx, 2 * ux * Fx + CS2 * (2 * ux * gx + ug), atol=1e-13)
    assert np.allclose(Sxy, ux * Fy + uy * Fx + CS2 * (ux * gy + uy * gx), atol=1e-13)
    assert np.allclose(Syy, 2 * uy * Fy + CS2 * (2 * uy * gy + ug), atol=1e-13)


def _smooth_binary_state(nx=12, ny=10, seed=5):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    base = np.stack([1.0 + 0.3 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny),
                     1.2 + 0.2 * np.cos(2 * np.pi * (x + 2 * y) / nx)])
    return base * (1 + 0.01 * rng.uniform(-1, 1, base.shape))


@pytest.mark.parametrize("velocity_force", ["lagged", "current"])
@pytest.mark.parametrize("stencil", ["isotropic", "central"])
def test_mass_conservation(stencil, velocity_force):
    mix = binary_mixture(Tr=1.1)
    mix.kappa = np.array([0.02, 0.03])   # keeps the "current" reading inside its stability range
    lat = lbm.Lattice(tau=0.9, stencil=stencil, velocity_force=velocity_force)
    g, F = lbm.init_at_rest(_smooth_binary_state())
    m0 = lbm.component_mass(g)
    g, F = lbm.run(g, F, mix, lat, 200)
    assert np.max(np.abs(lbm.component_mass(g) / m0 - 1)) < 1e-13
    assert np.abs(g).max() > 0 and np.isfinite(g).all()


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_collision_adds_exactly_the_force_to_the_momentum(tau):
    # Sum over a and i of g*_{a,i} e_a = J - (J - rho u) / tau + (1 - 1/(2 tau)) F with
    # rho u = J + F / 2 ("current" reading) is J + F whatever tau is.  Checked node by node
    # on the post-collision values (the step's streaming undone) of a moving two-phase state.
    mix = binary_mixture(Tr=1.1)
    mix.kappa = np.array([0.02, 0.03])
    lat = lbm.Lattice(tau=tau, stencil="isotropic", velocity_force="current")
    g, F = lbm.init_at_rest(_smooth_binary_state())
    g, F = lbm.run(g, F, mix, lat, 3)                   # a state with momentum
    g_new, F_tot, m = lbm.step(g, mix, lat, F, return_macro=True)
    gstar = np.empty_like(g_new)
    for a in range(9):
        gstar[:, a] = np.roll(g_new[:, a], shift=(-lbm.E[a, 1], -lbm.E[a, 0]), axis=(-2, -1))
    ex, ey = lbm.E[:, 0].astype(np.float64), lbm.E[:, 1].astype(np.float64)
    J = [np.einsum("a,iayx->yx", e, g) for e in (ex, ey)]
    Jstar = [np.einsum("a,iayx->yx", e, gstar) for e in (ex, ey)]
    scale = max(np.abs(J[0]).max(), np.abs(F_tot).max())
    assert scale > 1e-4
    for k in range(2):
        assert np.max(np.abs(Jstar[k] - (J[k] + F_tot[k]))) <= 1e-14 * max(1.0, np.abs(g).max())


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_collision_adds_exactly_the_force_to_the_momentum_lagged(tau):
    # The lagged reading puts the previous step's total force into the velocity:
    # rho u = J + F(t-1) / 2.  The equilibrium carries momentum rho u and the forcing term
    # carries F(t) (moment identities of Eqs. eqLBEMCb and eqLBEMCfinal3), so after the
    # collision of Eq. eqLBEMCa
    #   J* = J - (J - rho u) / tau + (1 - 1/(2 tau)) F(t) = J + F(t-1) / (2 tau) + (1 - 1/(2 tau)) F(t)
    # at every node.  F(t-1) and F(t) are taken here from the component forces the oracle
    # computed in those steps (summed over components by this test), not from the stored force
    # it hands on; and a chain of single steps must equal one call of run().
    mix = binary_mixture(Tr=1.1)
    mix.kappa = np.array([0.02, 0.03])
    lat = lbm.Lattice(tau=tau, stencil="isotropic", velocity_force="lagged")
    g0, F0 = lbm.init_at_rest(_smooth_binary_state())
    g, F = g0, F0
    for _ in range(2):
        g, F = lbm.step(g, mix, lat, F)
    g, F, m_prev = lbm.step(g, mix, lat, F, return_macro=True)          # step t - 1
    F_prev = [m_prev["Fx"].sum(axis=0), m_prev["Fy"].sum(axis=0)]
    g_new, F_new, m = lbm.step(g, mix, lat, F, return_macro=True)      # step t
    F_now = [m["Fx"].sum(axis=0), m["Fy"].sum(axis=0)]
    gstar = np.empty_like(g_new)
    for a in range(9):
        gstar[:, a] = np.roll(g_new[:, a], shift=(-lbm.E[a, 1], -lbm.E[a, 0]), axis=(-2, -1))
    ex, ey = lbm.E[:, 0].astype(np.float64), lbm.E[:, 1].astype(np.float64)
    J = [np.einsum("a,iayx->yx", e, g) for e in (ex, ey)]
    Jstar = [np.einsum("a,iayx->yx", e, gstar) for e in (ex, ey)]
    # the two forces differ (otherwise the lagged and current readings are indistinguishable)
    assert np.max(np.abs(F_now[0] - F_prev[0])) > 1e-3 * np.max(np.abs(F_now[0]))
    tol = 1e-14 * max(1.0, np.abs(g).max())
    for k in range(2):
        expect = J[k] + F_prev[k] / (2 * tau) + (1 - 1 / (2 * tau)) * F_now[k]
        assert np.max(np.abs(Jstar[k] - expect)) <= tol
    # the stored force the oracle hands to the next step is the total force of this step
    assert np.max(np.abs(F_new[0] - F_now[0])) <= tol and np.max(np.abs(F_new[1] - F_now[1])) <= tol
    # run() advances the stored force from step to step exactly as the chain above does
    g_run, F_run = lbm.run(g0, F0, mix, lat, 4)
    assert np.array_equal(g_run, g_new) and np.array_equal(F_run, F_new)


@pytest.mark.parametrize("stencil", ["isotropic", "central"])
def test_uniform_state_is_stationary(stencil):
    mix = binary_mixture()
    lat = lbm.Lattice(tau=1.0, stencil=stencil)
    rho = np.stack([np.full((6, 7), 2.0), np.full((6, 7), 1.5)])
    g0, F0 = lbm.init_at_rest(rho)
    g, F = lbm.run(g0, F0, mix, lat, 50)
    assert np.array_equal(g, g0)
    assert np.array_equal(F, np.zeros_like(F))


@pytest.mark.parametrize("stencil", ["isotropic", "central"])
def test_mirror_and_transpose_symmetry(stencil):
    mix = binary_mixture(Tr=1.1)
    lat = lbm.Lattice(tau=0.8, stencil=stencil)
    rho = _smooth_binary_state(nx=10, ny=10)
    g, F = lbm.init_at_rest(rho)
    g, F = lbm.run(g, F, mix, lat, 3)          # a state with flow
    g1, F1 = lbm.step(g, mix, lat, F)
    # mirror x -> -x maps direction a to the one with e_x negated
    E = lbm.E
    mirror = [int(np.where((E[:, 0] == -E[a, 0]) & (E[:, 1] == E[a, 1]))[0][0]) for a in range(9)]
    flip = lambda h: np.roll(h[..., ::-1], 1, axis=-1)   # x -> (-x) mod nx
    gm = flip(g[:, mirror])
    Fm = np.stack([-flip(F[0]), flip(F[1])])
    gm1, Fm1 = lbm.step(gm, mix, lat, Fm)
    assert np.allclose(gm1, flip(g1[:, mirror]), rtol=0, atol=1e-13)
    assert np.allclose(Fm1[0], -flip(F1[0]), atol=1e-13)
    # transpose x <-> y maps e = (ex, ey) to (ey, ex)
    swap = [int(np.where((E[:, 0] == E[a, 1]) & (E[:, 1] == E[a, 0]))[0][0]) for a in range(9)]
    T = lambda h: np.swapaxes(h, -1, -2)
    gt = T(g[:, swap])
    Ft = np.stack([T(F[1]), T(F[0])])
    gt1, Ft1 = lbm.step(gt, mix, lat, Ft)
    assert np.allclose(gt1, T(g1[:, swap]), rtol=0, atol=1e-13)


def test_isotropic_equals_central_on_flat_fields():
    mix = binary_mixture()
    s = slab_state(mix, [0.5, 0.5])
    rho = inputs.slab(s["rtV"], s["rtL"], 32, 3, 0.5, 4.0)
    gi, Fi = lbm.init_at_rest(rho)
    gc, Fc = gi.copy(), Fi.copy()
    li = lbm.Lattice(tau=1.0, stencil="isotropic")
    lc = lbm.Lattice(tau=1.0, stencil="central")
    for _ in range(20):
        gi, Fi = lbm.step(gi, mix, li, Fi)
        gc, Fc = lbm.step(gc, mix, lc, Fc)
    assert np.allclose(gi, gc, rtol=0, atol=1e-13)


def test_nonphysical_state_is_reported():
    mix = binary_mixture()
    rho = np.stack([np.full((4, 4), 1.0), np.full((4, 4), 1.0)])
    rho[1, 2, 3] = -1e-3
    g, F = lbm.init_at_rest(rho)
    with pytest.raises(lbm.NonPhysicalState) as ei:
        lbm.step(g, mix, lbm.Lattice(tau=1.0), F)
    assert (ei.value.comp, ei.value.y, ei.value.x) == (1, 2, 3)


def test_single_component_limit_reaches_maxwell_pair():
    # N = 1 is the single-component well-balanced free-energy LBM (Section II / III with
    # one species).  A flat slab relaxes to the PR coexistence pair found by the equal-area
    # (fugacity-equality) construction; the residual gap is the finite-difference error of
    # the interface, which the paper's scheme does not remove (tolerance 2e-4).
    Tc1, Pc1 = lattice_units()
    mix = Mixture("pr", 1.0, 0.85 * Tc1, Tc=[Tc1], Pc=[Pc1], omega=[0.011], kappa=[0.1])
    s = pure_coexistence(mix)
    nx = 128
    rho = inputs.slab([s["rtV"]], [s["rtL"]], nx, 1, 0.5, 4.0)
    g, F = lbm.init_at_rest(rho)
    g, F = lbm.run(g, F, mix, lbm.Lattice(tau=1.0, stencil="central"), 12000)
    r = g.sum(axis=1)[0, 0]
    assert abs(r[nx // 2] / s["rtL"] - 1) < 2e-4
    assert abs(r[0] / s["rtV"] - 1) < 2e-4
    # and the slab did move away from the tanh start (the test is not vacuous)
    assert np.max(np.abs(r - rho[0, 0])) > 1e-3


# --- the standard formulation of Section VI (Eq. eqLBE with the force of Eq. eqForceGen) ---

def test_standard_equilibrium_and_forcing_moments():
    # Eq. eqLBE's equilibrium carries the ideal-gas flux c_s^2 rho_i I that the well-balanced
    # form removes, and Guo's forcing term (Eq. eqLBEfinal3) has second moment u F + F u
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.1, 3.0, (2, 3, 4))
    ux = rng.uniform(-0.1, 0.1, (3, 4))
    uy = rng.uniform(-0.1, 0.1, (3, 4))
    geq, _ = lbm.init_at_rest(rho, formulation="standard")
    assert np.allclose(geq, lbm.W[None, :, None, None] * rho[:, None], atol=1e-15)   # rho_i w_a at rest
    geq = lbm.equilibrium(rho, ux, uy, standard=True)
    assert np.allclose(geq, lbm.equilibrium(rho, ux, uy, rho), atol=1e-15)   # Eq. eqLBEMCb, rho_0,i = rho_i
    E = lbm.E.astype(float)
    for a in range(9):
        eu = E[a, 0] * ux + E[a, 1] * uy
        expect = lbm.W[a] * rho * (1 + eu / CS2 + eu * eu / (2 * CS2 ** 2) - (ux * ux + uy * uy) / (2 * CS2))
        assert np.allclose(geq[:, a], expect, atol=1e-15)
    Pxx = np.tensordot(E[:, 0] ** 2, geq, axes=(0, 1))
    assert np.allclose(Pxx, rho * ux * ux + CS2 * rho, atol=1e-14)
    Fx, Fy = rng.normal(size=(2,) + rho.shape)
    z = np.zeros_like(Fx)
    Fa = lbm.forcing_term(Fx, Fy, z, z, ux, uy)
    assert np.allclose(Fa.sum(axis=1), 0.0, atol=1e-14)
    assert np.allclose(np.tensordot(E[:, 0], Fa, axes=(0, 1)), Fx, atol=1e-14)
    assert np.allclose(np.tensordot(E[:, 0] * E[:, 1], Fa, axes=(0, 1)), ux * Fy + uy * Fx, atol=1e-13)


def test_standard_form_conserves_mass_and_keeps_a_uniform_state():
    mix = binary_mixture(Tr=1.1)
    lat = lbm.Lattice(tau=0.9, stencil="isotropic", formulation="standard")
    g, F = lbm.init_at_rest(_smooth_binary_state(), formulation="standard")
    m0 = lbm.component_mass(g)
    g, F = lbm.run(g, F, mix, lat, 200)
    assert np.max(np.abs(lbm.component_mass(g) / m0 - 1)) < 1e-13
    rho = np.stack([np.full((6, 7), 2.0), np.full((6, 7), 1.5)])
    g0, F0 = lbm.init_at_rest(rho, formulation="standard")
    g, F = lbm.run(g0, F0, mix, lat, 50)
    # invariant up to the rounding of sum_a w_a rho_i (the well-balanced rest state puts
    # all of rho_i in a = 0 and is invariant bit for bit)
    assert np.allclose(g, g0, rtol=1e-14, atol=0) and np.max(np.abs(F)) < 1e-14


def test_standard_form_single_component_slab_deviates_slightly_from_maxwell():
    # Section VI: the standard formulation works with "slight deviations" from
    # thermodynamics.  The c_s^2 grad rho of Eq. eqForceGen cancels the LBE's own ideal-gas
    # pressure gradient only up to discretisation, which shows most in the vapour: at
    # T = 0.95 Tc the slab settles 0.7% (liquid) and 3.7% (vapour) off the Maxwell pair,
    # where the well-balanced form is within 7e-4 (at 0.85 Tc the vapour is 30% off, so
    # "slight" holds for moderate density ratios only).  A wrong sign of that term drives
    # the vapour negative within a few thousand steps.
    Tc1, Pc1 = lattice_units()
    mix = Mixture("pr", 1.0, 0.95 * Tc1, Tc=[Tc1], Pc=[Pc1], omega=[0.011], kappa=[0.1])
    s = pure_coexistence(mix)
    nx = 128
    rho = inputs.slab([s["rtV"]], [s["rtL"]], nx, 1, 0.5, 4.0)
    g, F = lbm.init_at_rest(rho, formulation="standard")
    g, F = lbm.run(g, F, mix, lbm.Lattice(tau=1.0, stencil="central", formulation="standard"), 8000)
    r = g.sum(axis=1)[0, 0]
    dL, dV = abs(r[nx // 2] / s["rtL"] - 1), abs(r[0] / s["rtV"] - 1)
    assert 3e-3 < dL < 0.012 and 0.02 < dV < 0.05, (dL, dV)
