"""Pins of the EOS / log-fugacity oracle (oracle/eos.py) against thermodynamics.

Each check ties the oracle to something other than its own formulas:
* the critical point of each cubic EOS of Appendix C (inflection at Tc, Pc, with the
  textbook critical compressibility), which fixes the printed constants and the form
  of every pressure expression;
* the reference state of Eq. eqfugdef2 (ideal-gas limit);
* Gibbs-Duhem at constant T, sum_i rho~_i d ln f_i = dp / RT, by finite differences;
* the residual-chemical-potential integral of Eq. eqfug2, evaluated by quadrature of
  the pressure alone (no fugacity formula involved);
* equality with the textbook phi-forms (Eqs. eqfugvdW/SRK/PR) where p > 0;
* splitting one component into two identical ones changes ln f only by ln x.
"""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import minimize_scalar

from oracle.eos import (Mixture, OMEGA, alpha_function, ln_phi_textbook, lnf_density_form,
                        pressure, pressure_from_volume, volume_roots)

EOSES = ["pr", "srk", "vdw"]
ZC = {"pr": 0.307401, "srk": 1.0 / 3.0, "vdw": 3.0 / 8.0}


def lattice_binary(eos="pr", Tr=0.8):
    oa, ob = OMEGA["pr"]
    Tc1 = (2 / 49) / (2 / 21) * ob / oa
    Pc1 = ob * Tc1 / (2 / 21)
    return Mixture(eos, 1.0, Tr * Tc1, Tc=[Tc1, 1.5 * Tc1], Pc=[Pc1, 0.9 * Pc1],
                   omega=[0.011, 0.2], kij=[[0, 0.03], [0.03, 0]], M=[1.0, 2.0])


def lattice_ternary(eos="pr"):
    oa, ob = OMEGA["pr"]
    Tc1 = (2 / 49) / (2 / 21) * ob / oa
    Pc1 = ob * Tc1 / (2 / 21)
    kij = np.full((3, 3), 0.02) - 0.02 * np.eye(3)
    return Mixture(eos, 1.0, 0.85 * Tc1, Tc=[Tc1, 1.3 * Tc1, 1.6 * Tc1],
                   Pc=[Pc1, 0.85 * Pc1, 0.7 * Pc1], omega=[0.011, 0.1, 0.25], kij=kij)


@pytest.mark.parametrize("eos", EOSES)
def test_critical_point_of_each_eos(eos):
    # At T = Tc the isotherm has an inflection with zero slope at p = Pc (Appendix C
    # constants are defined by this); its compressibility is the textbook Zc.
    Tc, Pc, R = 369.8, 42.48, 83.14462618
    mix = Mixture(eos, R, Tc, Tc=[Tc], Pc=[Pc], omega=[0.152])
    x = np.array([1.0])
    dpdv = lambda v: (pressure_from_volume(mix, v * (1 + 1e-6), x)
                      - pressure_from_volume(mix, v * (1 - 1e-6), x)) / (2e-6 * v)
    vguess = ZC[eos] * R * Tc / Pc
    res = minimize_scalar(lambda v: -dpdv(v), bounds=(0.5 * vguess, 2.0 * vguess), method="bounded",
                          options=dict(xatol=1e-10 * vguess))
    vc = res.x
    scale = R * Tc / vc**2
    assert abs(dpdv(vc)) / scale < 1e-6   # the printed constants carry 7-10 digits
    pc = pressure_from_volume(mix, vc, x)
    assert abs(pc / Pc - 1) < 2e-6
    assert abs(pc * vc / (R * Tc) - ZC[eos]) < 2e-4
    # alpha(Tc) = 1 for every EOS
    assert np.allclose(alpha_function(eos, np.array([0.1, 0.6]), np.array([1.0, 1.0])), 1.0)


@pytest.mark.parametrize("eos", EOSES)
def test_ideal_gas_limit(eos):
    # Eq. eqfugdef2: f_i / (x_i p) -> 1 as p -> 0, i.e. ln f_i -> ln(rho~_i R T).
    mix = lattice_ternary(eos)
    for scale in (1e-7, 1e-9):
        rt = np.array([0.3, 0.5, 0.2]) * scale
        lnf = lnf_density_form(mix, rt)
        assert np.max(np.abs(lnf - np.log(rt * mix.RT))) < 50 * scale


@pytest.mark.parametrize("eos", EOSES)
def test_gibbs_duhem(eos):
    # sum_i rho~_i d ln f_i = dp / RT at constant T, for arbitrary directions d rho~.
    mix = lattice_ternary(eos)
    rng = np.random.default_rng(7)
    done = 0
    while done < 20:
        rt = rng.uniform(0.05, 2.0, 3)
        if float(np.dot(mix.b, rt)) > 0.9:   # stay inside the EOS domain rho~ b_m < 1
            continue
        done += 1
        d = rng.normal(size=3)
        h = 1e-6
        dl = (lnf_density_form(mix, rt + h * d) - lnf_density_form(mix, rt - h * d)) / (2 * h)
        dp = (pressure(mix, rt + h * d) - pressure(mix, rt - h * d)) / (2 * h)
        lhs = float(np.sum(rt * dl))
        rhs = float(dp / mix.RT)
        assert abs(lhs - rhs) <= 1e-7 * (abs(rhs) + np.sum(np.abs(rt * dl)))


def _lnphi_by_quadrature(mix, n, V):
    """Eq. eqfug2 with p(n, V) from the EOS only:
    ln(f_i/(x_i p)) = -(1/RT) int_inf^V [(dp/dn_i)_{T,V,n_j} - RT/V] dV - ln Z."""
    RT = mix.RT
    N = n.size
    p_of = lambda nn, VV: float(pressure(mix, nn / VV))
    out = np.empty(N)
    for i in range(N):
        def integrand_u(u):
            # substitute V = 1/u; dV = -du/u^2; the integral from inf to V becomes
            # -int_0^{1/V} h(1/u) / u^2 du with h = dp/dn_i - RT/V
            VV = 1.0 / u
            hstep = 1e-5 * n[i]
            e = np.zeros(N)
            e[i] = hstep
            dpdn = (p_of(n + e, VV) - p_of(n - e, VV)) / (2 * hstep)
            return (dpdn - RT / VV) / u**2
        integral, _ = quad(integrand_u, 0.0, 1.0 / V, epsabs=0, epsrel=1e-12, limit=200)
        # int_inf^V h dV = -int_0^{1/V} h(1/u)/u^2 du
        out[i] = integral / RT
    p = p_of(n, V)
    Z = p * V / (np.sum(n) * RT)
    return out - np.log(Z)


@pytest.mark.parametrize("eos", EOSES)
def test_lnf_equals_residual_integral(eos):
    mix = lattice_binary(eos, Tr=1.3)  # single-phase states with p > 0 everywhere on the path
    for rt in (np.array([0.4, 0.9]), np.array([2.0, 1.1]), np.array([0.05, 0.01])):
        V = 1.0
        n = rt * V
        lnphi_q = _lnphi_by_quadrature(mix, n, V)
        x = rt / rt.sum()
        p = float(pressure(mix, rt))
        lnf = lnf_density_form(mix, rt)
        lnphi = lnf - np.log(x * p)
        assert np.max(np.abs(lnphi - lnphi_q)) < 2e-8


@pytest.mark.parametrize("eos", EOSES)
def test_density_form_equals_textbook_form(eos):
    mix = lattice_ternary(eos)
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(400):
        rt = rng.uniform(0.01, 2.5, 3) * rng.choice([0.05, 1.0])
        p = pressure(mix, rt)
        bm = float(np.dot(mix.b, rt / rt.sum()))
        if p <= 0 or bm * rt.sum() >= 1:
            continue
        x = rt / rt.sum()
        lhs = lnf_density_form(mix, rt)
        rhs = np.log(x * p) + ln_phi_textbook(mix, 1.0 / rt.sum(), x)
        assert np.max(np.abs(lhs - rhs)) < 1e-12 * max(1.0, np.max(np.abs(lhs)))
        checked += 1
    assert checked > 100


@pytest.mark.parametrize("eos", EOSES)
def test_split_identical_component(eos):
    # Two identical species (same Tc, Pc, omega, zero interaction) behave as one:
    # ln f_i(rho1, rho2) = ln x_i + ln f_pure(rho1 + rho2).
    oa, ob = OMEGA["pr"]
    Tc, Pc = 0.0729, 0.0596
    pure = Mixture(eos, 1.0, 0.9 * Tc, Tc=[Tc], Pc=[Pc], omega=[0.05])
    pair = Mixture(eos, 1.0, 0.9 * Tc, Tc=[Tc, Tc], Pc=[Pc, Pc], omega=[0.05, 0.05])
    for r1, r2 in [(0.3, 1.2), (2.0, 0.01), (4.0, 2.5)]:
        lnf2 = lnf_density_form(pair, np.array([r1, r2]))
        lnf1 = lnf_density_form(pure, np.array([r1 + r2]))[0]
        x = np.array([r1, r2]) / (r1 + r2)
        assert np.allclose(lnf2, np.log(x) + lnf1, rtol=1e-13, atol=1e-12)
        assert np.isclose(pressure(pair, np.array([r1, r2])), pressure(pure, np.array([r1 + r2])),
                          rtol=1e-14)


def test_volume_roots_solve_the_eos():
    mix = lattice_binary("pr", Tr=0.8)
    x = np.array([0.5, 0.5])
    for p in (1e-4, 3e-3, 1e-2):
        roots = volume_roots(mix, p, x)
        assert roots.size >= 1
        for v in roots:
            assert abs(pressure_from_volume(mix, v, x) / p - 1) < 1e-10
