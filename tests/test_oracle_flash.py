"""Pins of the phase-equilibrium oracle (oracle/flash.py).

* Maxwell equal-area rule for the pure-component coexistence found by fugacity
  equality: int_{vL}^{vV} p dv = p_sat (vV - vL), by adaptive quadrature.
* Flash results satisfy fugacity equality (density-form ln f of Eq. eqfugupdatePR,
  a formula the flash itself does not use) and the material balance.
* Pure-component limit of the bubble-point solver equals the Maxwell pair.
* Physical-unit C2/n-C5 at 387.70 K against the fugacities printed in Table tabFug.
"""
import json
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import brentq, fsolve

from oracle.eos import Mixture, OMEGA, ln_phi_textbook, lnf_density_form, pressure, pressure_from_volume
from oracle.flash import bubble_point_from_liquid, flash, pure_coexistence, slab_state, vapour_volume_fraction

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lattice_constants():
    oa, ob = OMEGA["pr"]
    Tc1 = (2 / 49) / (2 / 21) * ob / oa
    return Tc1, ob * Tc1 / (2 / 21)


@pytest.mark.parametrize("eos,Tr", [("pr", 0.8), ("pr", 0.95), ("srk", 0.8), ("vdw", 0.85)])
def test_pure_coexistence_obeys_equal_area(eos, Tr):
    Tc1, Pc1 = lattice_constants()
    mix = Mixture(eos, 1.0, Tr * Tc1, Tc=[Tc1], Pc=[Pc1], omega=[0.011])
    s = pure_coexistence(mix)
    x = np.array([1.0])
    area, _ = quad(lambda v: pressure_from_volume(mix, v, x), s["vL"], s["vV"], epsabs=0, epsrel=1e-13,
                   limit=400)
    assert abs(area - s["p"] * (s["vV"] - s["vL"])) <= 1e-10 * abs(area)
    assert abs(pressure_from_volume(mix, s["vL"], x) / s["p"] - 1) < 1e-10
    assert abs(pressure_from_volume(mix, s["vV"], x) / s["p"] - 1) < 1e-10


def test_pure_coexistence_lattice_units_value():
    # The lattice units of Section V (R = 1, a = 2/49, b = 2/21) at T = 0.8 Tc:
    # the liquid/vapour pair is a property of the PR EOS alone.
    Tc1, Pc1 = lattice_constants()
    mix = Mixture("pr", 1.0, 0.8 * Tc1, Tc=[Tc1], Pc=[Pc1], omega=[0.011])
    assert np.isclose(mix.a[0], 2 / 49, rtol=1e-14) and np.isclose(mix.b[0], 2 / 21, rtol=1e-14)
    s = pure_coexistence(mix)
    lnf = lnf_density_form(mix, np.array([[s["rtL"], s["rtV"]]]))
    assert abs(lnf[0, 0] - lnf[0, 1]) < 1e-11


@pytest.mark.parametrize("n", [2, 3])
def test_flash_fugacity_equality_and_balance(n):
    Tc1, Pc1 = lattice_constants()
    if n == 2:
        mix = Mixture("pr", 1.0, 0.8 * Tc1, Tc=[Tc1, 1.5 * Tc1], Pc=[Pc1, 0.9 * Pc1], omega=[0.011, 0.2])
        z = np.array([0.5, 0.5])
        p = 0.006
    else:
        kij = np.full((3, 3), 0.02) - 0.02 * np.eye(3)
        mix = Mixture("pr", 1.0, 0.85 * Tc1, Tc=[Tc1, 1.3 * Tc1, 1.6 * Tc1],
                      Pc=[Pc1, 0.85 * Pc1, 0.7 * Pc1], omega=[0.011, 0.1, 0.25], kij=kij)
        z = np.array([0.4, 0.3, 0.3])
        p = 0.006
    r = flash(mix, p, z)
    assert r["converged"]
    assert 0 < r["beta"] < 1
    lnfL = lnf_density_form(mix, r["rtL"])
    lnfV = lnf_density_form(mix, r["rtV"])
    assert np.max(np.abs(lnfL - lnfV)) < 1e-10
    assert np.allclose(r["beta"] * r["y"] + (1 - r["beta"]) * r["x"], z, rtol=0, atol=1e-13)
    assert abs(pressure(mix, r["rtL"]) / p - 1) < 1e-10
    assert abs(pressure(mix, r["rtV"]) / p - 1) < 1e-10


def test_slab_state_volume_fraction():
    Tc1, Pc1 = lattice_constants()
    mix = Mixture("pr", 1.0, 0.8 * Tc1, Tc=[Tc1, 1.5 * Tc1], Pc=[Pc1, 0.9 * Pc1], omega=[0.011, 0.2])
    s = slab_state(mix, [0.5, 0.5], S_V=0.5)
    assert abs(vapour_volume_fraction(s) - 0.5) < 1e-9
    assert np.max(np.abs(lnf_density_form(mix, s["rtL"]) - lnf_density_form(mix, s["rtV"]))) < 1e-10


def test_bubble_point_pure_limit_is_maxwell():
    Tc1, Pc1 = lattice_constants()
    mix = Mixture("pr", 1.0, 0.8 * Tc1, Tc=[Tc1, 1.5 * Tc1], Pc=[Pc1, 0.9 * Pc1], omega=[0.011, 0.2])
    pure = Mixture("pr", 1.0, 0.8 * Tc1, Tc=[Tc1], Pc=[Pc1], omega=[0.011])
    s = pure_coexistence(pure)
    eps = 1e-10
    b = bubble_point_from_liquid(mix, [1 - eps, eps], p0=s["p"] * 0.9)
    assert abs(b["p"] / s["p"] - 1) < 1e-7
    assert abs(b["rtL"].sum() / s["rtL"] - 1) < 1e-7
    assert abs(b["rtV"].sum() / s["rtV"] - 1) < 1e-7


def test_table_tabfug_c2_c5_physical_units():
    g = json.load(open(os.path.join(GOLDEN, "tabFug_c2c5_387K.json")))
    R = 83.14462618
    mix = Mixture("pr", R, g["T_K"], Tc=g["Tc_K"], Pc=g["Pc_bar"], omega=g["omega"])
    fL = np.array(g["fugacity_liquid_bar"])
    fV = np.array(g["fugacity_vapor_bar"])
    fmean = 0.5 * (fL + fV)
    z = np.array([0.62, 0.38])

    def f_liquid(p):
        r = flash(mix, p, z)
        return r["x"] * p * np.exp(ln_phi_textbook(mix, r["vL"], r["x"]))

    # flat-interface coexistence at the printed ethane fugacity predicts the pentane one
    p_star = brentq(lambda p: f_liquid(p)[0] - fmean[0], 40.0, 60.0, rtol=1e-13)
    f_pred = f_liquid(p_star)
    assert abs(f_pred[1] / fmean[1] - 1) < 5e-3
    # at the printed fugacities both a liquid and a vapour state exist, and the liquid is at
    # the slightly higher pressure (a curved interface around the liquid, Young-Laplace)
    r = flash(mix, p_star, z)
    sL = fsolve(lambda q: lnf_density_form(mix, np.exp(q)) - np.log(fL), np.log(r["rtL"]), xtol=1e-13)
    sV = fsolve(lambda q: lnf_density_form(mix, np.exp(q)) - np.log(fV), np.log(r["rtV"]), xtol=1e-13)
    assert np.allclose(lnf_density_form(mix, np.exp(sL)), np.log(fL), atol=1e-9)
    assert np.allclose(lnf_density_form(mix, np.exp(sV)), np.log(fV), atol=1e-9)
    pL, pV = pressure(mix, np.exp(sL)), pressure(mix, np.exp(sV))
    assert np.exp(sL).sum() > 1.5 * np.exp(sV).sum()
    assert 0 < (pL - pV) / pV < 1e-2


def test_section_v_e_density_ratio_c3_c5_340K_5bar():
    # Section V.E: the PR flash of propane / n-pentane at 340 K and 5 bar gives a density
    # ratio of 50.97 (the paper prints four figures); the phase compositions of a binary
    # flash do not depend on the feed
    from cases import paper_mixture, oracle_mixture
    mixd, _ = paper_mixture(["C3", "C5"], 340.0, "pr", physical=True)
    mix = oracle_mixture(mixd)
    M = np.array(mixd["M"])
    for z in ([0.4, 0.6], [0.3, 0.7]):
        r = flash(mix, 5.0, z)
        ratio = (r["rtL"] * M).sum() / (r["rtV"] * M).sum()
        assert abs(ratio - 50.97) < 0.006


def test_section_v_lattice_units_leave_phase_equilibria_unchanged():
    # R = 1, a = 2/49, b = 2/21, M = 1 for the most volatile component: temperatures and
    # pressures scale by fixed factors, so compositions and density ratios are unchanged
    from cases import paper_mixture, oracle_mixture
    for names, T, p, z, eos in ((["C3", "C5"], 370.03, 16.547, [0.4, 0.6], "pr"),
                                (["C3", "C5"], 370.03, 16.547, [0.4, 0.6], "srk"),
                                (["C1", "C2", "C3"], 216.483, 20.684, [0.4, 0.3, 0.3], "pr")):
        dl, sc = paper_mixture(names, T, eos)
        dp, _ = paper_mixture(names, T, eos, physical=True)
        oa, ob = OMEGA[eos]
        assert abs(oa * dl["Tc"][0] ** 2 / dl["Pc"][0] - 2.0 / 49.0) < 1e-15  # a_1 (R = 1)
        assert abs(ob * dl["Tc"][0] / dl["Pc"][0] - 2.0 / 21.0) < 1e-15       # b_1
        fl = flash(oracle_mixture(dl), p * sc["p"], z)
        fp = flash(oracle_mixture(dp), p, z)
        assert np.allclose(fl["x"], fp["x"], atol=1e-12) and np.allclose(fl["y"], fp["y"], atol=1e-12)
        ML, MP = np.array(dl["M"]), np.array(dp["M"])
        assert abs((fl["rtL"] * ML).sum() / (fl["rtV"] * ML).sum() / ((fp["rtL"] * MP).sum() / (fp["rtV"] * MP).sum()) - 1) < 1e-10
