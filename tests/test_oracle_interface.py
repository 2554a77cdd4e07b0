"""Pins of oracle/interface.py (Section V.E measures) against closed forms."""
import numpy as np

from oracle.interface import crossing_radius, interfacial_tension, lamb_period
from paper_2212_10680_gb300 import inputs


def test_tension_of_a_tanh_slab_matches_the_closed_form():
    # rho = a + b tanh(2 x / W) per interface: integral of (d rho/dx)^2 = 8 b^2 / (3 W).
    # Two components with profiles proportional to each other, kappa_ij = sqrt(k_i k_j):
    # sum_ij kappa_ij c_i c_j = (sum_i sqrt(k_i) c_i)^2 times the single-profile integral.
    # The central difference converges at second order in 1 / W.
    rV, rL = np.array([0.1, 0.3]), np.array([1.1, 2.3])
    kappa = [0.1, 0.15]
    b = 0.5 * (rL - rV)
    err = []
    for W in (40.0, 80.0):
        rho = inputs.slab(rV, rL, 8000, 1, 0.5, W)[:, 0, :]
        expect = (np.sqrt(kappa[0]) * b[0] + np.sqrt(kappa[1]) * b[1]) ** 2 * 8.0 / (3.0 * W)
        err.append(interfacial_tension(rho, kappa, n_interfaces=2) / expect - 1)
    assert abs(err[1]) < 2e-4
    assert 3.8 < err[0] / err[1] < 4.2


def test_lamb_period_formula():
    # n = 2: T = 2 pi sqrt(rho R^3 / (6 sigma)); sigma = 0.5, rho = 6, R = 10 -> 2 pi sqrt(2000)
    assert abs(lamb_period(0.5, 6.0, 10.0, 2) - 2 * np.pi * np.sqrt(2000.0)) < 1e-9
    # n = 3: factor n (n^2 - 1) = 24
    assert abs(lamb_period(2.4, 1.0, 1.0, 3) - 2 * np.pi / np.sqrt(57.6)) < 1e-12


def test_crossing_radius_of_a_sampled_tanh():
    x = np.arange(200, dtype=np.float64)
    R0, W = 37.3, 4.0
    prof = 5.0 - 4.0 * np.tanh(2.0 * (np.abs(x - 100.0) - R0) / W)
    r = crossing_radius(prof, 100.0, 5.0)
    # linear interpolation of a tanh between nodes 137 and 138: error below 0.02 node
    assert abs(r - R0) < 0.02
    assert np.isnan(crossing_radius(np.full(50, 1.0), 10.0, 5.0))
