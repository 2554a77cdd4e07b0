"""The paper's validation cases (Section V) on the GPU, in the paper's lattice units.

Mixtures come from Table tabCompProp with the mapping of Section V (R = 1; a = 2/49,
b = 2/21, M = 1 for the most volatile component; tests/cases.py: paper_mixture), the
set-ups from tests/golden/paper_cases.json.  Each case compares the lattice with the
FP64 flash oracle the way the paper does, and checks the result against a bound; the
numbers the paper prints (Tables tabcase1error, tabcase3, tabFug; the oscillation
periods of Section V.E) are the context for those bounds:

* V.A  propane / n-pentane flat interface, PR and SRK: bulk densities and compositions
       against the flash at the lattice's own pressure;
* V.B  ethane / n-pentane p-x and T-x envelope points, one batch of 18 lattices (the
       compositions against the flash at each lattice's pressure);
* V.C  methane / ethane / propane flat interface (PR): the same for three components;
* V.D  spinodal decomposition of ethane / n-pentane: equal fugacities in the two
       phases (iso-fugacity) and their values in bar against Table tabFug;
* V.E  oscillating propane / n-pentane droplet: the oscillation period against the
       paper's and against Lamb's period with the interfacial tension of Eq. eqMCsigma
       measured on a flat interface at the same conditions.

Step counts are shorter than the paper's (which ran 5e5 - 1e6 steps) where the bulk
values have settled well inside the bounds; the bounds and what was measured are
recorded with each case.
"""
import numpy as np
import pytest
from scipy.optimize import curve_fit

from cases import oracle_mixture, paper_cases, paper_mixture, slab_phases
from oracle.eos import lnf_density_form, pressure
from oracle.flash import flash, vapour_volume_fraction, volume_roots
from oracle.interface import crossing_radius, interfacial_tension, lamb_period
from paper_2212_10680_gb300 import inputs

pytestmark = pytest.mark.gpu
CASES = paper_cases()


@pytest.fixture(scope="module")
def fm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_10680_gb300 import fmlbm
    return fmlbm


def _relax(fm, mixd, rho, tau, steps, precision="fp64", stencil="central"):
    n, ny, nx = rho.shape
    lat = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, tau, stencil, precision, "lagged")
    lat.init(rho)
    lat.step(steps)
    r, u, lnf = lat.moments()  # raises on a latched non-physical state
    lat.close()
    return r, u, lnf


def _errors_percent(mix, M, L, V, z):
    """Relative errors (%) of Eq. eqerror against the flash at the vapour's pressure."""
    f = flash(mix, float(pressure(mix, V)), z)
    pct = lambda a, b: 100.0 * np.abs(a - b) / np.abs(b)
    dens = [pct((L * M).sum(), (f["rtL"] * M).sum()), pct((V * M).sum(), (f["rtV"] * M).sum())]
    comp = [pct(L / L.sum(), f["x"]), pct(V / V.sum(), f["y"])]
    return np.array(dens), np.array(comp)


def _flat_case(c, eos):
    mixd, sc = paper_mixture(c["components"], c["T_K"], eos, c["kappa"])
    mix = oracle_mixture(mixd)
    M = np.array(mixd["M"])
    f = flash(mix, c["p_bar"] * sc["p"], c["z"])
    rho = inputs.slab(f["rtV"] * M, f["rtL"] * M, c["nx"], c["ny"], vapour_volume_fraction(f), c["W"])
    return mixd, mix, M, rho


@pytest.mark.parametrize("eos", ["pr", "srk"])
def test_v_a_propane_pentane_flat_interface(fm, eos):
    # paper (Table tabcase1error): every relative error below 3e-4 %, after 1e6 steps.
    # Here, after the same 1e6 FP64 steps, bulk phases as node-pair means: density 2.7e-4 % /
    # 1.4e-4 %, compositions 1.0e-3 % / 5.3e-4 % (PR / SRK; after 5e5 steps the bulk is still
    # relaxing, up to 0.04 %); bound 2e-3 %.  Single nodes carry the alternation of the two
    # node parities (3.5e-5 / 8.8e-5 of the density) and stay about 5e-4 % / 2e-3 % off.
    c = CASES["c3c5_flat"]
    mixd, mix, M, rho = _flat_case(c, eos)
    r, u, _ = _relax(fm, mixd, rho, c["tau"], c["steps"])
    L, V = slab_phases(r, M)
    dens, comp = _errors_percent(mix, M, L, V, c["z"])
    print(eos, "density error %", dens, "composition error %", comp)
    assert np.max(dens) < 2e-3 and np.max(comp) < 2e-3, (dens, comp)
    assert np.max(np.abs(lnf_density_form(mix, L) - lnf_density_form(mix, V))) < 1e-4


def test_v_a_error_against_steps(fm):
    """V.A (PR) out to 2e6 steps: the pair-mean phases keep converging to the flash at the
    lattice's pressure (measured 1.8e-7 % in density, 6.6e-7 % in composition at 2e6 steps,
    1.3e-8 % / 4.8e-8 % at 4e6), far below Table tabcase1error's 3e-4 %, while single nodes
    stop near 5e-4 % / 2e-3 % from 1e6 steps on: the gap between the paper's table and a
    node-by-node reading is the alternation of the node parities, not unfinished relaxation."""
    c = CASES["c3c5_flat"]
    mixd, mix, M, rho = _flat_case(c, "pr")
    lat = fm.Lattice(fm.mixture_from_dict(mixd), c["nx"], c["ny"], c["tau"], "central", "fp64", "lagged")
    lat.init(rho)
    node_err = []
    for target in (1000000, 2000000):
        lat.step(1000000)
        r, u, _ = lat.moments()
        pair = _errors_percent(mix, M, *slab_phases(r, M), c["z"])
        node = _errors_percent(mix, M, *slab_phases(r, M, pair=False), c["z"])
        node_err.append(max(np.max(node[0]), np.max(node[1])))
        print(target, "pair %", pair, "node %", node)
    lat.close()
    assert np.max(pair[0]) < 1e-5 and np.max(pair[1]) < 1e-5, pair
    assert node_err[1] > 1e-4 and abs(node_err[1] / node_err[0] - 1) < 0.5, node_err


def test_v_c_methane_ethane_propane_flat_interface(fm):
    # paper (Table tabcase3, after 1e6 steps): density errors 0.07 %, composition errors up to
    # 0.92 %.  Here, after the same 1e6 FP64 steps, bulk phases as node-pair means: density
    # 0.078 %, compositions up to 0.91 % (single nodes: 0.14 % and 1.6 %, the alternation of
    # the node parities is 1.2e-3 of the density); bounds 0.1 % and 1.0 %.
    # The thin liquid slab (vapour fraction 0.78) translates slowly, so the bulk phases
    # are located on the profile rather than at fixed nodes.
    # The overall composition for the flash is the lattice's own (three components: the
    # phase compositions depend on it).
    c = CASES["c1c2c3_flat"]
    mixd, mix, M, rho = _flat_case(c, "pr")
    r, u, _ = _relax(fm, mixd, rho, c["tau"], 1000000)
    L, V = slab_phases(r, M)
    z = (r / M[:, None, None]).sum(axis=(1, 2))
    dens, comp = _errors_percent(mix, M, L, V, z / z.sum())
    print("ternary density error %", dens, "composition error %", comp)
    assert np.max(dens) < 0.1, dens
    assert np.max(comp) < 1.0, comp


def test_v_d_spinodal_decomposition_iso_fugacity(fm):
    # paper (Table tabFug): liquid 35.1276 / 4.4563 bar, vapour 35.1262 / 4.4567 bar.
    # A uniform C2/C5 state at 50 bar (the single volume root at x = 0.62 / 0.38) with a
    # seeded 1% fluctuation of the total density separates within 5e5 steps (the paper's
    # count).  FP64: at the densest and the least dense node the fugacities agree to 1e-3
    # (4e-4 measured) and lie within 1% of the table's (0.35% measured; the final pressure
    # depends on the curvature the separation ends with, which depends on the
    # fluctuation).  FP32 storage separates the same way but its fugacities agree only to
    # about 4e-3 (the force balance is computed in single precision).
    c = CASES["spinodal"]
    mixd, sc = paper_mixture(c["components"], c["T_K"], "pr", c["kappa"])
    mix = oracle_mixture(mixd)
    M = np.array(mixd["M"])
    x = np.array(c["x"])
    v = np.sort(volume_roots(mix, c["p_bar"] * sc["p"], x))
    rt = x / v[len(v) // 2]
    xi = inputs.uniform_noise(7, 0, 0, c["nx"] * c["ny"]).reshape(c["ny"], c["nx"])
    rho = (rt * M)[:, None, None] * (1.0 + 0.01 * xi)[None]
    r, u, _ = _relax(fm, mixd, rho, c["tau"], c["steps"], precision="fp64", stencil="isotropic")
    tot = r.sum(axis=0)
    assert tot.max() / tot.min() > 2.5  # two phases
    a = np.unravel_index(np.argmax(tot), tot.shape)
    b = np.unravel_index(np.argmin(tot), tot.shape)
    fL = np.exp(lnf_density_form(mix, r[:, a[0], a[1]] / M)) / sc["p"]   # bar
    fV = np.exp(lnf_density_form(mix, r[:, b[0], b[1]] / M)) / sc["p"]
    print("fugacities (bar) liquid", fL, "vapour", fV)
    assert np.max(np.abs(fL / fV - 1)) < 1e-3, (fL, fV)
    paper = 0.5 * (np.array(c["fugacity_liquid_bar"]) + np.array(c["fugacity_vapor_bar"]))
    assert np.max(np.abs(fL / paper - 1)) < 0.01, (fL, paper)


def test_v_e_oscillating_droplet_period(fm):
    # paper: period 1787.5 steps from the lattice, 1717.5 from Eq. eqPeriod (its sigma
    # is not printed).  Exploratory run here: about 1765 steps from the lattice and about
    # 1753 from Eq. eqPeriod with sigma of Eq. eqMCsigma on a flat interface at the same
    # state; bounds 3% against each.
    c = CASES["oscillating_droplet"]
    mixd, sc = paper_mixture(c["components"], c["T_K"], "pr", c["kappa"])
    mix = oracle_mixture(mixd)
    M = np.array(mixd["M"])
    f = flash(mix, c["p_bar"] * sc["p"], [0.4, 0.6])
    rhoL, rhoV = (f["rtL"] * M).sum(), (f["rtV"] * M).sum()
    assert abs(rhoL / rhoV - c["mass_density_ratio"]) < 0.006
    nx, ny = c["nx"], c["ny"]
    rho = inputs.droplet(f["rtV"] * M, f["rtL"] * M, nx, ny, c["R0"], c["W"], c["h"])
    lat = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, c["tau"], "isotropic", "fp64", "lagged")
    lat.init(rho)
    level = 0.5 * (rhoL + rhoV)
    t, rx = [], []
    for k in range(0, c["steps"] + 1, 10):
        if k:
            lat.step(10)
        tot = lat.moments()[0].sum(axis=0)
        t.append(k)
        rx.append(crossing_radius(tot[ny // 2, :], nx / 2, level))   # along the major (x) axis
    lat.close()
    t, rx = np.array(t, dtype=np.float64), np.array(rx)
    assert np.all(np.isfinite(rx))
    model = lambda s, A, T, ph, td, c0, c1: c0 + c1 * s + A * np.cos(2 * np.pi * s / T + ph) * np.exp(-s / td)
    p, _ = curve_fit(model, t, rx, p0=[rx[0] - rx[-1], 1750.0, 0.0, 2000.0, rx[-1], 0.0], maxfev=20000)
    period = abs(p[1])
    # sigma from a relaxed flat interface at the same state
    slab = inputs.slab(f["rtV"] * M, f["rtL"] * M, 200, 2, 0.5, c["W"])
    r1, _, _ = _relax(fm, mixd, slab, c["tau"], 100000, stencil="isotropic")
    sigma = interfacial_tension(r1[:, 0, :] / M[:, None], mixd["kappa"], n_interfaces=2)
    rho_liquid = float(r1[:, 0, 100].sum())
    Ta = lamb_period(sigma, rho_liquid, c["R0"] * np.sqrt(c["h"]), c["mode"])
    print("period", period, "Lamb", Ta, "sigma", sigma)
    assert abs(period / c["period_lbm_steps"] - 1) < 0.03, period
    assert abs(period / Ta - 1) < 0.03, (period, Ta)


def test_v_b_c2_c5_envelopes_in_one_batch(fm):
    # Section V.B: p-x points on the isotherms 274.96 K and 387.70 K and T-x points on the
    # isobars 30, 45 and 58 bar (200 x 2, tau 1.25, kappa (0.1, 0.2), W 4, S_V 0.5, 5e5
    # steps), all 18 lattices advanced together by one batch (each lattice its own mixture
    # temperature).  Phase compositions (x_C2 in the liquid, y_C2 in the vapour) against the
    # flash at each lattice's own pressure.  Measured on GB300 (FP64): below 0.01 % except
    # near the ends of the envelopes -- 0.12 % at 274.96 K / 10 bar and 4.7 % (liquid) at
    # 274.96 K / 4 bar, where the density ratio reaches 114 -- and 7e-3 % at 410 K / 58 bar
    # (density ratio 1.9, close to the critical locus).  Bounds: 0.05 % where the density
    # ratio is below 30, 0.2 % up to 50, 6 % beyond.
    c = CASES["c2c5_envelopes"]
    points = [(274.96, p) for p in (4.0, 10.0, 16.0, 22.0)] + [(387.70, p) for p in (13.0, 25.0, 40.0, 55.0)] + \
             [(T, 30.0) for T in (310.0, 360.0, 410.0, 450.0)] + [(T, 45.0) for T in (330.0, 380.0, 430.0)] + \
             [(T, 58.0) for T in (350.0, 380.0, 410.0)]
    b = fm.fmlbm_batch_create(2, "fp64", len(points))
    runs = []
    for T, p in points:
        mixd, sc = paper_mixture(c["components"], T, "pr", c["kappa"])
        mix = oracle_mixture(mixd)
        M = np.array(mixd["M"])
        f = flash(mix, p * sc["p"], [0.5, 0.5])
        rho = inputs.slab(f["rtV"] * M, f["rtL"] * M, c["nx"], c["ny"], c["S_V"], c["W"])
        L = fm.make_lattice(c["nx"], c["ny"], c["tau"], "central", "fp64", "lagged")
        runs.append((fm.fmlbm_batch_add(b, fm.mixture_from_dict(mixd), L, rho), T, p, mix, M))
    fm.fmlbm_batch_step(b, c["steps"])
    r = np.empty((2, c["ny"], c["nx"]))
    worst = []
    for slot, T, p, mix, M in runs:
        fm.fmlbm_batch_moments(b, slot, r)
        L, V = slab_phases(r, M)
        f = flash(mix, float(pressure(mix, V)), [0.5, 0.5])
        err = 100.0 * max(abs(L[0] / L.sum() - f["x"][0]) / f["x"][0], abs(V[0] / V.sum() - f["y"][0]) / f["y"][0])
        ratio = (L * M).sum() / (V * M).sum()
        bound = 0.05 if ratio < 30 else (0.2 if ratio < 50 else 6.0)
        worst.append((T, p, err, ratio))
        assert err < bound, (T, p, err, ratio)
    fm.fmlbm_batch_destroy(b)
    print("C2/C5 envelope errors (T, p, %, density ratio):", worst)
