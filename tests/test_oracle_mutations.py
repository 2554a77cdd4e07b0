"""The oracle's pins bind it: a plausible mistake planted in a copy of the oracle (on the
CPU) -- a dropped term, a wrong sign, factor, weight or index, transposed operands --
makes at least one of the pin tests fail.  Each case applies one text substitution to
an oracle module, loads the result as a separate module, points the pin
tests at it and counts the pins that fail.  (The unmodified oracle passes every pin: the
regular runs of these test modules.)  oracle/eos.py, oracle/flash.py, oracle/lbm.py and
oracle/interface.py are covered."""
import os
import sys
import types

import pytest

import test_oracle_eos as TE
import test_oracle_flash as TF
import test_oracle_interface as TI
import test_oracle_lbm as TL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the planted mistakes make logarithms of negative numbers and failing quadratures on purpose
pytestmark = pytest.mark.filterwarnings("ignore")


def _mutated(module: str, old: str, new: str):
    src = open(os.path.join(ROOT, "oracle", module + ".py")).read()
    assert src.count(old) >= 1, f"{old!r} not in oracle/{module}.py"
    name = f"oracle._planted_{module}_{abs(hash((old, new)))}"
    mod = types.ModuleType(name)
    mod.__package__ = "oracle"
    mod.__file__ = os.path.join(ROOT, "oracle", module + ".py")
    sys.modules[name] = mod
    exec(compile(src.replace(old, new, 1), mod.__file__, "exec"), mod.__dict__)
    return mod


def _failures(pins) -> list:
    """The first pin (in the order given, cheapest first) that fails, or [] if none does."""
    for pin, args in pins:
        try:
            pin(*args)
        except (AssertionError, FloatingPointError, ValueError, ArithmeticError, RuntimeError) as e:
            return [(pin.__name__, args, type(e).__name__)]
    return []


EOS_NAMES = ("Mixture", "alpha_function", "ln_phi_textbook", "lnf_density_form", "pressure",
             "pressure_from_volume", "volume_roots")
EOS_PINS = [(TE.test_critical_point_of_each_eos, (e,)) for e in TE.EOSES] + \
           [(TE.test_ideal_gas_limit, (e,)) for e in TE.EOSES] + \
           [(TE.test_gibbs_duhem, (e,)) for e in TE.EOSES] + \
           [(TE.test_lnf_equals_residual_integral, (e,)) for e in TE.EOSES] + \
           [(TE.test_density_form_equals_textbook_form, (e,)) for e in TE.EOSES] + \
           [(TE.test_split_identical_component, (e,)) for e in TE.EOSES]

EOS_MISTAKES = {
    "wrong sign of the PR attraction term of ln f":
        ("lnx + rep - ln_free + (aam / (2.0 * SQRT2", "lnx + rep - ln_free - (aam / (2.0 * SQRT2"),
    "dropped b_i / b_m in the repulsion term":
        ("rep = (b / bm) * (p * v / RT - 1.0)", "rep = (p * v / RT - 1.0)"),
    "factor 2 lost in the attraction bracket of ln f":
        ("bracket = b / bm - (2.0 / aam) * S", "bracket = b / bm - (1.0 / aam) * S"),
    "wrong sign of b_m^2 in the PR denominator":
        ("return v * v + 2.0 * bm * v - bm * bm", "return v * v + 2.0 * bm * v + bm * bm"),
    "mole fractions dropped from (a alpha)_m":
        ("aam = np.sum(x * S, axis=0)", "aam = np.sum(S, axis=0)"),
    "ln x_i left out of the density form":
        ("    lnx = np.log(x)\n", "    lnx = 0.0 * np.log(x)\n"),
}


@pytest.mark.parametrize("mistake", sorted(EOS_MISTAKES))
def test_planted_eos_mistake_fails_a_pin(mistake, monkeypatch):
    mod = _mutated("eos", *EOS_MISTAKES[mistake])
    for n in EOS_NAMES:
        monkeypatch.setattr(TE, n, getattr(mod, n))
    assert _failures(EOS_PINS), f"no pin caught: {mistake}"


LBM_PINS = [(TL.test_d2q9_isotropy, ()), (TL.test_equilibrium_moments, (0.0,)), (TL.test_forcing_term_moments, ()),
            (TL.test_collision_adds_exactly_the_force_to_the_momentum, (0.8,)),
            (TL.test_collision_adds_exactly_the_force_to_the_momentum_lagged, (0.8,)),
            (TL.test_uniform_state_is_stationary, ("isotropic",)),
            (TL.test_mirror_and_transpose_symmetry, ("isotropic",)),
            (TL.test_mirror_and_transpose_symmetry, ("central",)),
            (TL.test_isotropic_equals_central_on_flat_fields, ()),
            (TL.test_mass_conservation, ("isotropic", "lagged"))]

LBM_MISTAKES = {
    "wrong diagonal weight":
        ("[1 / 36] * 4, dtype=np.float64)", "[1 / 18] * 4, dtype=np.float64)"),
    "forcing prefactor (1 - 1/(2 tau)) dropped":
        ("(1.0 - 1.0 / (2.0 * lat.tau)) * Fa", "1.0 * Fa"),
    "full force instead of half in the velocity":
        ("ux = (jx.sum(axis=0) + 0.5 * Fu_x) / rho_tot", "ux = (jx.sum(axis=0) + 1.0 * Fu_x) / rho_tot"),
    "wrong sign of the -u . grad rho part of the forcing term":
        ("tG = (-ux * grx - uy * gry)", "tG = (ux * grx + uy * gry)"),
    "factor 2 lost in the second-order equilibrium term":
        ("eu * eu / (2.0 * CS2 * CS2)", "eu * eu / (CS2 * CS2)"),
    "streaming with x and y swapped":
        ("shift=(E[a, 1], E[a, 0]), axis=(-2, -1))\n    if return_macro",
         "shift=(E[a, 0], E[a, 1]), axis=(-2, -1))\n    if return_macro"),
    "central Laplacian with -2 h":
        ("+ neighbour(h, 0, -1)\n                - 4.0 * h)", "+ neighbour(h, 0, -1)\n                - 2.0 * h)"),
    "force on one component with the other's density":
        ("Fx[i] = -rt[i] * mix.RT * glx - rt[i] * gmx", "Fx[i] = -rt[i - 1] * mix.RT * glx - rt[i] * gmx"),
    # the lagged reading of the velocity (the default on every hot path)
    "stored force of one component instead of the total":
        ("F_tot = np.stack([Fx.sum(axis=0), Fy.sum(axis=0)])", "F_tot = np.stack([Fx[0], Fy[0]])"),
    "stored force not advanced from step to step":
        ("        g, F_prev = step(g, mix, lat, F_prev)\n", "        g, _ = step(g, mix, lat, F_prev)\n"),
    "current force used under the lagged reading":
        ("Fu_x, Fu_y = F_prev[0], F_prev[1]", "Fu_x, Fu_y = Fx.sum(axis=0), Fy.sum(axis=0)"),
    "lagged force put into the velocity without the half":
        ("ux = (jx.sum(axis=0) + 0.5 * Fu_x) / rho_tot\n    uy = (jy.sum(axis=0) + 0.5 * Fu_y) / rho_tot",
         "ux = (jx.sum(axis=0) + Fu_x) / rho_tot\n    uy = (jy.sum(axis=0) + Fu_y) / rho_tot"),
}


@pytest.mark.parametrize("mistake", sorted(LBM_MISTAKES))
def test_planted_lbm_mistake_fails_a_pin(mistake, monkeypatch):
    mod = _mutated("lbm", *LBM_MISTAKES[mistake])
    monkeypatch.setattr(TL, "lbm", mod)
    assert _failures(LBM_PINS), f"no pin caught: {mistake}"


FLASH_NAMES = ("flash", "pure_coexistence", "slab_state", "bubble_point_from_liquid", "vapour_volume_fraction")
FLASH_PINS = [(TF.test_pure_coexistence_lattice_units_value, ()),
              (TF.test_pure_coexistence_obeys_equal_area, ("pr", 0.8)),
              (TF.test_flash_fugacity_equality_and_balance, (2,)),
              (TF.test_flash_fugacity_equality_and_balance, (3,)),
              (TF.test_table_tabfug_c2_c5_physical_units, ()),
              (TF.test_section_v_e_density_ratio_c3_c5_340K_5bar, ())]

FLASH_MISTAKES = {
    "K-value update inverted (vapour over liquid)":
        ("lnK_new = ln_phi_textbook(mix, vL, x) - ln_phi_textbook(mix, vV, y)",
         "lnK_new = ln_phi_textbook(mix, vV, y) - ln_phi_textbook(mix, vL, x)"),
    "liquid and vapour roots swapped":
        ('return float(roots[0] if phase == "liquid" else roots[-1])',
         'return float(roots[-1] if phase == "liquid" else roots[0])'),
    "Rachford-Rice liquid composition with K + 1":
        ("        x = z / (1.0 + beta * (K - 1.0))\n        y = K * x\n        x = x / x.sum()\n        y = y / y.sum()\n        vL",
         "        x = z / (1.0 + beta * (K + 1.0))\n        y = K * x\n        x = x / x.sum()\n        y = y / y.sum()\n        vL"),
    "coexistence from the liquid root twice":
        ('        vV = phase_volume(mix, p, x, "vapor")\n        return float(',
         '        vV = phase_volume(mix, p, x, "liquid")\n        return float('),
}


@pytest.mark.parametrize("mistake", sorted(FLASH_MISTAKES))
def test_planted_flash_mistake_fails_a_pin(mistake, monkeypatch):
    mod = _mutated("flash", *FLASH_MISTAKES[mistake])
    for n in FLASH_NAMES:
        monkeypatch.setattr(TF, n, getattr(mod, n))
    assert _failures(FLASH_PINS), f"no pin caught: {mistake}"


INTERFACE_NAMES = ("crossing_radius", "interfacial_tension", "lamb_period")
INTERFACE_PINS = [(TI.test_lamb_period_formula, ()), (TI.test_crossing_radius_of_a_sampled_tanh, ()),
                  (TI.test_tension_of_a_tanh_slab_matches_the_closed_form, ())]

INTERFACE_MISTAKES = {
    "kappa_ij = kappa_i kappa_j instead of its square root":
        ("k = np.sqrt(np.outer(kappa, kappa))", "k = np.outer(kappa, kappa)"),
    "cross terms kappa_ij (i != j) dropped":
        ("k = np.sqrt(np.outer(kappa, kappa))", "k = np.diag(np.asarray(kappa, dtype=float))"),
    "n (n^2 + 1) in the Lamb period":
        ("n * (n * n - 1) * sigma", "n * (n * n + 1) * sigma"),
    "crossing interpolated from the wrong node":
        ("return k + (p[k] - level) / (p[k] - p[k + 1]) - centre", "return k + 1 - (p[k] - level) / (p[k] - p[k + 1]) - centre"),
}


@pytest.mark.parametrize("mistake", sorted(INTERFACE_MISTAKES))
def test_planted_interface_mistake_fails_a_pin(mistake, monkeypatch):
    mod = _mutated("interface", *INTERFACE_MISTAKES[mistake])
    for n in INTERFACE_NAMES:
        monkeypatch.setattr(TI, n, getattr(mod, n))
    assert _failures(INTERFACE_PINS), f"no pin caught: {mistake}"


STANDARD_PINS = [(TL.test_standard_equilibrium_and_forcing_moments, ()),
                 (TL.test_standard_form_conserves_mass_and_keeps_a_uniform_state, ()),
                 (TL.test_standard_form_single_component_slab_deviates_slightly_from_maxwell, ())]

STANDARD_MISTAKES = {
    "wrong sign of c_s^2 grad rho_i in the force of Eq. eqForceGen":
        ("Fx[i] = Fx[i] + CS2 * grx[i]", "Fx[i] = Fx[i] - CS2 * grx[i]"),
    "the 1 dropped from the standard equilibrium rho_i w_a (1 + S)":
        ("geq[:, a] = W[a] * rho_i * (1.0 + S)", "geq[:, a] = W[a] * rho_i * S"),
}


@pytest.mark.parametrize("mistake", sorted(STANDARD_MISTAKES))
def test_planted_standard_form_mistake_fails_a_pin(mistake, monkeypatch):
    mod = _mutated("lbm", *STANDARD_MISTAKES[mistake])
    monkeypatch.setattr(TL, "lbm", mod)
    assert _failures(STANDARD_PINS), f"no pin caught: {mistake}"
