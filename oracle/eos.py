"""Cubic equations of state, van der Waals mixing rules and log-fugacities (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Everything here follows Appendix C of the paper ("Common equations of state and
their respective fugacity expressions") and the density-explicit log-fugacity
forms recommended at the end of Section IV (Eqs. eqfugupdateVDW, eqfugupdateSRK,
eqfugupdatePR).  Notation: ``rt`` is the vector of component molar densities
rho~_i, ``v`` = 1 / sum_i rho~_i the molar volume, ``x`` the mole fractions,
``aa_ij`` the mixture attraction matrix (a alpha)_ij (plain a_ij for vdW).

Pins (tests/test_oracle_eos.py): critical point of every EOS at (Tc, Pc);
ideal-gas limit of ln f_i (Eq. eqfugdef2); Gibbs-Duhem at constant T; ln f_i
against the residual-chemical-potential integral of Eq. eqfug2 evaluated by
quadrature of the pressure alone; equality of the density form and the textbook
phi form where p > 0; pure-component reduction.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SQRT2 = np.sqrt(2.0)

# Appendix C constants: a_i = OMEGA_A R^2 Tc^2 / Pc,  b_i = OMEGA_B R Tc / Pc.
OMEGA = {
    "vdw": (27.0 / 64.0, 1.0 / 8.0),
    "srk": (0.4274802, 0.08664035),
    "pr": (0.457235529, 0.077796074),
}


def alpha_function(eos: str, omega: np.ndarray, Tr: np.ndarray) -> np.ndarray:
    """alpha_i(T) of Appendix C.  vdW has none (alpha = 1).

    SRK: [1 + (0.48 + 1.574 w - 0.176 w^2)(1 - Tr^0.5)]^2.
    PR:  two branches in the acentric factor w, split at w = 0.49.
    """
    omega = np.asarray(omega, dtype=np.float64)
    Tr = np.asarray(Tr, dtype=np.float64)
    if eos == "vdw":
        return np.ones_like(Tr)
    if eos == "srk":
        m = 0.48 + 1.574 * omega - 0.176 * omega**2
    elif eos == "pr":
        m_lo = 0.374640 + 1.54226 * omega - 0.26992 * omega**2
        m_hi = 0.379642 + 1.48503 * omega - 0.164423 * omega**2 + 0.016666 * omega**3
        m = np.where(omega <= 0.49, m_lo, m_hi)
    else:
        raise ValueError(f"unknown EOS {eos!r}")
    return (1.0 + m * (1.0 - np.sqrt(Tr))) ** 2


@dataclass
class Mixture:
    """A mixture at fixed temperature, in whatever consistent units R, T, Tc, Pc use.

    ``kij`` is the binary interaction matrix (called delta_ij in Appendix C);
    ``kappa`` the pure-component interface strengths (Eq. eqkappa); ``M`` the
    molar masses (Section III.B step 2).
    """

    eos: str
    R: float
    T: float
    Tc: np.ndarray
    Pc: np.ndarray
    omega: np.ndarray
    M: np.ndarray = None
    kappa: np.ndarray = None
    kij: np.ndarray = None
    a: np.ndarray = field(init=False)
    b: np.ndarray = field(init=False)
    aa: np.ndarray = field(init=False)      # (a alpha)_i
    aa_ij: np.ndarray = field(init=False)   # (a alpha)_ij

    def __post_init__(self):
        self.eos = self.eos.lower()
        self.Tc = np.atleast_1d(np.asarray(self.Tc, dtype=np.float64))
        self.Pc = np.atleast_1d(np.asarray(self.Pc, dtype=np.float64))
        self.omega = np.atleast_1d(np.asarray(self.omega, dtype=np.float64))
        n = self.Tc.size
        self.M = np.ones(n) if self.M is None else np.atleast_1d(np.asarray(self.M, dtype=np.float64))
        self.kappa = np.zeros(n) if self.kappa is None else np.atleast_1d(np.asarray(self.kappa, dtype=np.float64))
        self.kij = np.zeros((n, n)) if self.kij is None else np.asarray(self.kij, dtype=np.float64).reshape(n, n)
        oa, ob = OMEGA[self.eos]
        # Appendix C: a_i and b_i from the critical constants.
        self.a = oa * self.R**2 * self.Tc**2 / self.Pc
        self.b = ob * self.R * self.Tc / self.Pc
        self.aa = self.a * alpha_function(self.eos, self.omega, self.T / self.Tc)
        # Eq. eqmixingrulesaSRK2 (and eqmixingrulesavdW2): geometric mean times (1 - delta_ij).
        self.aa_ij = np.sqrt(np.outer(self.aa, self.aa)) * (1.0 - self.kij)

    @property
    def n(self) -> int:
        return self.Tc.size

    @property
    def RT(self) -> float:
        return self.R * self.T


def _as_columns(rt: np.ndarray) -> np.ndarray:
    rt = np.asarray(rt, dtype=np.float64)
    return rt.reshape(rt.shape[0], -1) if rt.ndim > 1 else rt.reshape(-1, 1)


def mixing(mix: Mixture, x: np.ndarray):
    """Van der Waals one-fluid mixing rules (Eqs. eqmixingrulesaSRK, eqmixingrulesbm).

    ``x`` has shape (N, ...).  Returns (b_m, S, aa_m) with S_i = sum_j x_j (a alpha)_ij,
    so that (a alpha)_m = sum_i x_i S_i = sum_i sum_j x_i x_j (a alpha)_ij.
    """
    x = np.asarray(x, dtype=np.float64)
    bm = np.tensordot(mix.b, x, axes=(0, 0))
    S = np.tensordot(mix.aa_ij, x, axes=(1, 0))
    aam = np.sum(x * S, axis=0)
    return bm, S, aam


def _attraction_denominator(eos: str, v, bm):
    """The attraction denominator D(v) of each EOS: p = RT/(v - b_m) - (a alpha)_m / D(v)."""
    if eos == "vdw":
        return v * v                                   # Eq. eqvdwEOS
    if eos == "srk":
        return v * (v + bm)                            # Eq. eqSRKEOS
    return v * v + 2.0 * bm * v - bm * bm              # Eq. eqPREOS


def pressure_from_volume(mix: Mixture, v, x):
    """Pressure of the EOS at molar volume v and composition x (Section III.B step 4)."""
    bm, _, aam = mixing(mix, x)
    return mix.RT / (v - bm) - aam / _attraction_denominator(mix.eos, v, bm)


def molar_state(mix: Mixture, rt: np.ndarray):
    """Section III.B step 2: total molar density, mole fractions and molar volume."""
    rt = np.asarray(rt, dtype=np.float64)
    rtot = np.sum(rt, axis=0)
    x = rt / rtot
    v = 1.0 / rtot
    return rtot, x, v


def pressure(mix: Mixture, rt: np.ndarray):
    """Pressure from the component molar densities rho~_i (steps 2-4 of Section III.B)."""
    _, x, v = molar_state(mix, rt)
    return pressure_from_volume(mix, v, x)


def lnf_density_form(mix: Mixture, rt: np.ndarray):
    """ln f_i evaluated directly from the local molar densities (steps 2-5).

    This is the form the paper recommends for the lattice because the pressure may
    be negative inside an interface (Section IV, Eqs. eqfugupdateVDW, eqfugupdateSRK,
    eqfugupdatePR): the term ln[(v - b_m) p / RT] of the textbook form is split so
    that no logarithm of p appears.  Written here term by term as printed.
    """
    rt = np.asarray(rt, dtype=np.float64)
    _, x, v = molar_state(mix, rt)
    bm, S, aam = mixing(mix, x)
    RT = mix.RT
    b = mix.b.reshape((-1,) + (1,) * (rt.ndim - 1))
    lnx = np.log(x)
    ln_free = np.log((v - bm) / RT)
    if mix.eos == "vdw":
        # Eq. eqfugupdateVDW
        return lnx + b / (v - bm) - ln_free - (2.0 / (RT * v)) * S
    p = pressure_from_volume(mix, v, x)
    rep = (b / bm) * (p * v / RT - 1.0)
    bracket = b / bm - (2.0 / aam) * S
    if mix.eos == "srk":
        # Eq. eqfugupdateSRK
        return lnx + rep - ln_free + (aam / (bm * RT)) * bracket * np.log(1.0 + bm / v)
    # Eq. eqfugupdatePR
    ratio = (v + (1.0 + SQRT2) * bm) / (v + (1.0 - SQRT2) * bm)
    return lnx + rep - ln_free + (aam / (2.0 * SQRT2 * bm * RT)) * bracket * np.log(ratio)


def ln_phi_textbook(mix: Mixture, v, x):
    """ln(f_i / (x_i p)) in the textbook form (Eqs. eqfugvdW, eqfugSRK, eqfugPR).

    Needs p > 0 (it takes ln[(v - b_m) p / RT]); used by the flash, where every
    phase is a bulk phase at positive pressure.
    """
    x = np.asarray(x, dtype=np.float64)
    bm, S, aam = mixing(mix, x)
    RT = mix.RT
    b = mix.b.reshape((-1,) + (1,) * (x.ndim - 1))
    p = pressure_from_volume(mix, v, x)
    Z = p * v / RT
    ln_zb = np.log((v - bm) * p / RT)
    if mix.eos == "vdw":
        return b / (v - bm) - ln_zb - (2.0 / (RT * v)) * S
    bracket = b / bm - (2.0 / aam) * S
    if mix.eos == "srk":
        return (b / bm) * (Z - 1.0) - ln_zb + (aam / (bm * RT)) * bracket * np.log(1.0 + bm / v)
    ratio = (v + (1.0 + SQRT2) * bm) / (v + (1.0 - SQRT2) * bm)
    return (b / bm) * (Z - 1.0) - ln_zb + (aam / (2.0 * SQRT2 * bm * RT)) * bracket * np.log(ratio)


def volume_roots(mix: Mixture, p: float, x) -> np.ndarray:
    """Real molar-volume roots v > b_m of p = RT/(v - b_m) - (a alpha)_m / D(v) at fixed p, x.

    Clearing denominators gives the cubic p (v - b_m) D(v) - RT D(v) + (a alpha)_m (v - b_m) = 0;
    its coefficients are built by polynomial products and solved with numpy.roots.
    """
    bm, _, aam = mixing(mix, np.asarray(x, dtype=np.float64))
    bm = float(bm)
    aam = float(aam)
    if mix.eos == "vdw":
        D = np.array([1.0, 0.0, 0.0])
    elif mix.eos == "srk":
        D = np.array([1.0, bm, 0.0])
    else:
        D = np.array([1.0, 2.0 * bm, -bm * bm])
    cubic = np.polymul([p, -p * bm], D)
    cubic = np.polysub(cubic, mix.RT * D)
    cubic = np.polyadd(cubic, [aam, -aam * bm])
    roots = np.roots(cubic)
    real = np.sort(roots[np.abs(roots.imag) <= 1e-9 * np.abs(roots.real)].real)
    real = real[real > bm]
    # polish each root with a few Newton steps on the cubic itself
    dcubic = np.polyder(cubic)
    out = []
    for v in real:
        for _ in range(4):
            d = np.polyval(dcubic, v)
            if d == 0.0:
                break
            v_new = v - np.polyval(cubic, v) / d
            if not (v_new > bm):
                break
            v = v_new
        out.append(float(v))
    return np.array(sorted(out))
