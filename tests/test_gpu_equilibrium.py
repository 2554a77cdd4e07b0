"""Equilibrium on the GPU against the FP64 flash oracle (flat interfaces, quasi-1-D strips).

The paper compares equilibrated flat-interface lattices with a flash at the lattice's own
pressure (Sections V.A-V.C).  Here a slab is run to a residual below 1e-12 per 10,000
steps and its bulk liquid (strip centre) and vapour (strip edge) are compared with:
* the Maxwell pair of the PR EOS for one component (tolerance 1e-4);
* the PT flash of the binary at the pressure of the lattice's bulk vapour (tolerance 3e-4,
  the accuracy the method reaches at this interface resolution; it degrades for sharper
  interfaces) and equal fugacities between the bulk phases.
"""
import numpy as np
import pytest

from cases import PC1, TC1, oracle_mixture
from oracle.eos import lnf_density_form, pressure
from oracle.flash import flash, pure_coexistence, slab_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_10680_gb300 import fmlbm
    return fmlbm


def _equilibrate(fm, mixd, rho, steps):
    n, ny, nx = rho.shape
    lat = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, 1.0, "central", "fp64", "lagged")
    lat.init(rho)
    lat.diagnostics()
    res = np.inf
    for _ in range(steps // 10000):
        lat.step(10000)
        res = lat.diagnostics()[1]
    r, u, lnf = lat.moments()
    lat.close()
    return r, u, res


def test_single_component_slab_reaches_the_maxwell_pair(fm):
    from paper_2212_10680_gb300 import inputs
    mixd = dict(eos="pr", R=1.0, T=0.85 * TC1, Tc=[TC1], Pc=[PC1], omega=[0.011], M=[1.0], kappa=[0.1], kij=[0.0])
    mix = oracle_mixture(mixd)
    s = pure_coexistence(mix)
    rho = inputs.slab([s["rtV"]], [s["rtL"]], 256, 4, 0.5, 4.0)
    r, u, res = _equilibrate(fm, mixd, rho, 200000)
    assert res < 1e-12
    assert abs(r[0, 2, 128] / s["rtL"] - 1) < 1e-4
    assert abs(r[0, 2, 0] / s["rtV"] - 1) < 1e-4
    assert np.max(np.abs(u)) < 1e-8


def test_binary_slab_matches_the_flash_at_its_pressure(fm):
    from paper_2212_10680_gb300 import inputs
    mixd = dict(eos="pr", R=1.0, T=0.95 * TC1, Tc=[TC1, 1.3 * TC1], Pc=[PC1, 0.9 * PC1], omega=[0.011, 0.2],
                M=[1.0, 1.0], kappa=[0.10, 0.15], kij=[0.0, 0.0, 0.0, 0.0])
    mix = oracle_mixture(mixd)
    s = slab_state(mix, [0.5, 0.5])
    rho = inputs.slab(s["rtV"], s["rtL"], 256, 4, 0.5, 4.0)
    r, u, res = _equilibrate(fm, mixd, rho, 400000)
    assert res < 1e-8
    L, V = r[:, 2, 128], r[:, 2, 0]
    f = flash(mix, float(pressure(mix, V)), [0.5, 0.5])
    assert np.max(np.abs(L / f["rtL"] - 1)) < 3e-4
    assert np.max(np.abs(V / f["rtV"] - 1)) < 3e-4
    assert np.max(np.abs(L / L.sum() - f["x"]) / f["x"]) < 3e-4
    assert np.max(np.abs(V / V.sum() - f["y"]) / f["y"]) < 3e-4
    assert np.max(np.abs(lnf_density_form(mix, L) - lnf_density_form(mix, V))) < 1e-4
