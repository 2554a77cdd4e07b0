"""Equilibrium on the GPU against the FP64 flash oracle (flat interfaces, quasi-1-D strips).

The paper compares equilibrated flat-interface lattices with a flash at the lattice's own
pressure (Sections V.A-V.C).  Here a slab is run to a residual below 1e-12 per 10,000
steps and its bulk liquid (strip centre) and vapour (strip edge) are compared with:
* the Maxwell pair of the PR EOS for one component (tolerance 1e-4);
* the PT flash of the binary at the pressure of the lattice's bulk vapour (tolerance 3e-4,
  the accuracy the method reaches at this interface resolution; it degrades for sharper
  interfaces) and equal fugacities between the bulk phases.
The 1024 x 1024 droplet of the throughput benchmark is checked against the flash at its
vapour's pressure, for equal fugacities across the curved interface, and for Laplace's law.
"""
import numpy as np
import pytest

from cases import PC1, TC1, oracle_mixture, slab_phases, workloads
from oracle.eos import lnf_density_form, pressure
from oracle.flash import flash, pure_coexistence, slab_state
from oracle.interface import crossing_radius, interfacial_tension

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


def test_droplet_1024_fp32_against_the_flash(fm):
    # The throughput configuration's physics: the 1024 x 1024 binary droplet (radius 200,
    # FP32, tau 1, 1% noise) after 50,000 steps.  The curved interface compresses the liquid,
    # so the flat flash is not the liquid's reference: the vapour far from the droplet is
    # compared with the flash at its own pressure, and the droplet centre with the far vapour
    # (equal fugacities across the interface).  The bulk phases are read as means over 4 x 4
    # windows: the sharp interface leaves a node-to-node alternation in both phases that the
    # force does not see (the flat slab of the same mixture is 2-3 % off the flash node by node,
    # 1e-4 as a mean over node pairs).  Tolerance 1e-2: measured 4.8e-3 in density and
    # composition and 7.5e-3 in ln f after 50,000 steps, with the droplet still relaxing and
    # carrying spurious currents of about 1e-4 (FP32 cannot reach a 1e-8 residual).  The droplet keeps its size (crossing radius),
    # and Eq. eqMCsigma over its own profile gives the sigma of a flat interface of the same
    # mixture (a strip run alongside) to 2 %: at R / W ~ 50 the tension does not depend on
    # the curvature.
    import bench
    w = bench.workload("droplet1024")
    mixd = w["mixture"]
    mix = oracle_mixture(mixd)
    n = w["nx"]
    lat = fm.Lattice(fm.mixture_from_dict(mixd), n, n, w["tau"], w["stencil"], "fp32", "lagged")
    lat.init(w["rho"])
    lat.step(50000)
    r, u, lnf = lat.moments()
    lat.close()
    c = n // 2
    # 4 x 4 windows: an even number of nodes of each parity, so the node-to-node alternation
    # the sharp interface leaves in the bulk phases averages out
    L = r[:, c - 2:c + 2, c - 2:c + 2].mean(axis=(1, 2))      # droplet centre (M = 1: molar)
    V = r[:, 0:4, 0:4].mean(axis=(1, 2))                      # farthest from the droplet
    f = flash(mix, float(pressure(mix, V)), [0.5, 0.5])
    print("droplet: vapour density", np.max(np.abs(V / f["rtV"] - 1)), "composition",
          np.max(np.abs((V / V.sum() - f["y"]) / f["y"])), "ln f across",
          np.max(np.abs(lnf_density_form(mix, L) - lnf_density_form(mix, V))))
    assert np.max(np.abs(V / f["rtV"] - 1)) < 1e-2
    assert np.max(np.abs((V / V.sum() - f["y"]) / f["y"])) < 1e-2
    assert np.max(np.abs(lnf_density_form(mix, L) - lnf_density_form(mix, V))) < 1e-2
    row = r[:, c, :].astype(np.float64)                        # crosses two interfaces
    R = crossing_radius(row.sum(axis=0), c, 0.5 * (L.sum() + V.sum()))
    assert 190 < R < 210
    from paper_2212_10680_gb300 import inputs
    strip = inputs.slab(V, L, n, 4, 0.5, 4.0)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), n, 4, w["tau"], w["stencil"], "fp32", "lagged")
    lat.init(strip)
    lat.step(50000)
    rs, _, _ = lat.moments()
    lat.close()
    sigma_flat = interfacial_tension(rs[:, 2, :].astype(np.float64), mixd["kappa"], n_interfaces=2)
    sigma_drop = interfacial_tension(row, mixd["kappa"], n_interfaces=2)
    assert abs(sigma_drop / sigma_flat - 1) < 2e-2, (sigma_drop, sigma_flat)


@pytest.mark.parametrize("kscale,bound", [(1.0, 3e-4), (2.0, 5e-5)])
def test_benchmark_binary_slab_against_the_flash_as_node_pair_means(fm, kscale, bound):
    """The binary of the throughput benchmark (T = 0.8 Tc1, kappa = (0.05, 0.075) x kscale),
    flat slab from its flash at z = (0.5, 0.5), 256 x 4, FP64, 4e5 steps.  Its interface is
    three nodes wide (x1) or five (x2), and the transient leaves the bulk phases alternating
    from node to node (3.3e-2 and 5.3e-3 of the density), which the force does not see.  As
    node-pair means the phases match the flash at the lattice's vapour pressure to 1.0e-4 (x1)
    and 1.3e-5 (x2) in density and composition; node by node they are 1.9e-2 / 3.1e-2 (x1) and
    2.8e-3 / 5.1e-3 (x2) off.  kappa x3 leaves the EOS domain."""
    from paper_2212_10680_gb300 import inputs
    mixd = dict(workloads()["binary"]["mixture"])
    mixd["kappa"] = [k * kscale for k in mixd["kappa"]]
    mix = oracle_mixture(mixd)
    s = slab_state(mix, [0.5, 0.5])
    rho = inputs.slab(s["rtV"], s["rtL"], 256, 4, 0.5, 4.0)
    r, u, res = _equilibrate(fm, mixd, rho, 400000)
    M = np.ones(2)
    L, V = slab_phases(r[:, 2:3, :], M)
    Ln, Vn = slab_phases(r[:, 2:3, :], M, pair=False)

    def dev(L, V):
        f = flash(mix, float(pressure(mix, V)), [0.5, 0.5])
        return max(np.max(np.abs(L / f["rtL"] - 1)), np.max(np.abs(V / f["rtV"] - 1)),
                   np.max(np.abs(L / L.sum() - f["x"]) / f["x"]), np.max(np.abs(V / V.sum() - f["y"]) / f["y"]))
    pair, node = dev(L, V), dev(Ln, Vn)
    print(f"kappa x{kscale}: pair {pair:.2e} node {node:.2e}")
    assert pair < bound and node > 10 * pair, (pair, node)
    assert np.max(np.abs(u)) < 1e-8
