"""16-bit deviation storage (FP16DEV / BF16DEV) against the FP64 oracle.

With rho_0 = 0 (Eq. eqLBEMCb) the rest value of every g_a, a != 0, is w_a rho_0 = 0, so the
stored 16-bit value is the deviation itself; g_0 (close to rho_i) stays in float.  Each step
rounds every stored g_a (a != 0) once, with relative error at most eps16 (2^-11 for FP16,
2^-8 for BF16), so after k steps the distributions differ from the oracle by at most about
k eps16 max|g_a|, a != 0, plus the FP32 arithmetic error; the test allows 4x that bound.
The densities carry the sum of the nine rounding errors of each node.
"""
import numpy as np
import pytest

from cases import oracle_mixture, run_oracle, slab_state_binary, workloads

pytestmark = pytest.mark.gpu

EPS16 = {"fp16dev": 2.0 ** -11, "bf16dev": 2.0 ** -8, "fp16dev_lnf64": 2.0 ** -11, "bf16dev_lnf64": 2.0 ** -8}


@pytest.fixture(scope="module")
def fm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_10680_gb300 import fmlbm
    return fmlbm


@pytest.mark.parametrize("precision", ["fp16dev", "bf16dev", "fp16dev_lnf64", "bf16dev_lnf64"])
def test_deviation_storage_parity(fm, precision):
    mixd, rho = slab_state_binary(70, 37, seed=11)
    rec = (1, 5, 20)
    ora = run_oracle(mixd, rho, 1.0, "isotropic", "lagged", max(rec), rec)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 70, 37, 1.0, "isotropic", precision, "lagged")
    lat.init(rho)
    done = 0
    for k in rec:
        lat.step(k - done)
        done = k
        g, F = lat.distributions()
        r, u, lnf = lat.moments()
        go = ora[k]["g"]
        dev_max = np.max(np.abs(go[:, 1:]))
        bound_g = 4 * k * EPS16[precision] * dev_max + 1e-5 * np.max(np.abs(go))
        assert np.max(np.abs(g - go)) <= bound_g, (k, np.max(np.abs(g - go)), bound_g)
        bound_rho = 9 * bound_g
        assert np.max(np.abs(r - ora[k]["rho"])) <= bound_rho
    lat.close()


@pytest.mark.parametrize("precision", ["fp16dev", "bf16dev", "bf16dev_lnf64"])
def test_deviation_storage_conserves_mass_to_float_rounding(fm, precision):
    wl = workloads()["ternary"]
    from paper_2212_10680_gb300 import inputs
    rho = inputs.with_noise(inputs.slab(wl["slab"]["rt_vapour"], wl["slab"]["rt_liquid"], 128, 64, 0.5, 4.0),
                            0.01, 3)
    lat = fm.Lattice(fm.mixture_from_dict(wl["mixture"]), 128, 64, 1.0, "isotropic", precision, "lagged")
    lat.init(rho)
    m0, _, _ = lat.diagnostics()
    lat.step(200)
    m1, _, _ = lat.diagnostics()
    # the 16-bit rounding of the moving parts does not telescope; mass drifts by at most
    # the rounding of the streamed deviations over the run
    assert np.max(np.abs(m1 / m0 - 1)) < 200 * EPS16[precision] * 0.05
    lat.close()


@pytest.mark.parametrize("precision", ["fp16dev_lnf64", "bf16dev_lnf64"])
def test_lnf64_forms_evaluate_ln_f_in_double(fm, precision):
    # The _LNF64 forms evaluate ln f (Eq. eqfugupdatePR) in double from the float densities and
    # round it to float once: at every node it is the definition (the oracle's ln f at the same
    # densities, in FP64) rounded to float, to within one float ulp.  The all-float form carries
    # the rounding of its float evaluation on top (several ulp at some nodes).
    from oracle.eos import lnf_density_form
    mixd, rho = slab_state_binary(70, 37, seed=12)
    assert mixd["M"] == [1.0, 1.0]          # rho~_i = rho_i: the densities are the GPU's own floats
    worst = {}
    for prec in (precision, precision.replace("_lnf64", "")):
        lat = fm.Lattice(fm.mixture_from_dict(mixd), 70, 37, 1.0, "isotropic", prec, "lagged")
        lat.init(rho)
        lat.step(3)
        r, _, lnf = lat.moments()
        lat.close()
        ref = lnf_density_form(oracle_mixture(mixd), r).astype(np.float32)
        ulp = np.spacing(np.abs(ref))
        worst[prec] = float(np.max(np.abs(lnf.astype(np.float32) - ref) / ulp))
    assert worst[precision] <= 1.0, worst
    assert worst[precision.replace("_lnf64", "")] > worst[precision], worst
