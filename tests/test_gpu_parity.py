"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by
element on the same seeded inputs.

Tolerances (normwise, max |gpu - oracle| / max |oracle| per field): FP64 storage
1e-12, FP32 storage 1e-5; densities and distributions also element by element,
|gpu - oracle| <= tol |oracle| + 16 ulp of the field's maximum.  Grid sizes span several 32 x 8 tiles with ragged tails
in both directions, plus degenerate lattices (one row, one column, a single node).
"""
import numpy as np
import pytest

from cases import (mixture_dict, normwise, oracle_mixture, run_oracle, slab_state_binary, smooth_state,
                   workloads)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def fm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_10680_gb300 import fmlbm
    return fmlbm


def _gpu_run(fm, mixd, rho, tau, stencil, precision, velocity_force, steps, record, formulation="well_balanced"):
    lat = fm.Lattice(fm.mixture_from_dict(mixd), rho.shape[2], rho.shape[1], tau, stencil, precision, velocity_force,
                     formulation=formulation)
    lat.init(rho)
    out = {}
    done = 0
    for k in sorted(record):
        lat.step(k - done)
        done = k
        g, F = lat.distributions()
        r, u, lnf = lat.moments()
        out[k] = dict(g=g, F=F, rho=r, u=u, lnf=lnf)
    lat.close()
    return out


EPS32 = float(np.finfo(np.float32).eps)
EPS64 = float(np.finfo(np.float64).eps)
# absolute floor of the per-element checks, in units of the storage type's eps times the
# field's largest value: room for the rounding of the terms that cancel in a small value
# (a vapour density, a near-zero distribution), far below the normwise budget (1e-5 of the
# maximum is 84 FP32 ulp of it; 1e-12 is 4500 FP64 ulp)
FLOOR_ULPS = 16


def elementwise_ratio(a, b, tol, eps):
    """max over elements of |a - b| / (tol |b| + FLOOR_ULPS eps max|b|): <= 1 means every
    element meets the relative tolerance up to a floor of a few ulp of the field's maximum."""
    b = np.asarray(b, dtype=np.float64)
    den = tol * np.abs(b) + FLOOR_ULPS * eps * np.max(np.abs(b))
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - b) / np.maximum(den, 1e-300)))


def _compare(gpu, ora, tol, mixd=None, fields=("rho", "u", "lnf", "g", "F")):
    """Normwise comparison per field: max |gpu - oracle| <= tol max |oracle|.

    In FP32 the force F_i = rho~_i (G_i - RT grad ln f_i) is a difference quotient, so its
    error follows the errors of what it differentiates rather than the size of F:
      |dF| <= tol max|F| + RT max(rho~) (32 eps32 max|ln f| + max|d ln f|) + 8 max(kappa) max(rho~) max|d rho|
    (rounding of ln f, the propagated ln f and density errors through the stencils), and the
    velocity inherits half of it divided by the smallest total density."""
    worst = {}
    for k in ora:
        o, gk = ora[k], gpu[k]
        extra_F = 0.0
        if tol >= 1e-6 and mixd is not None:
            RT = mixd["R"] * mixd["T"]
            rmax = np.max(o["rho"])
            d_lnf = np.max(np.abs(gk["lnf"] - o["lnf"]))
            d_rho = np.max(np.abs(gk["rho"] - o["rho"]))
            extra_F = (RT * rmax * (32 * EPS32 * np.max(np.abs(o["lnf"])) + d_lnf)
                       + 8 * max(mixd["kappa"]) * rmax * d_rho)
        for f in fields:
            a, b = gk[f], o[f]
            err = np.max(np.abs(a - b))
            bound = tol * np.max(np.abs(b))
            if f == "F":
                bound += extra_F
            elif f == "u":
                bound += 0.5 * extra_F / np.min(o["rho"].sum(axis=0))
            worst[f] = max(worst.get(f, 0.0), err / max(bound, 1e-300))
            assert err <= bound, f"step {k} field {f}: max error {err:.3e} > bound {bound:.3e}"
        # densities and distributions element by element (vapour nodes and small g_a included)
        eps = EPS64 if tol < 1e-9 else EPS32
        for f in ("rho", "g"):
            q = elementwise_ratio(gk[f], o[f], tol, eps)
            worst[f + "_elem"] = max(worst.get(f + "_elem", 0.0), q)
            assert q <= 1.0, f"step {k} field {f}: an element exceeds tol |oracle| + {FLOOR_ULPS} ulp of max ({q:.3f})"
    return worst


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("stencil", ["isotropic", "central"])
def test_binary_slab_parity(fm, precision, stencil):
    # two-phase binary slab of the flat-interface workloads: 70 x 37 spans 3 x 5 tiles
    mixd, rho = slab_state_binary(70, 37, seed=11)
    rec = (1, 2, 10, 40)
    ora = run_oracle(mixd, rho, 1.0, stencil, "lagged", max(rec), rec)
    gpu = _gpu_run(fm, mixd, rho, 1.0, stencil, precision, "lagged", max(rec), rec)
    _compare(gpu, ora, TOL[precision], mixd)


def test_small_binary_fp64_two_thousand_steps(fm):
    # The small parity configuration: the binary slab on 64 x 64 in FP64 for 2000 steps
    # (tau 1, isotropic stencils, lagged force, 1% noise), compared at steps 1, 2, 10, 100,
    # 1000 and 2000.  rho, g and ln f: 1e-12 of their largest value.  F and u decay towards
    # zero as the slab equilibrates while the terms that cancel in them stay O(1), so their
    # rounding differences are bounded relative to those terms: 1e-12 RT max(rho~) max|ln f|
    # for F (the size of rho~ RT grad ln f) and half of that over the smallest total density
    # for u = (j + F/2) / rho.  (Perturbing the oracle's input by 1e-15 moves F by 3e-15 and u
    # by 3e-16 at every one of these steps.)  Component masses: conserved to 1e-13.
    mixd, rho = slab_state_binary(64, 64, seed=1)
    rec = (1, 2, 10, 100, 1000, 2000)
    ora = run_oracle(mixd, rho, 1.0, "isotropic", "lagged", max(rec), rec)
    gpu = _gpu_run(fm, mixd, rho, 1.0, "isotropic", "fp64", "lagged", max(rec), rec)
    RT = mixd["R"] * mixd["T"]
    for k in rec:
        o, gk = ora[k], gpu[k]
        for f in ("rho", "g", "lnf"):
            assert normwise(gk[f], o[f]) <= 1e-12, (k, f, normwise(gk[f], o[f]))
        for f in ("rho", "g"):
            q = elementwise_ratio(gk[f], o[f], 1e-12, EPS64)
            assert q <= 1.0, (k, f, q)
        f_scale = RT * float(np.max(o["rho"])) * float(np.max(np.abs(o["lnf"])))
        dF = float(np.max(np.abs(gk["F"] - o["F"])))
        du = float(np.max(np.abs(gk["u"] - o["u"])))
        assert dF <= 1e-12 * f_scale, (k, dF, f_scale)
        assert du <= 1e-12 * (float(np.max(np.abs(o["u"]))) + 0.5 * f_scale / float(np.min(o["rho"].sum(axis=0)))), (k, du)
    mass0 = rho.sum(axis=(1, 2))
    assert np.max(np.abs(gpu[2000]["rho"].sum(axis=(1, 2)) / mass0 - 1)) <= 1e-13


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("eos", ["pr", "srk", "vdw"])
def test_components_and_eos_parity(fm, n, eos, precision):
    # every component count and EOS branch, in FP64 and in FP32 storage (for two components
    # the FP32 step is the parked, plane-addressed form)
    mixd = mixture_dict(n=n, eos=eos, Tr=1.05, kappa_scale=0.5, M=[1.0, 1.7, 0.8, 2.2][:n], kij=0.03)
    rho = smooth_state(n, 45, 19, seed=5 + n)
    rec = (1, 5, 20)
    ora = run_oracle(mixd, rho, 0.9, "isotropic", "lagged", max(rec), rec)
    gpu = _gpu_run(fm, mixd, rho, 0.9, "isotropic", precision, "lagged", max(rec), rec)
    _compare(gpu, ora, TOL[precision], mixd if precision == "fp32" else None)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_current_force_reading_parity(fm, precision):
    mixd = mixture_dict(n=2, Tr=1.1, kappa_scale=0.2)
    rho = smooth_state(2, 33, 9, seed=2)
    rec = (1, 3, 15)
    ora = run_oracle(mixd, rho, 0.8, "central", "current", max(rec), rec)
    gpu = _gpu_run(fm, mixd, rho, 0.8, "central", precision, "current", max(rec), rec)
    _compare(gpu, ora, TOL[precision], mixd)


@pytest.mark.parametrize("shape", [(1, 1), (1, 40), (40, 1), (2, 3), (5, 7), (64, 2), (3, 33)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_degenerate_lattices(fm, shape, precision):
    # one node, one row, one column, lattices smaller than the 2-node halo: every tile
    # wraps onto itself (FP32: the parked two-component form)
    nx, ny = shape
    mixd = mixture_dict(n=2, Tr=1.05, kappa_scale=0.5)
    rho = smooth_state(2, nx, ny, seed=nx * 100 + ny)
    rec = (1, 4)
    ora = run_oracle(mixd, rho, 1.0, "isotropic", "lagged", max(rec), rec)
    gpu = _gpu_run(fm, mixd, rho, 1.0, "isotropic", precision, "lagged", max(rec), rec)
    _compare(gpu, ora, TOL[precision], mixd if precision == "fp32" else None)


def test_ternary_slab_parity(fm):
    wl = workloads()["ternary"]
    from paper_2212_10680_gb300 import inputs
    rho = inputs.with_noise(inputs.slab(wl["slab"]["rt_vapour"], wl["slab"]["rt_liquid"], 96, 20, 0.5, 4.0),
                            0.01, 3)
    rec = (1, 25)
    for precision in ("fp64", "fp32"):
        ora = run_oracle(wl["mixture"], rho, 1.0, "isotropic", "lagged", max(rec), rec)
        gpu = _gpu_run(fm, wl["mixture"], rho, 1.0, "isotropic", precision, "lagged", max(rec), rec)
        _compare(gpu, ora, TOL[precision], wl["mixture"])


def test_set_distributions_mid_run(fm):
    # start both sides from an oracle state with flow (not a rest state)
    mixd, rho = slab_state_binary(40, 24, seed=4)
    from oracle import lbm
    mix = oracle_mixture(mixd)
    lat_o = lbm.Lattice(tau=1.0, stencil="isotropic")
    g, F = lbm.init_at_rest(rho)
    g, F = lbm.run(g, F, mix, lat_o, 15)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 40, 24, 1.0, "isotropic", "fp64", "lagged")
    lat.set_distributions(g, F)
    g0, F0 = lat.distributions()
    assert normwise(g0, g) == 0.0 and normwise(F0, F) == 0.0
    lat.step(5)
    g1, F1 = lbm.run(g, F, mix, lat_o, 5)
    gg, FF = lat.distributions()
    assert normwise(gg, g1) < 1e-12 and normwise(FF, F1) < 1e-12
    lat.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mass_conservation_and_diagnostics(fm, precision):
    mixd, rho = slab_state_binary(96, 40, seed=8)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 96, 40, 1.0, "isotropic", precision, "lagged")
    lat.init(rho)
    m0, r0, s0 = lat.diagnostics()
    assert s0 == 0 and np.isinf(r0)
    assert np.allclose(m0, rho.sum(axis=(1, 2)), rtol=1e-7 if precision == "fp32" else 1e-13)
    lat.step(300)
    rho_a, _, _ = lat.moments()
    m1, r1, s1 = lat.diagnostics()
    assert s1 == 300
    tol = 1e-13 if precision == "fp64" else 2e-5
    assert np.max(np.abs(m1 / m0 - 1)) < tol
    # residual definition: ||rho(t) - rho(t_prev)|| / ||rho(t)||
    lat.step(50)
    rho_b, _, _ = lat.moments()
    m2, r2, s2 = lat.diagnostics()
    expect = np.sqrt(np.sum((rho_b - rho_a) ** 2)) / np.sqrt(np.sum(rho_b ** 2))
    assert abs(r2 / expect - 1) < (1e-10 if precision == "fp64" else 1e-5)
    lat.close()


def test_checkpoint_resume_is_bitwise(fm):
    mixd, rho = slab_state_binary(50, 30, seed=9)
    for precision in ("fp64", "fp32"):
        a = fm.Lattice(fm.mixture_from_dict(mixd), 50, 30, 1.0, "isotropic", precision, "lagged")
        a.init(rho)
        a.step(20)
        state = fm.fmlbm_get_state(a.h)
        a.step(30)
        ga, Fa = a.distributions()
        b = fm.Lattice(fm.mixture_from_dict(mixd), 50, 30, 1.0, "isotropic", precision, "lagged")
        fm.fmlbm_set_state(b.h, state)
        b.step(30)
        gb, Fb = b.distributions()
        assert np.array_equal(ga, gb) and np.array_equal(Fa, Fb)
        a.close()
        b.close()


def test_nonphysical_state_is_reported(fm):
    mixd = mixture_dict(n=2, Tr=1.05)
    rho = smooth_state(2, 20, 10, seed=1)
    rho[1, 6, 13] = -1e-3
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 20, 10, 1.0, "isotropic", "fp64", "lagged")
    lat.init(rho)
    lat.step(1)
    with pytest.raises(fm.FmlbmError) as ei:
        lat.synchronize()
    assert ei.value.status == fm.E_NONPHYSICAL
    assert fm.fmlbm_error_node(lat.h) == (1, 13, 6)
    # a fresh init clears the latch
    lat.init(smooth_state(2, 20, 10, seed=2))
    lat.step(2)
    lat.synchronize()
    lat.close()


def test_invalid_arguments_are_rejected(fm):
    mixd = mixture_dict(n=2)
    with pytest.raises(fm.FmlbmError) as ei:
        fm.Lattice(fm.mixture_from_dict(mixd), 0, 10, 1.0)
    assert ei.value.status == 1
    with pytest.raises(fm.FmlbmError):
        fm.Lattice(fm.mixture_from_dict(mixd), 10, 10, 0.5)
    bad = fm.mixture_from_dict(mixd)
    bad.n_components = 5
    with pytest.raises(fm.FmlbmError):
        fm.Lattice(bad, 10, 10, 1.0)


def test_full_size_sampled_parity(fm):
    # the 1024 x 1024 binary droplet in FP32 (the throughput configuration): after some
    # steps, one more GPU step is compared at sampled nodes with the oracle applied to a
    # periodic patch of radius 5 around each node (the update of a node depends only on
    # the state within 4 nodes).
    from oracle import lbm
    from paper_2212_10680_gb300 import inputs
    wl = workloads()["binary"]
    n = 1024
    rho = inputs.with_noise(inputs.droplet(wl["slab"]["rt_vapour"], wl["slab"]["rt_liquid"], n, n, 200.0, 4.0),
                            0.01, 2)
    lat = fm.Lattice(fm.mixture_from_dict(wl["mixture"]), n, n, 1.0, "isotropic", "fp32", "lagged")
    lat.init(rho)
    lat.step(30)
    g, F = lat.distributions()
    lat.step(1)
    g1, F1 = lat.distributions()
    lat.close()
    mix = oracle_mixture(wl["mixture"])
    olat = lbm.Lattice(tau=1.0, stencil="isotropic", velocity_force="lagged")
    rng = np.random.default_rng(0)
    # nodes on the droplet interface, in the bulk and at the periodic edges
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (512, 512 + 200), (512 + 141, 512 + 141)]
    pts += [tuple(p) for p in rng.integers(0, n, (20, 2))]
    R = 5
    for (y, x) in pts:
        ys = np.arange(y - R, y + R + 1) % n
        xs = np.arange(x - R, x + R + 1) % n
        gp = g[:, :, ys][:, :, :, xs].astype(np.float64)
        Fp = F[:, ys][:, :, xs]
        go, Fo = lbm.step(gp, mix, olat, Fp)
        ref = go[:, :, R, R]
        got = g1[:, :, y, x]
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(g1)), (y, x)
        # force bound as in _compare: FP32 rounding of ln f enters through its gradient
        lnf_scale = 20.0  # |ln f| of the binary workload stays below this (ln of the trace density)
        dF = 32 * float(np.finfo(np.float32).eps) * mix.RT * float(np.max(rho)) * lnf_scale
        assert np.max(np.abs(F1[:, y, x] - Fo[:, R, R])) <= 1e-5 * np.max(np.abs(F1)) + dF, (y, x)


@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
def test_full_size_sampled_parity_ternary(fm, precision):
    # the 4096 x 4096 ternary slab (the second throughput configuration) in the storage
    # forms the benchmark times: one GPU step after 30 is compared at sampled nodes with the
    # oracle applied to a periodic patch around each node.  BF16 deviation storage rounds the
    # stored g_a (a != 0) to 8 significant bits (FP16: 11): |error| <= 2^-8 |g_a| (2^-11) on top
    # of the FP32 bound; g_0 and the force are stored in FP32.
    from oracle import lbm
    from paper_2212_10680_gb300 import inputs
    wl = workloads()["ternary"]
    n = 4096
    rho = inputs.with_noise(inputs.slab(wl["slab"]["rt_vapour"], wl["slab"]["rt_liquid"], n, n, 0.5, 4.0), 0.01, 3)
    lat = fm.Lattice(fm.mixture_from_dict(wl["mixture"]), n, n, 1.0, "isotropic", precision, "lagged")
    lat.init(rho)
    del rho
    lat.step(30)
    g, F = lat.distributions()
    lat.step(1)
    g1, F1 = lat.distributions()
    lat.close()
    mix = oracle_mixture(wl["mixture"])
    olat = lbm.Lattice(tau=1.0, stencil="isotropic", velocity_force="lagged")
    rng = np.random.default_rng(1)
    # both slab interfaces (x = n/4, 3n/4), the bulk phases and the periodic edges
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (2048, 1024), (100, 3072), (4000, 2048), (3, 10)]
    pts += [tuple(p) for p in rng.integers(0, n, (16, 2))]
    R = 5
    gmax = float(np.max(np.abs(g1)))
    rel = np.zeros((g1.shape[1], 1))
    if precision in ("fp16dev", "bf16dev"):
        rel[1:] = 2.0 ** -8 if precision == "bf16dev" else 2.0 ** -11
    for (y, x) in pts:
        ys = np.arange(y - R, y + R + 1) % n
        xs = np.arange(x - R, x + R + 1) % n
        gp = g[:, :, ys][:, :, :, xs].astype(np.float64)
        Fp = F[:, ys][:, :, xs]
        go, Fo = lbm.step(gp, mix, olat, Fp)
        ref = go[:, :, R, R]
        got = g1[:, :, y, x]
        bound = 1e-5 * gmax + rel.T * np.abs(ref)
        assert np.all(np.abs(got - ref) <= bound), (y, x, float(np.max(np.abs(got - ref) - bound)))
        lnf = lbm.moments(gp, Fp, mix, olat)["lnf"]
        dF = 32 * EPS32 * mix.RT * float(np.max(gp.sum(axis=1))) * float(np.max(np.abs(lnf)))
        assert np.max(np.abs(F1[:, y, x] - Fo[:, R, R])) <= 1e-5 * np.max(np.abs(F1)) + dF, (y, x)


def test_tile_heights_are_bit_identical(fm):
    mixd, rho = slab_state_binary(100, 70, seed=12)
    out = []
    for ty in (8, 16, 32):
        lat = fm.Lattice(fm.mixture_from_dict(mixd), 100, 70, 1.0, "isotropic", "fp32", "lagged")
        fm.fmlbm_set_step_variant(lat.h, "plain")
        fm.fmlbm_set_tile_height(lat.h, ty)
        lat.init(rho)
        lat.step(25)
        out.append(lat.distributions())
        lat.close()
    for k in (1, 2):
        assert np.array_equal(out[0][0], out[k][0]) and np.array_equal(out[0][1], out[k][1])


@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("shape", [(200, 100), (96, 24)])
def test_step_variants_are_bit_identical(fm, precision, n, shape):
    # 200 x 100: ragged in both directions, many wrap-free inner tiles for the bulk-copy
    # path, a last paired tile half outside the lattice; 96 x 24: the smallest kind of
    # lattice with one row of inner tiles.  The paired step packs two nodes per float
    # operation; the others run one node per thread: the same bits per node.
    from paper_2212_10680_gb300 import inputs
    nx, ny = shape
    wl = workloads()["binary" if n == 2 else "ternary"]
    rho = inputs.with_noise(inputs.slab(wl["slab"]["rt_vapour"], wl["slab"]["rt_liquid"], nx, ny, 0.5, 4.0),
                            0.01, 5)
    out = []
    for variant in ("plain", "tma", "tma_tile", "pair"):
        lat = fm.Lattice(fm.mixture_from_dict(wl["mixture"]), nx, ny, 1.0, "isotropic", precision, "lagged")
        fm.fmlbm_set_step_variant(lat.h, variant)
        assert fm.fmlbm_get_step_variant(lat.h) == variant
        lat.init(rho)
        lat.step(30)
        out.append(lat.distributions())
        lat.close()
    for k in (1, 2, 3):
        assert np.array_equal(out[0][0], out[k][0]) and np.array_equal(out[0][1], out[k][1]), k


@pytest.mark.parametrize("precision", ["fp32", "bf16dev"])
@pytest.mark.parametrize("velocity_force", ["lagged", "current"])
@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(70, 37), (5, 7), (64, 8), (130, 17), (1, 40)])
def test_paired_step_is_bit_identical_to_plain(fm, precision, velocity_force, n, shape):
    # every component count and both readings of the velocity, lattices narrower than one
    # paired tile, exactly one tile, and ragged ones (the second node of a pair outside)
    nx, ny = shape
    mixd = mixture_dict(n=n, Tr=1.05, kappa_scale=0.5 if velocity_force == "lagged" else 0.2,
                        M=[1.0, 1.7, 0.8, 2.2][:n], kij=0.03)
    rho = smooth_state(n, nx, ny, seed=31 + n + nx)
    out = []
    for variant in ("plain", "pair"):
        lat = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, 0.9, "isotropic", precision, velocity_force)
        fm.fmlbm_set_step_variant(lat.h, variant)
        lat.init(rho)
        lat.step(12)
        out.append(lat.distributions())
        lat.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_tma_path_oracle_parity(fm):
    # the persistent bulk-copy step against the oracle
    mixd, rho = slab_state_binary(136, 40, seed=13)
    rec = (1, 10, 30)
    ora = run_oracle(mixd, rho, 1.0, "isotropic", "lagged", max(rec), rec)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 136, 40, 1.0, "isotropic", "fp32", "lagged")
    fm.fmlbm_set_step_variant(lat.h, "tma")
    lat.init(rho)
    gpu, done = {}, 0
    for k in rec:
        lat.step(k - done)
        done = k
        g, F = lat.distributions()
        r, u, lnf = lat.moments()
        gpu[k] = dict(g=g, F=F, rho=r, u=u, lnf=lnf)
    lat.close()
    _compare(gpu, ora, TOL["fp32"], mixd)


def test_tma_unavailable_is_reported(fm):
    mixd, _ = slab_state_binary(70, 37)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 70, 37, 1.0, "isotropic", "fp32", "lagged")
    assert fm.fmlbm_get_step_variant(lat.h) == "plain"   # the default (nx not a multiple of 4 either)
    fm.fmlbm_set_step_variant(lat.h, "pair")             # the paired step has no shape condition
    assert fm.fmlbm_get_step_variant(lat.h) == "pair"
    with pytest.raises(fm.FmlbmError) as ei:
        fm.fmlbm_set_step_variant(lat.h, "tma")
    assert ei.value.status == 8
    lat.close()
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 64, 64, 1.0, "isotropic", "fp64", "lagged")
    assert fm.fmlbm_get_step_variant(lat.h) == "plain"   # the FP64 reference path has no TMA or paired variant
    with pytest.raises(fm.FmlbmError) as ei:
        fm.fmlbm_set_step_variant(lat.h, "pair")
    assert ei.value.status == 8
    lat.close()


def test_autotune_keeps_results(fm):
    mixd, rho = slab_state_binary(256, 96, seed=14)
    a = fm.Lattice(fm.mixture_from_dict(mixd), 256, 96, 1.0, "isotropic", "fp32", "lagged")
    a.init(rho)
    variant, ty, ms = fm.fmlbm_autotune(a.h, 2)
    assert variant in ("plain", "tma", "tma_tile", "pair") and ty in (8, 16, 32) and ms > 0
    done = fm.fmlbm_diagnostics(a.h, 2)[2]
    a.step(7)
    g1, F1 = a.distributions()
    a.close()
    b = fm.Lattice(fm.mixture_from_dict(mixd), 256, 96, 1.0, "isotropic", "fp32", "lagged")
    fm.fmlbm_set_step_variant(b.h, "plain")
    b.init(rho)
    b.step(done + 7)
    g2, F2 = b.distributions()
    b.close()
    assert np.array_equal(g1, g2) and np.array_equal(F1, F2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("stencil,velocity_force", [("isotropic", "lagged"), ("central", "current")])
def test_standard_formulation_parity(fm, precision, stencil, velocity_force):
    # Section VI: Eq. eqLBE per component with the force of Eq. eqForceGen, against the
    # oracle's standard formulation (70 x 37: ragged tiles in both directions).  A smooth
    # near-critical field: the standard form drives the vapour of the benchmark slab at
    # 0.8 Tc negative within a few steps (its errors grow with the density ratio).
    mixd = mixture_dict(n=2, Tr=1.05 if velocity_force == "lagged" else 1.1, kappa_scale=0.5 if velocity_force ==
                        "lagged" else 0.2, M=[1.0, 1.6])
    rho = smooth_state(2, 70, 37, seed=18)
    rec = (1, 3, 12)
    ora = run_oracle(mixd, rho, 0.9, stencil, velocity_force, max(rec), rec, formulation="standard")
    gpu = _gpu_run(fm, mixd, rho, 0.9, stencil, precision, velocity_force, max(rec), rec, formulation="standard")
    _compare(gpu, ora, TOL[precision], mixd)


def test_standard_formulation_limits(fm):
    mixd, rho = slab_state_binary(64, 16, seed=19)
    # the 16-bit forms hold deviations from the well-balanced rest state only
    with pytest.raises(fm.FmlbmError) as ei:
        fm.Lattice(fm.mixture_from_dict(mixd), 64, 16, 1.0, "isotropic", "bf16dev", "lagged", formulation="standard")
    assert ei.value.status == 1
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 64, 64, 1.0, "isotropic", "fp32", "lagged", formulation="standard")
    with pytest.raises(fm.FmlbmError) as ei:
        fm.fmlbm_set_step_variant(lat.h, "tma_tile")
    assert ei.value.status == 8
    lat.close()
    # the rest state is w_a rho_i(r) in every direction, as the oracle's
    from oracle import lbm
    for precision, tol in (("fp64", 1e-15), ("fp32", 1e-7)):
        lat = fm.Lattice(fm.mixture_from_dict(mixd), 64, 16, 1.0, "isotropic", precision, "lagged",
                         formulation="standard")
        lat.init(rho)
        g, F = lat.distributions()
        lat.close()
        g_ref, _ = lbm.init_at_rest(rho, formulation="standard")
        assert np.max(np.abs(g - g_ref)) <= tol * np.max(np.abs(g_ref)) and not F.any()


@pytest.mark.parametrize("variant", ["tma_tile", "tma"])
def test_a_bounded_wait_that_runs_out_is_reported(fm, variant):
    # The bulk-copy steps wait for each tile's copy with a bounded number of polls.  With a
    # bound of zero the first wait of every block gives up at once: the block latches the
    # timeout, waits (at the default bound) for its copies in flight and leaves, and the next
    # synchronising call reports FMLBM_E_TIMEOUT.  Nothing faults: a new lattice on the same
    # context then steps as usual.
    mixd, rho = slab_state_binary(96, 24, seed=21)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 96, 24, 1.0, "isotropic", "fp32", "lagged")
    fm.fmlbm_set_step_variant(lat.h, variant)
    with pytest.raises(fm.FmlbmError) as ei:
        fm.fmlbm_set_wait_limit(lat.h, -1)
    assert ei.value.status == 1
    fm.fmlbm_set_wait_limit(lat.h, 0)
    lat.init(rho)
    lat.step(1)
    with pytest.raises(fm.FmlbmError) as ei:
        lat.synchronize()
    assert ei.value.status == fm.E_TIMEOUT
    lat.close()
    out = []
    for v in (variant, "plain"):
        lat = fm.Lattice(fm.mixture_from_dict(mixd), 96, 24, 1.0, "isotropic", "fp32", "lagged")
        fm.fmlbm_set_step_variant(lat.h, v)
        lat.init(rho)
        lat.step(5)
        lat.synchronize()
        out.append(lat.distributions())
        lat.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_large_lattice_beyond_the_former_index_limit(fm):
    # 16384 x 16384 with two components: 9 N nx ny = 4.8e9 distribution values, beyond 2^31
    # (the element indices of a plane stay 32-bit; planes are addressed by base address or a
    # 64-bit offset).  A uniform state must stay uniform, bit for bit (all gradients vanish),
    # and keep its mass.
    import torch
    n, side = 2, 16384
    mixd = mixture_dict(n=2, Tr=1.05)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), side, side, 1.0, "isotropic", "fp32", "lagged")
    rho = torch.empty((n, side, side), dtype=torch.float64, device="cuda")
    rho[0].fill_(0.8)
    rho[1].fill_(0.5)
    fm.fmlbm_init_device(lat.h, rho.data_ptr())
    del rho
    m0, _, _ = lat.diagnostics()
    lat.step(3)
    m1, r1, s1 = lat.diagnostics()
    lat.close()
    assert s1 == 3 and r1 == 0.0
    # FP32 storage holds float(0.8) and float(0.5) at every node; the sums are exact to ~2^-44
    expect = [float(np.float32(0.8)) * side * side, float(np.float32(0.5)) * side * side]
    assert np.allclose(m0, expect, rtol=1e-12, atol=0)
    assert np.array_equal(m0, m1)
