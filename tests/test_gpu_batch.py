"""Batched lattices: bit-identical to single lattices, retirement, slots, autotuning."""
import numpy as np
import pytest

from cases import block_phases, mixture_dict, slab_state_binary, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_10680_gb300 import fmlbm
    return fmlbm


def _single(fm, mixd, rho, steps, precision, tile_y):
    ny, nx = rho.shape[1:]
    lat = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, 1.0, "isotropic", precision, "lagged")
    fm.fmlbm_set_step_variant(lat.h, "plain")
    fm.fmlbm_set_tile_height(lat.h, tile_y)
    lat.init(rho)
    lat.step(steps)
    out = lat.distributions()
    lat.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16dev"])
def test_batch_equals_single_lattices_bitwise(fm, precision):
    from paper_2212_10680_gb300 import inputs
    wl = workloads()
    sizes = [(70, 37), (64, 64), (100, 33), (40, 96)]
    b = fm.fmlbm_batch_create(2, precision, 8)
    cases = []
    for k, (nx, ny) in enumerate(sizes):
        st = wl["binary_sweep"][90 + 40 * k]   # mid-sweep feeds (the extreme ones diverge)
        mixd = dict(wl["binary"]["mixture"])
        if k == 3:
            mixd = mixture_dict(n=2, Tr=1.05, kappa_scale=0.5, M=[1.0, 1.7])
            rho = inputs.with_noise(np.stack([np.full((ny, nx), 1.0), np.full((ny, nx), 1.2)]), 0.01, 9)
        else:
            rho = inputs.with_noise(inputs.slab(st["rt_vapour"], st["rt_liquid"], nx, ny, 0.5, 4.0), 0.01, k)
        L = fm.make_lattice(nx, ny, 1.0, "isotropic", precision, "lagged")
        slot = fm.fmlbm_batch_add(b, fm.mixture_from_dict(mixd), L, rho)
        cases.append((slot, mixd, rho))
    fm.fmlbm_batch_step(b, 25)
    for slot, mixd, rho in cases:
        ny, nx = rho.shape[1:]
        g = np.empty((2, 9, ny, nx))
        F = np.empty((2, ny, nx))
        fm.fmlbm_batch_get_distributions(b, slot, g, F)
        gs, Fs = _single(fm, mixd, rho, 25, precision, 16)
        assert np.array_equal(g, gs) and np.array_equal(F, Fs), slot
    fm.fmlbm_batch_destroy(b)


@pytest.mark.parametrize("precision", ["fp32", "bf16dev"])
def test_batch_moments_equal_single_lattice_moments(fm, precision):
    # a lattice below 64 rows takes the 8-row moments kernel (for two components in float
    # storage the form that parks values and addresses planes through launch parameters),
    # a taller one the 16-row kernel; both against the single-lattice handle, bitwise
    from paper_2212_10680_gb300 import inputs
    wl = workloads()
    mixd = wl["binary"]["mixture"]
    b = fm.fmlbm_batch_create(2, precision, 4)
    cases = []
    for k, (nx, ny) in enumerate([(70, 37), (40, 96)]):
        st = wl["binary_sweep"][100 + 30 * k]
        rho = inputs.with_noise(inputs.slab(st["rt_vapour"], st["rt_liquid"], nx, ny, 0.5, 4.0), 0.01, 20 + k)
        L = fm.make_lattice(nx, ny, 1.0, "isotropic", precision, "lagged")
        cases.append((fm.fmlbm_batch_add(b, fm.mixture_from_dict(mixd), L, rho), rho))
    fm.fmlbm_batch_step(b, 10)
    for slot, rho in cases:
        ny, nx = rho.shape[1:]
        r, u, lnf = np.empty((2, ny, nx)), np.empty((2, ny, nx)), np.empty((2, ny, nx))
        fm.fmlbm_batch_moments(b, slot, r, u, lnf)
        lat = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, 1.0, "isotropic", precision, "lagged")
        lat.init(rho)
        lat.step(10)
        rs, us, ls = lat.moments()
        lat.close()
        assert np.array_equal(r, rs) and np.array_equal(u, us) and np.array_equal(lnf, ls), (nx, ny)
        # the phases: 2 x 2 block means of rho~ (= rho / M) at the blocks of largest and
        # smallest total molar density, first in row-major block order on ties, from the same
        # densities and in the same order of additions
        liq, vap = fm.fmlbm_batch_phases(b, slot, 2)
        want_l, want_v = block_phases(r, np.asarray(mixd["M"], dtype=np.float64))
        assert np.array_equal(liq, want_l) and np.array_equal(vap, want_v)
    fm.fmlbm_batch_destroy(b)


def test_batch_alone_equals_in_the_mix_and_after_retirements(fm):
    mixd, rho = slab_state_binary(64, 48, seed=3)
    alone = _single(fm, mixd, rho, 60, "fp32", 16)
    b = fm.fmlbm_batch_create(2, "fp32", 4)
    L = fm.make_lattice(64, 48, 1.0, "isotropic", "fp32", "lagged")
    s0 = fm.fmlbm_batch_add(b, fm.mixture_from_dict(mixd), L, rho)
    # a second lattice that is paused half way
    m2, r2 = slab_state_binary(96, 40, seed=5)
    s1 = fm.fmlbm_batch_add(b, fm.mixture_from_dict(m2), fm.make_lattice(96, 40, 1.0), r2)
    fm.fmlbm_batch_step(b, 30)
    fm.fmlbm_batch_set_active(b, s1, False)
    fm.fmlbm_batch_step(b, 30)
    assert fm.fmlbm_batch_slot_info(b, s0)[0] == 60 and fm.fmlbm_batch_slot_info(b, s1)[0] == 30
    g = np.empty((2, 9, 48, 64))
    F = np.empty((2, 48, 64))
    fm.fmlbm_batch_get_distributions(b, s0, g, F)
    assert np.array_equal(g, alone[0]) and np.array_equal(F, alone[1])
    fm.fmlbm_batch_remove(b, s1)
    fm.fmlbm_batch_destroy(b)


def test_batch_run_retires_each_lattice(fm):
    # uniform single-phase lattices are exactly stationary: residual 0 at the second check
    b = fm.fmlbm_batch_create(2, "fp32", 6)
    mixd = mixture_dict(n=2, Tr=1.1, kappa_scale=0.5)
    slots = []
    for k, n in enumerate((32, 48, 64)):
        rho = np.stack([np.full((n, n), 1.0 + 0.1 * k), np.full((n, n), 0.8)])
        slots.append(fm.fmlbm_batch_add(b, fm.mixture_from_dict(mixd), fm.make_lattice(n, n, 1.0), rho))
    # and one that cannot converge within the step limit
    m2, r2 = slab_state_binary(64, 64, seed=2)
    slow = fm.fmlbm_batch_add(b, fm.mixture_from_dict(m2), fm.make_lattice(64, 64, 1.0), r2)
    steps, res, st = fm.fmlbm_batch_run(b, 6, max_steps=400, check_every=100, tol=1e-12)
    for s in slots:
        assert st[s] == 0 and res[s] == 0.0 and steps[s] == 100
    assert st[slow] == fm.E_NOT_CONVERGED and steps[slow] == 400 and res[slow] > 1e-12
    fm.fmlbm_batch_destroy(b)


def test_batch_reports_a_nonphysical_lattice_without_stopping_others(fm):
    b = fm.fmlbm_batch_create(2, "fp64", 4)
    mixd = mixture_dict(n=2, Tr=1.1, kappa_scale=0.5)
    good = np.stack([np.full((24, 24), 1.0), np.full((24, 24), 0.8)])
    bad = good.copy()
    bad[0, 5, 7] = -0.5
    sg = fm.fmlbm_batch_add(b, fm.mixture_from_dict(mixd), fm.make_lattice(24, 24, 1.0, precision="fp64"), good)
    sb = fm.fmlbm_batch_add(b, fm.mixture_from_dict(mixd), fm.make_lattice(24, 24, 1.0, precision="fp64"), bad)
    steps, res, st = fm.fmlbm_batch_run(b, 4, max_steps=300, check_every=50, tol=1e-12)
    assert st[sb] == fm.E_NONPHYSICAL
    assert st[sg] == 0
    fm.fmlbm_batch_destroy(b)


def test_batch_autotune_keeps_results(fm):
    mixd, rho = slab_state_binary(128, 96, seed=7)
    b = fm.fmlbm_batch_create(2, "fp32", 2)
    s = fm.fmlbm_batch_add(b, fm.mixture_from_dict(mixd), fm.make_lattice(128, 96, 1.0), rho)
    ty, blocks, ms = fm.fmlbm_batch_autotune(b, 3)
    assert ty in (8, 16) and blocks > 0 and ms > 0
    steps = fm.fmlbm_batch_slot_info(b, s)[0]
    fm.fmlbm_batch_step(b, 10)
    g = np.empty((2, 9, 96, 128))
    fm.fmlbm_batch_get_distributions(b, s, g, None)
    ref = _single(fm, mixd, rho, steps + 10, "fp32", 16)[0]
    assert np.array_equal(g, ref)
    fm.fmlbm_batch_destroy(b)


def test_batch_against_the_oracle_on_ragged_lattices(fm):
    # three lattices of different shapes (ragged in both directions, one narrower than a tile)
    # and mixtures in one batch, each against the FP64 oracle on the same seeded input: the
    # FP32 bound of the single-lattice parity tests, normwise and element by element
    from cases import mixture_dict, run_oracle, smooth_state
    from test_gpu_parity import EPS32, elementwise_ratio
    cases = [((70, 37), mixture_dict(n=2, Tr=1.05, kappa_scale=0.5, M=[1.0, 1.7], kij=0.03)),
             ((40, 24), mixture_dict(n=2, Tr=1.1, kappa_scale=0.3)),
             ((21, 50), mixture_dict(n=2, eos="srk", Tr=1.05, kappa_scale=0.5))]
    b = fm.fmlbm_batch_create(2, "fp32", 4)
    slots = []
    for k, ((nx, ny), mixd) in enumerate(cases):
        rho = smooth_state(2, nx, ny, seed=60 + k)
        slots.append((fm.fmlbm_batch_add(b, fm.mixture_from_dict(mixd), fm.make_lattice(nx, ny, 0.9, "isotropic",
                                                                                        "fp32", "lagged"), rho),
                      rho, mixd))
    fm.fmlbm_batch_step(b, 20)
    for slot, rho, mixd in slots:
        ny, nx = rho.shape[1:]
        g = np.empty((2, 9, ny, nx))
        F = np.empty((2, ny, nx))
        fm.fmlbm_batch_get_distributions(b, slot, g, F)
        ora = run_oracle(mixd, rho, 0.9, "isotropic", "lagged", 20, (20,))[20]
        assert np.max(np.abs(g - ora["g"])) <= 1e-5 * np.max(np.abs(ora["g"])), (nx, ny)
        assert elementwise_ratio(g, ora["g"], 1e-5, EPS32) <= 1.0, (nx, ny)
    fm.fmlbm_batch_destroy(b)
