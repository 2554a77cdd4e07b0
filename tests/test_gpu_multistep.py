"""The multi-step kernel (FMLBM_VARIANT_MULTI, temporal blocking): several time steps of the
periodic update (Eq. eqLBEMCa, Section III.B steps 1-9) in one cooperative launch, each tile
waiting only for its 3 x 3 neighbourhood of tiles to complete the previous step.

It performs the arithmetic of the single-step kernel, so K steps in one launch must give the
same bits as K single launches, whatever the lattice shape (ragged tiles, one row of tiles,
one tile, fewer tiles than resident blocks), the storage form and the way the steps are split
into calls.  Its waits are bounded: a bound of zero makes the first unsatisfied wait give up,
which the next synchronising call reports as FMLBM_E_TIMEOUT, and nothing is left hanging.
"""
import numpy as np
import pytest

from cases import slab_state_binary, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_10680_gb300 import fmlbm
    return fmlbm


def _slab(n, nx, ny, seed):
    from paper_2212_10680_gb300 import inputs
    wl = workloads()["binary" if n == 2 else "ternary"]
    rho = inputs.with_noise(inputs.slab(wl["slab"]["rt_vapour"], wl["slab"]["rt_liquid"], nx, ny, 0.5, 4.0),
                            0.01, seed)
    return wl["mixture"], rho


def _run(fm, mixd, rho, precision, variant, chunks, diag_at=()):
    ny, nx = rho.shape[1], rho.shape[2]
    lat = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, 1.0, "isotropic", precision, "lagged")
    fm.fmlbm_set_step_variant(lat.h, variant)
    lat.init(rho)
    sums = []
    for k, c in enumerate(chunks):
        t = fm.fmlbm_diagnostics_async(lat.h) if k in diag_at else None
        lat.step(c)
        if t is not None:
            sums.append(fm.fmlbm_diagnostics_wait(lat.h, t, len(mixd["Tc"]))[:2])
    lat.synchronize()
    g, F = lat.distributions()
    lat.close()
    return g, F, sums


@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("shape", [(200, 100), (130, 38), (64, 8), (32, 8), (40, 16), (1024, 64)])
def test_multi_step_launch_is_bit_identical_to_single_steps(fm, precision, n, shape):
    # 200 x 100 and 130 x 38: ragged tiles in both directions; 64 x 8 and 32 x 8: one row of
    # tiles and one tile (a tile is its own periodic neighbour); 40 x 16: four tiles, each
    # neighbour of all others; 1024 x 64: more tiles than some blocks have rounds
    nx, ny = shape
    mixd, rho = _slab(n, nx, ny, seed=7 + nx)
    g0, F0, _ = _run(fm, mixd, rho, precision, "plain", [41])
    for chunks in ([41], [2, 1, 17, 21]):
        g1, F1, _ = _run(fm, mixd, rho, precision, "multi", chunks)
        assert np.array_equal(g0, g1) and np.array_equal(F0, F1), chunks


def test_multi_step_serves_pending_diagnostics(fm):
    # a pending diagnostics request is served by a single step, the rest of the call runs in
    # one launch: same distributions and same sums as with single steps
    mixd, rho = _slab(2, 96, 40, seed=3)
    ref = _run(fm, mixd, rho, "fp32", "plain", [5, 7, 9], diag_at=(0, 2))
    got = _run(fm, mixd, rho, "fp32", "multi", [5, 7, 9], diag_at=(0, 2))
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    for (m0, r0), (m1, r1) in zip(ref[2], got[2]):
        assert np.array_equal(m0, m1) and r0 == r1


def test_multi_step_is_offered_only_where_it_exists(fm):
    # FP64 storage, the SRK EOS, central stencils and the current-force reading have no
    # multi-step kernel: asking for it is refused and the handle keeps its variant
    mixd, rho = slab_state_binary(64, 16, seed=4)
    for kwargs in (dict(precision="fp64"), dict(stencil="central"), dict(velocity_force="current")):
        args = dict(tau=1.0, stencil="isotropic", precision="fp32", velocity_force="lagged")
        args.update(kwargs)
        lat = fm.Lattice(fm.mixture_from_dict(mixd), 64, 16, args["tau"], args["stencil"], args["precision"],
                         args["velocity_force"])
        with pytest.raises(fm.FmlbmError) as ei:
            fm.fmlbm_set_step_variant(lat.h, "multi")
        assert ei.value.status == fm.E_UNSUPPORTED
        assert fm.fmlbm_get_step_variant(lat.h) == "plain"
        lat.close()
    srk = dict(mixd, eos="srk")
    lat = fm.Lattice(fm.mixture_from_dict(srk), 64, 16, 1.0, "isotropic", "fp32", "lagged")
    with pytest.raises(fm.FmlbmError) as ei:
        fm.fmlbm_set_step_variant(lat.h, "multi")
    assert ei.value.status == fm.E_UNSUPPORTED
    lat.close()


def test_a_multi_step_wait_that_runs_out_is_reported(fm):
    # 128 x 64: 32 tiles, one per block.  With a wait bound of zero, a block that finishes its
    # tile of step 0 before one of its neighbours finds that neighbour's counter behind and
    # gives up at once; the first block to finish always does.  The blocks waiting on the ones
    # that left give up too, the launch ends, and the next synchronising call reports the
    # timeout.  A new lattice then steps normally and matches single steps.
    mixd, rho = _slab(2, 128, 64, seed=11)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 128, 64, 1.0, "isotropic", "fp32", "lagged")
    fm.fmlbm_set_step_variant(lat.h, "multi")
    fm.fmlbm_set_wait_limit(lat.h, 0)
    lat.init(rho)
    lat.step(4)
    with pytest.raises(fm.FmlbmError) as ei:
        lat.synchronize()
    assert ei.value.status == fm.E_TIMEOUT
    lat.close()
    g0, F0, _ = _run(fm, mixd, rho, "fp32", "plain", [10])
    g1, F1, _ = _run(fm, mixd, rho, "fp32", "multi", [10])
    assert np.array_equal(g0, g1) and np.array_equal(F0, F1)
