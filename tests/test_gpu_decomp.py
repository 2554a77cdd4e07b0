"""One lattice split into y-slabs with a halo exchange after every step (fmlbm_decomp_*)
against the same lattice undivided.

The streaming of Eq. eqLBEMCa (Section III.B, step 9) is periodic in y; each slab keeps three
ghost rows above and below its own rows (the reach of the fused step: the pulls of the 2-node
halo of rho~) and receives them from its neighbours after every step.  The slabs' own rows
must then be bit for bit those of the undivided lattice, for any number of slabs, storage
precision and velocity reading.  All slabs run on one GPU here (the copies between them are
the ones a multi-GPU split makes between devices).
"""
import numpy as np
import pytest

from cases import mixture_dict, slab_state_binary, smooth_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_10680_gb300 import fmlbm
    return fmlbm


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16dev"])
@pytest.mark.parametrize("nslabs", [2, 4])
def test_slabs_evolve_bit_identically_to_the_whole_lattice(fm, precision, nslabs):
    # the two-phase binary slab turned on its side, so that its interfaces cross the slab
    # boundaries: 70 x 64, 100 steps
    mixd, rho = slab_state_binary(64, 70, seed=41)
    rho = np.ascontiguousarray(np.transpose(rho, (0, 2, 1)))   # interfaces along x, crossing y-slabs
    n, ny, nx = rho.shape
    whole = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, 1.0, "isotropic", precision, "lagged")
    whole.init(rho)
    whole.step(100)
    g_ref, F_ref = whole.distributions()
    whole.close()
    d = fm.Decomposition(fm.mixture_from_dict(mixd), nx, ny, 1.0, nslabs, "isotropic", precision, "lagged")
    d.init(rho)
    d.step(100)
    g, F = d.distributions()
    d.close()
    assert np.array_equal(g, g_ref) and np.array_equal(F, F_ref)


def test_slabs_with_the_current_velocity_reading_and_central_stencils(fm):
    mixd = mixture_dict(n=3, Tr=1.1, kappa_scale=0.2, M=[1.0, 1.7, 0.8], kij=0.03)
    rho = smooth_state(3, 45, 36, seed=42)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 45, 36, 0.8, "central", "fp64", "current")
    lat.init(rho)
    lat.step(40)
    g_ref, F_ref = lat.distributions()
    lat.close()
    d = fm.Decomposition(fm.mixture_from_dict(mixd), 45, 36, 0.8, 3, "central", "fp64", "current")
    d.init(rho)
    d.step(40)
    g, F = d.distributions()
    d.close()
    assert np.array_equal(g, g_ref) and np.array_equal(F, F_ref)


def test_slab_shapes_are_checked(fm):
    mixd = mixture_dict(n=2)
    for ny, nslabs in ((30, 4), (8, 4), (10, 0)):      # not divisible; 2 rows per slab; no slab
        with pytest.raises(fm.FmlbmError) as ei:
            fm.Decomposition(fm.mixture_from_dict(mixd), 16, ny, 1.0, nslabs)
        assert ei.value.status == 1
