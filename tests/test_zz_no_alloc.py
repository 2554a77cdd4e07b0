"""The allocation-free reduction entry point against the regular one.

fmlbm_diagnostics_noalloc serves callers that cannot allocate device memory (a
host callback or real-time loop that must not block on cudaMalloc, a process whose
memory belongs to another allocator's pool, an embedding that forbids allocation
after start-up): they pass their own device buffers and the library uses a fixed
device array for its partial sums.  Here it must give the same component masses
and residual as fmlbm_diagnostics on the same states, on two calls in a row (the
second one reusing the density snapshot the first one wrote).

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from cases import slab_state_binary

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16dev": 1e-5, "bf16dev": 1e-5}
# D2Q9 directions in the library's order
E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]


def storage_layout(g):
    """Post-streaming g_a(r) -> the stored post-collision buffer b_a(r) = g_a(r + e_a)."""
    out = np.empty_like(g)
    for a, (ex, ey) in enumerate(E):
        out[:, a] = np.roll(g[:, a], shift=(-ey, -ex), axis=(-2, -1))
    return out


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_10680_gb300 import fmlbm
    return torch, fmlbm


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev", "bf16dev"])
def test_noalloc_matches_diagnostics_twice(env, precision):
    torch, fm = env
    nx, ny = 96, 40
    mixd, rho = slab_state_binary(nx, ny, seed=21)
    n = len(mixd["Tc"])
    dtype = torch.float64 if precision == "fp64" else torch.float32   # the storage arithmetic type
    dev16 = {"fp16dev": torch.float16, "bf16dev": torch.bfloat16}.get(precision)
    lat = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, 1.0, "isotropic", precision, "lagged")
    lat.init(rho)
    rho_prev = torch.zeros(n * ny * nx, dtype=dtype, device="cuda")
    out = torch.zeros(n + 2, dtype=torch.float64, device="cuda")
    have_prev = False
    for steps in (10, 7):
        lat.step(steps)
        g, _ = lat.distributions()
        mass_ref, res_ref, _ = lat.diagnostics()
        stored = storage_layout(g)
        g0 = None
        if dev16 is None:
            buf = torch.tensor(stored, dtype=dtype, device="cuda").contiguous()
        else:
            # the deviation forms keep a = 0 in float planes [N][ny][nx] and a = 1..8 in 16-bit
            # planes [N][8][ny][nx]; the handle's values convert exactly to either
            buf = torch.tensor(stored[:, 1:], dtype=dev16, device="cuda").contiguous()
            g0 = torch.tensor(stored[:, 0], dtype=torch.float32, device="cuda").contiguous()
        torch.cuda.synchronize()
        fm.fmlbm_diagnostics_noalloc(n, nx, ny, precision, buf.data_ptr(), 0 if g0 is None else g0.data_ptr(),
                                     rho_prev.data_ptr(), have_prev, out.data_ptr(), 0)
        torch.cuda.synchronize()
        res = out.cpu().numpy()
        mass = res[:n]
        assert np.max(np.abs(mass / mass_ref - 1)) <= TOL[precision]
        if have_prev:
            residual = np.sqrt(res[n] / res[n + 1])
            assert residual > 0 and abs(residual / res_ref - 1) <= TOL[precision]
        else:
            assert res[n] == 0.0 and np.isinf(res_ref)
        have_prev = True
    lat.close()


def test_noalloc_rejects_lattices_beyond_its_fixed_scratch(env):
    torch, fm = env
    tiny = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(fm.FmlbmError) as ei:
        # 4096 x 4096 with two components needs 65536 * 4 partial sums: above the fixed 65536
        fm.fmlbm_diagnostics_noalloc(2, 4096, 4096, "fp32", tiny.data_ptr(), 0, tiny.data_ptr(), False,
                                     tiny.data_ptr(), 0)
    assert ei.value.status == 1
    with pytest.raises(fm.FmlbmError):
        fm.fmlbm_diagnostics_noalloc(2, 8, 8, "fp32", 0, 0, tiny.data_ptr(), False, tiny.data_ptr(), 0)
    # buffers smaller than the lattice (a 512 x 512 lattice needs 19 MB: more than the whole
    # allocator segment the small tensor lives in, which is what the check can see), host
    # memory, and the deviation forms without their a = 0 planes
    with pytest.raises(fm.FmlbmError) as ei:
        fm.fmlbm_diagnostics_noalloc(2, 512, 512, "fp32", tiny.data_ptr(), 0, tiny.data_ptr(), False,
                                     tiny.data_ptr(), 0)
    assert ei.value.status == 1
    host = np.zeros(1 << 16, dtype=np.float64)
    with pytest.raises(fm.FmlbmError) as ei:
        fm.fmlbm_diagnostics_noalloc(1, 4, 4, "fp64", host.ctypes.data, 0, tiny.data_ptr(), False, tiny.data_ptr(), 0)
    assert ei.value.status == 1
    with pytest.raises(fm.FmlbmError) as ei:
        fm.fmlbm_diagnostics_noalloc(1, 4, 4, "bf16dev", tiny.data_ptr(), 0, tiny.data_ptr(), False, tiny.data_ptr(), 0)
    assert ei.value.status == 1
