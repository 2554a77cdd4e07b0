"""Caller-owned device buffers (fmlbm_create_with_buffers): the same run as with the
handle's own buffers, bit for bit, and the storage stays the caller's."""
import numpy as np
import pytest

from cases import slab_state_binary

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_10680_gb300 import fmlbm
    return fmlbm


def _tensors(fm, precision, nx, ny):
    import torch
    gb, g0b, fb = fm.fmlbm_buffer_sizes(2, fm.make_lattice(nx, ny, 1.0, "isotropic", precision, "lagged"))
    mk = lambda n: [torch.zeros(n, dtype=torch.uint8, device="cuda") for _ in range(2)]  # noqa: E731
    return mk(gb), (mk(g0b) if g0b else None), mk(fb)


def _addr(ts, off=0):
    return None if ts is None else [t.data_ptr() + off for t in ts]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16dev"])
def test_caller_buffers_run_bit_identically(fm, precision):
    import torch
    nx, ny = 70, 37
    mixd, rho = slab_state_binary(nx, ny, seed=21)
    gt, g0t, ft = _tensors(fm, precision, nx, ny)
    out = []
    for bufs in (dict(g=_addr(gt), g0=_addr(g0t), force=_addr(ft)), None):
        lat = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, 1.0, "isotropic", precision, "lagged", buffers=bufs)
        lat.init(rho)
        lat.step(15)
        t = fm.fmlbm_diagnostics_async(lat.h)
        lat.step(2)
        out.append((lat.distributions(), fm.fmlbm_diagnostics_wait(lat.h, t, 2)))
        lat.close()
    (g1, F1), d1 = out[0]
    (g2, F2), d2 = out[1]
    assert np.array_equal(g1, g2) and np.array_equal(F1, F2)
    assert np.array_equal(np.asarray(d1[0]), np.asarray(d2[0])) and d1[1] == d2[1]
    # the handle ran in the caller's storage and freed none of it
    torch.cuda.synchronize()
    assert all(bool(t.any()) for t in gt + ft)
    for t in gt + ft + (g0t or []):
        t.fill_(1)
    torch.cuda.synchronize()


def test_caller_buffers_are_checked(fm):
    nx, ny = 64, 32
    mixd, _ = slab_state_binary(nx, ny)
    mix = fm.mixture_from_dict(mixd)
    gt, _, ft = _tensors(fm, "fp32", nx, ny)
    _, g0t, _ = _tensors(fm, "bf16dev", nx, ny)
    host = np.zeros(1 << 20, dtype=np.uint8)
    bad = [
        ("fp32", dict(g=_addr(gt, 4), g0=None, force=_addr(ft))),                        # unaligned
        ("fp32", dict(g=[host.ctypes.data] * 2, g0=None, force=_addr(ft))),              # host memory
        ("fp32", dict(g=_addr(gt), g0=_addr(g0t), force=_addr(ft))),                     # a = 0 planes not used
        ("bf16dev", dict(g=_addr(gt), g0=None, force=_addr(ft))),                        # a = 0 planes missing
        ("fp32", dict(g=[_addr(gt)[0]] * 2, g0=None, force=_addr(ft))),                  # both steps in one buffer
        ("fp32", dict(g=_addr(gt), g0=None, force=[_addr(ft)[1]] * 2)),                  # one force buffer twice
        ("fp32", dict(g=_addr(gt), g0=None, force=[_addr(gt)[0], _addr(ft)[1]])),        # force inside g
    ]
    for prec, bufs in bad:
        with pytest.raises(fm.FmlbmError) as ei:
            fm.Lattice(mix, nx, ny, 1.0, "isotropic", prec, "lagged", buffers=bufs)
        assert ei.value.status == 1, (prec, bufs)


def test_undersized_caller_buffers_are_rejected(fm):
    # a buffer whose own allocation is smaller than fmlbm_buffer_sizes asks for is refused
    # before any kernel could touch it (checked against the allocation that contains the
    # pointer: the cache is emptied so the half-size tensor gets an allocation of its own)
    import torch
    nx, ny = 512, 512
    mixd, _ = slab_state_binary(nx, ny)
    mix = fm.mixture_from_dict(mixd)
    gt, _, ft = _tensors(fm, "fp32", nx, ny)
    torch.cuda.empty_cache()
    half = [torch.zeros(gt[0].numel() // 2, dtype=torch.uint8, device="cuda") for _ in range(2)]
    with pytest.raises(fm.FmlbmError) as ei:
        fm.Lattice(mix, nx, ny, 1.0, "isotropic", "fp32", "lagged",
                   buffers=dict(g=_addr(half), g0=None, force=_addr(ft)))
    assert ei.value.status == 1
    # the full-size buffers are accepted
    lat = fm.Lattice(mix, nx, ny, 1.0, "isotropic", "fp32", "lagged", buffers=dict(g=_addr(gt), g0=None, force=_addr(ft)))
    lat.close()


def test_handles_on_two_threads_with_large_shared_tiles(fm):
    # Launch attributes are kept per device and set safely from any thread: two threads
    # create and step their own lattices at the same time with 32-row tiles of four FP64
    # components (the step then needs more than 48 KB of dynamic shared memory), and each
    # gets the result of the same lattice stepped alone.
    import threading
    from cases import mixture_dict, smooth_state
    mixd = mixture_dict(n=4, Tr=1.05, kappa_scale=0.5)
    rho = smooth_state(4, 40, 64, seed=70)

    def run(out, k):
        try:
            lat = fm.Lattice(fm.mixture_from_dict(mixd), 40, 64, 1.0, "isotropic", "fp64", "lagged")
            fm.fmlbm_set_step_variant(lat.h, "plain")
            fm.fmlbm_set_tile_height(lat.h, 32)
            lat.init(rho)
            lat.step(10)
            out[k] = lat.distributions()
            lat.close()
        except Exception as e:  # reported below
            out[k] = e

    out = [None, None]
    ts = [threading.Thread(target=run, args=(out, k)) for k in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not any(isinstance(o, Exception) for o in out), out
    ref = [None]
    run(ref, 0)
    for o in out:
        assert np.array_equal(o[0], ref[0][0]) and np.array_equal(o[1], ref[0][1])


@pytest.mark.parametrize("precision", ["fp32", "bf16dev"])
def test_init_from_page_locked_host_memory(fm, precision):
    # page-locked host densities are read in place by the initialisation kernel; the call waits
    # for the read, so the buffer may be overwritten on return: the state equals the one
    # initialised from ordinary (pageable) host memory
    import torch
    mixd, rho = slab_state_binary(100, 60, seed=8)
    pinned = torch.from_numpy(rho.copy()).pin_memory()
    pinned_np = pinned.numpy()
    out = []
    for src in (rho, pinned_np):
        lat = fm.Lattice(fm.mixture_from_dict(mixd), 100, 60, 1.0, "isotropic", precision, "lagged")
        lat.init(src)
        if src is pinned_np:
            pinned.fill_(-1.0)
        lat.step(3)
        out.append(lat.distributions())
        lat.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
