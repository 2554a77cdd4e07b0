"""Asynchronous diagnostics: the reduction fused into the next step against the separate
reduction kernel, bit for bit, and the ticket rules of fmlbm_diagnostics_async / _wait.

The fused form sums the same node values (the pulled densities the step reads anyway) in
the same shuffle tree and the same 32 x 8 strips as the separate kernel, so masses and
residuals must agree exactly, for every tile height and on ragged lattices; the state
the lattice reaches must not depend on whether diagnostics were asked for.
"""
import math

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


def _pair(fm, shape, precision, tile_y, seed):
    nx, ny = shape
    mixd, rho = slab_state_binary(nx, ny, seed=seed)
    lats = []
    for _ in range(2):
        lat = fm.Lattice(fm.mixture_from_dict(mixd), nx, ny, 1.0, "isotropic", precision, "lagged")
        fm.fmlbm_set_tile_height(lat.h, tile_y)
        lat.init(rho)
        lats.append(lat)
    return lats


def _same(a, b):
    ma, ra, sa = a
    mb, rb, sb = b
    assert sa == sb
    assert np.array_equal(ma, mb)
    assert (math.isinf(ra) and math.isinf(rb)) or ra == rb


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16dev"])
@pytest.mark.parametrize("tile_y", [8, 16, 32])
@pytest.mark.parametrize("shape", [(70, 37), (100, 61)])
def test_fused_diagnostics_bit_identical(fm, precision, tile_y, shape):
    ref, fused = _pair(fm, shape, precision, tile_y, seed=31)
    steps = 6
    expect = []
    for _ in range(steps):
        ref.step(1)
        expect.append(ref.diagnostics())  # requested and waited at once: the separate kernel
    tickets = []
    for _ in range(steps):
        fused.step(1)                     # computes the previous request inside its first step
        tickets.append(fm.fmlbm_diagnostics_async(fused.h))
    got = [fm.fmlbm_diagnostics_wait(fused.h, t, 2) for t in tickets[-3:]]  # the last one: separate kernel
    # the ring keeps four results: the earlier tickets have expired
    with pytest.raises(fm.FmlbmError) as ei:
        fm.fmlbm_diagnostics_wait(fused.h, tickets[0], 2)
    assert ei.value.status == 1
    for e, g in zip(expect[-3:], got):
        _same(e, g)
    g1, F1 = ref.distributions()
    g2, F2 = fused.distributions()
    assert np.array_equal(g1, g2) and np.array_equal(F1, F2)
    ref.close()
    fused.close()


def test_fused_diagnostics_every_step_read_behind(fm):
    # the pipelined loop of the end-to-end benchmark: ask every step, read two steps behind
    ref, fused = _pair(fm, (96, 40), "fp32", 8, seed=32)
    expect, got, tickets = [], [], []
    for k in range(8):
        ref.step(1)
        expect.append(ref.diagnostics())
        fused.step(1)
        tickets.append(fm.fmlbm_diagnostics_async(fused.h))
        if k >= 2:
            got.append(fm.fmlbm_diagnostics_wait(fused.h, tickets[k - 2], 2))
    for t in tickets[-2:]:
        got.append(fm.fmlbm_diagnostics_wait(fused.h, t, 2))
    assert [s for _, _, s in got] == list(range(1, 9))
    for e, g in zip(expect, got):
        _same(e, g)
    ref.close()
    fused.close()


def test_ticket_rules(fm):
    lat, other = _pair(fm, (64, 24), "fp32", 8, seed=33)
    t0 = fm.fmlbm_diagnostics_async(lat.h)
    assert fm.fmlbm_diagnostics_async(lat.h) == t0      # same state: same ticket
    first = fm.fmlbm_diagnostics_wait(lat.h, t0, 2)      # no step followed: separate kernel
    assert first[2] == 0 and math.isinf(first[1])
    _same(first, fm.fmlbm_diagnostics_wait(lat.h, t0, 2))  # waiting twice returns the same
    other_first = other.diagnostics()
    _same(first, other_first)
    lat.step(3)
    t1 = fm.fmlbm_diagnostics_async(lat.h)
    assert t1 != t0
    lat.init(slab_state_binary(64, 24, seed=33)[1])      # replaces the state before it was computed
    with pytest.raises(fm.FmlbmError) as ei:
        fm.fmlbm_diagnostics_wait(lat.h, t1, 2)
    assert ei.value.status == 1
    with pytest.raises(fm.FmlbmError):
        fm.fmlbm_diagnostics_wait(lat.h, 12345, 2)       # never issued
    lat.close()
    other.close()


def test_tma_variants_fuse_requests_with_the_same_bits(fm):
    # the bulk-copy step kernels serve requests inside the step too (same strips and sums);
    # 128 x 48 has wrap-free inner tiles for the copies and edge tiles for the pulls
    mixd, rho = slab_state_binary(128, 48, seed=34)
    outs = []
    for variant in ("plain", "tma_tile", "tma", "pair"):
        lat = fm.Lattice(fm.mixture_from_dict(mixd), 128, 48, 1.0, "isotropic", "fp32", "lagged")
        fm.fmlbm_set_step_variant(lat.h, variant)
        lat.init(rho)
        tickets = []
        for _ in range(4):
            lat.step(2)
            tickets.append(fm.fmlbm_diagnostics_async(lat.h))
        outs.append([fm.fmlbm_diagnostics_wait(lat.h, t, 2) for t in tickets])
        lat.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            _same(a, b)


def test_request_served_inside_a_captured_graph(fm):
    # A request pending while the handle's stream is captured is served on that stream
    # (no cross-stream events): the graph's first step computes it, and replaying the graph
    # gives the same state and diagnostics as stepping directly.
    import torch
    ref, lat = None, None
    mixd, rho = slab_state_binary(96, 40, seed=35)
    ref = fm.Lattice(fm.mixture_from_dict(mixd), 96, 40, 1.0, "isotropic", "fp32", "lagged")
    ref.init(rho)
    expect = ref.diagnostics()
    ref.step(2)
    g_ref, F_ref = ref.distributions()
    ref.close()
    s = torch.cuda.Stream()
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 96, 40, 1.0, "isotropic", "fp32", "lagged", stream=s.cuda_stream)
    lat.init(rho)
    fm.fmlbm_synchronize(lat.h)
    t = fm.fmlbm_diagnostics_async(lat.h)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        fm.fmlbm_step(lat.h, 2)
    graph.replay()
    torch.cuda.synchronize()
    _same(expect, fm.fmlbm_diagnostics_wait(lat.h, t, 2))
    g, F = lat.distributions()
    assert np.array_equal(g, g_ref) and np.array_equal(F, F_ref)
    lat.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16dev"])
def test_step_diagnostics_matches_the_per_step_loop(fm, precision):
    # fmlbm_step_diagnostics runs the per-step loop (ask, step, read three behind) inside the
    # library: the same rows, bit for bit, and the same final state; 0, 1, 2 and 9 steps
    # (fewer steps than the kept results, and more)
    mixd, rho = slab_state_binary(100, 60, seed=12)
    n = len(mixd["Tc"])
    for nsteps in (0, 1, 2, 9):
        ref, got = [], []
        lat = fm.Lattice(fm.mixture_from_dict(mixd), 100, 60, 1.0, "isotropic", precision, "lagged")
        lat.init(rho)
        tickets = []
        for k in range(nsteps):
            tickets.append(fm.fmlbm_diagnostics_async(lat.h))
            lat.step(1)
            if k >= 3:  # four results are kept: read three behind
                m, r, _ = fm.fmlbm_diagnostics_wait(lat.h, tickets[k - 3], n)
                ref.append((m, r))
        for t in tickets[max(0, nsteps - 3):]:
            m, r, _ = fm.fmlbm_diagnostics_wait(lat.h, t, n)
            ref.append((m, r))
        g0 = lat.distributions()
        lat.close()
        lat = fm.Lattice(fm.mixture_from_dict(mixd), 100, 60, 1.0, "isotropic", precision, "lagged")
        lat.init(rho)
        mass, res = fm.fmlbm_step_diagnostics(lat.h, nsteps, n)
        g1 = lat.distributions()
        lat.close()
        assert mass.shape == (nsteps, n) and res.shape == (nsteps,)
        for k, (m, r) in enumerate(ref):
            assert np.array_equal(mass[k], m) and (res[k] == r or (np.isinf(res[k]) and np.isinf(r))), (nsteps, k)
        assert np.array_equal(g0[0], g1[0]) and np.array_equal(g0[1], g1[1])
