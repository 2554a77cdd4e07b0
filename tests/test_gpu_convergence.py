"""The phase measure and the PHASE convergence criterion on the GPU.

fmlbm_phase_measure (lambda_i = mean over the nodes of ln rho_i) against the oracle's
``lbm.phase_measure`` on the oracle's own densities, and against its definition on the
handle's densities; a batch's per-check phase change against the change of the
single-lattice measure; sweep lattices and served requests retiring at the criterion, with
their phases against the FP64 flash at their own vapour pressure.
"""
import numpy as np
import pytest

from cases import oracle_mixture, run_oracle, slab_state_binary, workloads
from oracle import lbm
from oracle.eos import pressure
from oracle.flash import flash

pytestmark = pytest.mark.gpu

TOL = 2e-6          # phase-measure change over one check interval of 500 steps
CHECK = 500


@pytest.fixture(scope="module")
def fm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_10680_gb300 import fmlbm
    return fmlbm


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_phase_measure_against_the_oracle(fm, precision, tol):
    mixd, rho = slab_state_binary(70, 37, seed=8)
    steps = 40
    lat = fm.Lattice(fm.mixture_from_dict(mixd), 70, 37, 1.0, "isotropic", precision, "lagged")
    lat.init(rho)
    lat.step(steps)
    lam = lat.phase_measure()
    r_gpu, _, _ = lat.moments()
    lat.close()
    # the definition, on the handle's own densities (the reduction alone)
    own = np.log(r_gpu).reshape(2, -1).mean(axis=1)
    assert np.max(np.abs(lam - own)) <= (1e-14 if precision == "fp64" else 1e-6)
    # the oracle's densities after the same steps (the step and the reduction)
    rec = run_oracle(mixd, rho, 1.0, "isotropic", "lagged", steps, record=(steps,))
    ref = lbm.phase_measure(rec[steps]["rho"])
    assert np.max(np.abs(lam - ref)) <= tol, (lam, ref)


def test_batch_phase_change_equals_the_single_lattice_measure(fm):
    cases = [slab_state_binary(64, 48, seed=3), slab_state_binary(96, 40, seed=5)]
    b = fm.fmlbm_batch_create(2, "fp32", 4)
    fm.fmlbm_batch_set_criterion(b, "phase")
    slots = [fm.fmlbm_batch_add(b, fm.mixture_from_dict(m), fm.make_lattice(r.shape[2], r.shape[1], 1.0), r)
             for m, r in cases]
    fm.fmlbm_batch_run_chunk(b, 100)       # first check: the snapshot
    assert all(np.isinf(fm.fmlbm_batch_slot_phase_change(b, s)) for s in slots)
    fm.fmlbm_batch_run_chunk(b, 150)
    for s, (m, r) in zip(slots, cases):
        lat = fm.Lattice(fm.mixture_from_dict(m), r.shape[2], r.shape[1], 1.0, "isotropic", "fp32", "lagged")
        lat.init(r)
        lat.step(100)
        l1 = lat.phase_measure()
        lat.step(150)
        l2 = lat.phase_measure()
        lat.close()
        want = float(np.max(np.abs(l2 - l1)))
        got = fm.fmlbm_batch_slot_phase_change(b, s)
        assert want > 1e-6 and abs(got - want) <= 1e-12 + 1e-9 * want, (got, want)
    fm.fmlbm_batch_destroy(b)


def _sweep_lattice(k, n):
    from paper_2212_10680_gb300 import inputs
    st = workloads()["binary_sweep"][k]
    return st, inputs.slab(st["rt_vapour"], st["rt_liquid"], n, n, 0.5, 4.0)


def test_sweep_lattices_retire_at_the_phase_criterion_near_the_flash(fm):
    """Unperturbed flat slabs of three sweep feeds (Section V.B initialisation) retire with
    FMLBM_OK; the residual criterion with the same tolerance would not retire them; their
    phases are within the accuracy of this interface resolution of the FP64 flash at their
    own vapour pressure, with equal fugacities across the interface."""
    wl = workloads()
    mixd = wl["binary"]["mixture"]
    mix = oracle_mixture(mixd)
    feeds = [(60, 64), (128, 80), (200, 96)]
    b = fm.fmlbm_batch_create(2, "fp32", 4)
    fm.fmlbm_batch_set_criterion(b, "phase")
    states = []
    for k, n in feeds:
        st, rho = _sweep_lattice(k, n)
        states.append(st)
        fm.fmlbm_batch_add(b, fm.mixture_from_dict(mixd), fm.make_lattice(n, n, 1.0), rho)
    steps, measure, status = fm.fmlbm_batch_run(b, 4, max_steps=300000, check_every=CHECK, tol=TOL)
    for j, st in enumerate(states):
        assert status[j] == 0 and steps[j] < 300000 and measure[j] < TOL, (j, steps[j], measure[j], status[j])
        liq, vap = fm.fmlbm_batch_phases(b, j, 2)
        f = flash(mix, float(pressure(mix, vap)), st["z"])
        dens = max(np.max(np.abs(liq / f["rtL"] - 1)), np.max(np.abs(vap / f["rtV"] - 1)))
        comp = max(np.max(np.abs(liq / liq.sum() - f["x"]) / f["x"]),
                   np.max(np.abs(vap / vap.sum() - f["y"]) / f["y"]))
        print(f"feed z1={st['z'][0]:.3f}: retired at {steps[j]} steps, density {dens:.2e}, composition {comp:.2e}")
        assert dens < 2e-2 and comp < 2e-2
    fm.fmlbm_batch_destroy(b)


def test_served_requests_retire_at_the_phase_criterion(fm):
    import time
    wl = workloads()
    mixd = wl["binary"]["mixture"]
    s = fm.fmlbm_server_create(2, "fp32", 8, CHECK, TOL, 300000, 1 << 30, criterion="phase")
    ids = []
    for k, n in [(90, 64), (170, 72)]:
        _, rho = _sweep_lattice(k, n)
        ids.append(fm.fmlbm_server_submit(s, fm.mixture_from_dict(mixd), fm.make_lattice(n, n, 1.0), rho, tag=k))
    res, t0 = [], time.time()
    while len(res) < len(ids) and time.time() - t0 < 120:
        res += fm.fmlbm_server_poll(s)
        time.sleep(0.01)
    fm.fmlbm_server_destroy(s)
    assert len(res) == len(ids)
    for r in res:
        assert r["status"] == 0 and r["residual"] < TOL and r["steps"] % CHECK == 0, r
