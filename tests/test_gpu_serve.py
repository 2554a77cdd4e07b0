"""Serving: continuous batching of vapour-liquid solves (admission, retirement, budget,
results independent of the mix)."""
import time

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


def _wait(fm, s, n, timeout=120.0):
    got, t0 = [], time.time()
    while len(got) < n and time.time() - t0 < timeout:
        got += fm.fmlbm_server_poll(s)
        time.sleep(0.005)
    return got


def _req(fm, nx, ny, seed, k=120):
    from paper_2212_10680_gb300 import inputs
    wl = workloads()
    st = wl["binary_sweep"][k]
    rho = inputs.with_noise(inputs.slab(st["rt_vapour"], st["rt_liquid"], nx, ny, 0.5, 4.0), 0.01, seed)
    return fm.mixture_from_dict(wl["binary"]["mixture"]), fm.make_lattice(nx, ny, 1.0, "isotropic", "fp32"), rho


def test_result_is_the_same_alone_and_in_the_mix(fm):
    mix, lat, rho = _req(fm, 96, 64, seed=1)
    alone = np.empty_like(rho)
    s = fm.fmlbm_server_create(2, "fp32", 8, 100, 1e-30, 600, 1 << 34)
    fm.fmlbm_server_submit(s, mix, lat, rho, alone, tag=1)
    r = _wait(fm, s, 1)
    assert len(r) == 1 and r[0]["steps"] == 600 and r[0]["status"] == fm.E_NOT_CONVERGED
    fm.fmlbm_server_destroy(s)
    # the same request among others of other sizes, submitted before and after it
    s = fm.fmlbm_server_create(2, "fp32", 8, 100, 1e-30, 600, 1 << 34)
    mixed = np.empty_like(rho)
    for k, (nx, ny) in enumerate([(64, 64), (128, 40)]):
        m2, l2, r2 = _req(fm, nx, ny, seed=10 + k, k=100 + 20 * k)
        fm.fmlbm_server_submit(s, m2, l2, r2, tag=10 + k)
    time.sleep(0.05)
    fm.fmlbm_server_submit(s, mix, lat, rho, mixed, tag=1)
    m3, l3, r3 = _req(fm, 200, 48, seed=3, k=140)
    fm.fmlbm_server_submit(s, m3, l3, r3, tag=3)
    res = _wait(fm, s, 4)
    fm.fmlbm_server_destroy(s)
    assert len(res) == 4
    mine = [r for r in res if r["tag"] == 1][0]
    assert mine["steps"] == 600
    assert np.array_equal(alone, mixed)
    # the phases of the result are the returned field's densest and least dense 2 x 2 blocks
    # (M = 1: molar = mass densities)
    liq, vap = block_phases(mixed, np.ones(2))
    assert mine["rho_liquid"] == [float(v) for v in liq]
    assert mine["rho_vapour"] == [float(v) for v in vap]
    assert mine["rho_liquid"][0] + mine["rho_liquid"][1] > 5 * (mine["rho_vapour"][0] + mine["rho_vapour"][1])


def test_admission_respects_the_budget_and_orders_times(fm):
    mix, lat, rho = _req(fm, 128, 128, seed=4)
    per = fm.fmlbm_lattice_bytes(2, lat)
    # room for one lattice at a time: the second is admitted only after the first retires
    s = fm.fmlbm_server_create(2, "fp32", 8, 50, 1e-30, 200, per + per // 2)
    for t in range(3):
        fm.fmlbm_server_submit(s, mix, lat, rho, tag=t)
    res = sorted(_wait(fm, s, 3), key=lambda r: r["tag"])
    fm.fmlbm_server_destroy(s)
    assert [r["tag"] for r in res] == [0, 1, 2]
    for r in res:
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"] and r["steps"] == 200
    assert res[1]["t_admit"] >= res[0]["t_done"] - 1e-3
    assert res[2]["t_admit"] >= res[1]["t_done"] - 1e-3


def test_converged_and_failed_requests_retire_independently(fm):
    s = fm.fmlbm_server_create(2, "fp64", 8, 100, 1e-12, 5000, 1 << 34)
    mixd = mixture_dict(n=2, Tr=1.1, kappa_scale=0.5)
    good = np.stack([np.full((32, 32), 1.0), np.full((32, 32), 0.8)])   # stationary: converges at 2nd check
    bad = good.copy()
    bad[1, 3, 3] = -1.0
    L = fm.make_lattice(32, 32, 1.0, precision="fp64")
    fm.fmlbm_server_submit(s, fm.mixture_from_dict(mixd), L, good, tag=1)
    fm.fmlbm_server_submit(s, fm.mixture_from_dict(mixd), L, bad, tag=2)
    res = {r["tag"]: r for r in _wait(fm, s, 2)}
    fm.fmlbm_server_destroy(s)
    assert res[1]["status"] == 0 and res[1]["steps"] == 200 and res[1]["residual"] == 0.0
    assert res[2]["status"] == fm.E_NONPHYSICAL


def test_submit_rejects_mismatches_and_a_full_queue(fm):
    mix, lat, rho = _req(fm, 64, 64, seed=5)
    s = fm.fmlbm_server_create(2, "fp32", 1, 100, 1e-30, 100000, 1 << 34, queue_capacity=2)
    with pytest.raises(fm.FmlbmError):
        fm.fmlbm_server_submit(s, mix, fm.make_lattice(64, 64, 1.0, precision="fp64"), rho)
    statuses = []
    for k in range(6):
        try:
            fm.fmlbm_server_submit(s, mix, lat, rho, tag=k)
            statuses.append(0)
        except fm.FmlbmError as e:
            statuses.append(e.status)
    assert fm.E_BUSY in statuses
    fm.fmlbm_server_destroy(s)   # drops the queued and running requests
