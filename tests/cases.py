"""Shared test cases: mixtures and initial states used by both the oracle and the
CUDA path (test-side helpers only; the two implementations share nothing else)."""
import json
import os

import numpy as np

from oracle import lbm
from oracle.eos import Mixture, OMEGA
from paper_2212_10680_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
WORKLOADS = os.path.join(HERE, "golden", "workloads.json")
PAPER_CASES = os.path.join(HERE, "golden", "paper_cases.json")
R_BAR = 83.14462618  # bar cm^3 / (mol K)

OA, OB = OMEGA["pr"]
TC1 = (2.0 / 49.0) / (2.0 / 21.0) * OB / OA
PC1 = OB * TC1 / (2.0 / 21.0)


def workloads() -> dict:
    with open(WORKLOADS) as f:
        return json.load(f)


def mixture_dict(n=2, eos="pr", Tr=0.8, kappa_scale=1.0, M=None, kij=0.0):
    tc = [1.0, 1.5, 1.3, 1.2][:n]
    pc = [1.0, 0.9, 0.85, 0.95][:n]
    om = [0.011, 0.2, 0.1, 0.15][:n]
    ka = [0.10, 0.15, 0.12, 0.08][:n]
    return dict(eos=eos, R=1.0, T=Tr * TC1, Tc=[r * TC1 for r in tc], Pc=[r * PC1 for r in pc], omega=om,
                M=list(M) if M is not None else [1.0] * n, kappa=[k * kappa_scale for k in ka],
                kij=(np.full((n, n), kij) - kij * np.eye(n)).ravel().tolist())


def oracle_mixture(d: dict) -> Mixture:
    n = len(d["Tc"])
    return Mixture(d["eos"], d["R"], d["T"], Tc=d["Tc"], Pc=d["Pc"], omega=d["omega"], M=d["M"],
                   kappa=d["kappa"], kij=np.asarray(d["kij"]).reshape(n, n))


def smooth_state(n, nx, ny, seed=3, base=(1.0, 1.2, 0.8, 0.6), amp=0.25):
    """A smooth single-phase-ish density field with 1% seeded noise."""
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    rho = np.stack([base[i] * (1 + amp * np.sin(2 * np.pi * (x / nx + (i + 1) * y / max(ny, 1)) + i))
                    for i in range(n)])
    return inputs.with_noise(rho, 0.01, seed)


def slab_state_binary(nx, ny, seed=1, W=4.0):
    wl = workloads()["binary"]
    rho = inputs.slab(wl["slab"]["rt_vapour"], wl["slab"]["rt_liquid"], nx, ny, 0.5, W)
    return wl["mixture"], inputs.with_noise(rho, 0.01, seed)


def run_oracle(mixd, rho, tau, stencil, velocity_force, steps, record=(), formulation="well_balanced"):
    mix = oracle_mixture(mixd)
    lat = lbm.Lattice(tau=tau, stencil=stencil, velocity_force=velocity_force, formulation=formulation)
    g, F = lbm.init_at_rest(rho, formulation=formulation)
    out = {}
    for k in range(1, steps + 1):
        g, F = lbm.step(g, mix, lat, F)
        if k in record:
            m = lbm.moments(g, F, mix, lat)
            out[k] = dict(g=g.copy(), F=F.copy(), rho=m["rho"], u=np.stack([m["ux"], m["uy"]]), lnf=m["lnf"])
    return out


def block_phases(r, M):
    """Block-mean phases of fmlbm_batch_phases, on the host: blocks of nodes 2bx, 2bx + 1 by
    2by, 2by + 1 (periodic at an odd edge), summed node by node, component by component."""
    n, ny, nx = r.shape
    rt = [r[i] / M[i] for i in range(n)]
    xs0 = 2 * np.arange((nx + 1) // 2)
    ys0 = 2 * np.arange((ny + 1) // 2)
    xs1 = np.where(xs0 + 1 < nx, xs0 + 1, 0)
    ys1 = np.where(ys0 + 1 < ny, ys0 + 1, 0)
    corners = [(ys0, xs0), (ys0, xs1), (ys1, xs0), (ys1, xs1)]
    tot = np.zeros((ys0.size, xs0.size))
    for ys, xs in corners:
        for i in range(n):
            tot = tot + rt[i][np.ix_(ys, xs)]
    out = []
    for k in (int(np.argmax(tot)), int(np.argmin(tot))):
        by, bx = divmod(k, xs0.size)
        v = np.zeros(n)
        for ys, xs in corners:
            v = v + np.array([rt[i][ys[by], xs[bx]] for i in range(n)])
        out.append(0.25 * v)
    return out


def slab_phases(r, M, pair=True):
    """Molar densities at the middle of the liquid run and of the vapour run of a 1-D
    periodic profile (the slab may sit anywhere: a flat slab can translate), as means over
    two neighbouring nodes (pair=True) or at single nodes.  The force of Eqs. eqforcefinal and
    eq1stder differences each field over two nodes, so a node-to-node alternation left by the
    transient feels no force and stays in the bulk phases; the pair mean is the phase."""
    tot = r[:, 0, :].sum(axis=0)
    nx = tot.size
    liquid = tot > 0.5 * (tot.max() + tot.min())
    start = int(np.argmin(tot))           # a vapour node: the liquid run is contiguous after it
    idx = np.nonzero(np.roll(liquid, -start))[0]
    iL = (start + (idx[0] + idx[-1]) // 2) % nx
    iV = (iL + nx // 2) % nx
    if not pair:
        return r[:, 0, iL] / M, r[:, 0, iV] / M
    return (0.5 * (r[:, 0, iL] + r[:, 0, (iL + 1) % nx]) / M,
            0.5 * (r[:, 0, iV] + r[:, 0, (iV + 1) % nx]) / M)


def normwise(a, b):
    """max |a - b| / max |b| (0 if both vanish)."""
    den = np.max(np.abs(b))
    num = np.max(np.abs(a - b))
    return num / den if den > 0 else num


def paper_cases() -> dict:
    with open(PAPER_CASES) as f:
        return json.load(f)


def paper_mixture(names, T_K, eos="pr", kappa=None, physical=False):
    """A mixture of the components of Table tabCompProp at T_K.

    physical=True: bar, K, cm^3/mol (R = 83.14462618).  Otherwise the lattice units of
    Section V: R = 1 and, for the most volatile component (the first listed), a = 2/49,
    b = 2/21, M = 1; since a = Omega_a R^2 Tc^2 / Pc and b = Omega_b R Tc / Pc this fixes
    that component's Tc and Pc, and every temperature and pressure scales by the same
    factors (reduced temperatures and pressures, and so alpha(T) and every phase
    equilibrium, are unchanged); molar masses scale by the first one's.
    Returns (mixture dict, scale) with scale = dict(T=..., p=...) lattice per physical."""
    comp = paper_cases()["components"]
    c = [comp[n] for n in names]
    n = len(names)
    kappa = [0.0] * n if kappa is None else list(kappa)
    if physical:
        d = dict(eos=eos, R=R_BAR, T=T_K, Tc=[q["Tc_K"] for q in c], Pc=[q["Pc_bar"] for q in c],
                 omega=[q["omega"] for q in c], M=[q["M"] for q in c], kappa=kappa, kij=[0.0] * (n * n))
        return d, dict(T=1.0, p=1.0)
    oa, ob = OMEGA[eos]
    a1, b1 = 2.0 / 49.0, 2.0 / 21.0
    tc1 = (a1 / b1) * ob / oa
    pc1 = ob * tc1 / b1
    sT, sp = tc1 / c[0]["Tc_K"], pc1 / c[0]["Pc_bar"]
    d = dict(eos=eos, R=1.0, T=T_K * sT, Tc=[q["Tc_K"] * sT for q in c], Pc=[q["Pc_bar"] * sp for q in c],
             omega=[q["omega"] for q in c], M=[q["M"] / c[0]["M"] for q in c], kappa=kappa, kij=[0.0] * (n * n))
    return d, dict(T=sT, p=sp)
