"""Writes tests/golden/workloads.json: the mixtures of the synthetic vapour-liquid
workloads and their flash states, computed by the FP64 oracle (oracle/ only).

Lattice units follow Section V of the paper: R = 1 and the most volatile component
has a = 2/49, b = 2/21 (so Tc1, Pc1 follow from the PR constants of Appendix C);
the other components are given by ratios of Tc, Pc to it.

Every flat-slab workload is initialised from the two-phase state at the pressure
where the feed z splits into a vapour volume fraction S_V = 0.5 (Section V.B).

Run:  python tests/golden/make_workloads.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.eos import Mixture, OMEGA  # noqa: E402
from oracle.flash import slab_state  # noqa: E402

OA, OB = OMEGA["pr"]
TC1 = (2.0 / 49.0) / (2.0 / 21.0) * OB / OA
PC1 = OB * TC1 / (2.0 / 21.0)


def mixture_dict(Tr, tc_ratio, pc_ratio, omega, kappa, kij):
    n = len(tc_ratio)
    return dict(eos="pr", R=1.0, T=Tr * TC1, Tc=[r * TC1 for r in tc_ratio], Pc=[r * PC1 for r in pc_ratio],
                omega=list(omega), M=[1.0] * n, kappa=list(kappa),
                kij=(np.full((n, n), kij) - kij * np.eye(n)).ravel().tolist())


def to_mix(d):
    return Mixture(d["eos"], d["R"], d["T"], Tc=d["Tc"], Pc=d["Pc"], omega=d["omega"], M=d["M"],
                   kappa=d["kappa"], kij=np.array(d["kij"]).reshape(len(d["Tc"]), -1))


def state(d, z):
    s = slab_state(to_mix(d), z, S_V=0.5)
    return dict(z=list(map(float, z)), p=float(s["p"]), rt_liquid=s["rtL"].tolist(),
                rt_vapour=s["rtV"].tolist(), x=s["x"].tolist(), y=s["y"].tolist(), beta=float(s["beta"]),
                S_V=float(s["S_V"]))


def main():
    binary = mixture_dict(0.8, [1.0, 1.3], [1.0, 0.9], [0.011, 0.2], [0.05, 0.075], 0.0)
    ternary = mixture_dict(0.85, [1.0, 1.3, 1.6], [1.0, 0.85, 0.7], [0.011, 0.1, 0.25], [0.05, 0.10, 0.15], 0.02)
    out = dict(
        lattice_units=dict(R=1.0, a1=2.0 / 49.0, b1=2.0 / 21.0, Tc1=TC1, Pc1=PC1),
        binary=dict(mixture=binary, slab=state(binary, [0.5, 0.5])),
        ternary=dict(mixture=ternary, slab=state(ternary, [0.4, 0.3, 0.3])),
    )
    sweep = []
    for k in range(256):
        z1 = 0.05 + 0.9 * k / 255.0
        try:
            sweep.append(state(binary, [z1, 1.0 - z1]))
        except ArithmeticError as e:  # recorded, not hidden
            sweep.append(dict(z=[z1, 1.0 - z1], error=str(e)))
    out["binary_sweep"] = sweep
    # request templates for the serving workload: random temperature and feed per template
    # (seeded), flash state at S_V = 0.5
    rng = np.random.default_rng(5)
    serve = []
    for k in range(48):
        if k % 2 == 0:
            Tr = float(rng.uniform(0.80, 0.92))
            z1 = float(rng.uniform(0.35, 0.65))
            d = mixture_dict(Tr, [1.0, 1.3], [1.0, 0.9], [0.011, 0.2], [0.05, 0.075], 0.0)
            z = [z1, 1.0 - z1]
        else:
            Tr = float(rng.uniform(0.85, 0.92))
            w = rng.dirichlet([8.0, 6.0, 6.0])
            d = mixture_dict(Tr, [1.0, 1.3, 1.6], [1.0, 0.85, 0.7], [0.011, 0.1, 0.25], [0.05, 0.10, 0.15], 0.02)
            z = [float(v) for v in w]
        try:
            serve.append(dict(Tr=Tr, mixture=d, slab=state(d, z)))
        except ArithmeticError as e:
            serve.append(dict(Tr=Tr, mixture=d, z=z, error=str(e)))
    out["serve_templates"] = serve
    with open(os.path.join(HERE, "workloads.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
