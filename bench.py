"""Throughput benchmark of the fused lattice update (component-GLUPS).

Default workload: the binary PR vapour-liquid system in lattice units, a circular
liquid droplet of radius 200 in vapour on a periodic 1024 x 1024 D2Q9 lattice, FP32
storage and arithmetic, isotropic stencils, lagged velocity force, tau = 1.0, seeded
1% noise.  One "step" is one time step of the whole method (one fused kernel
launch).  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own independent lattice (weak scaling, no
data-path collective; a barrier and a max-reduction of the timings only).
``--impl reference`` times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALGO_BYTES = {"fp64": 144.0, "fp32": 72.0, "fp16dev": 40.0, "bf16dev": 40.0}  # per component-node update
L2_FLUSH_BYTES = 256 << 20
KERNEL_SOURCES = ["paper_2212_10680_gb300/csrc/fmlbm_kernels.cuh", "paper_2212_10680_gb300/csrc/fmlbm_launch.cuh",
                  "paper_2212_10680_gb300/csrc/fmlbm_tma.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured")
    return dict(hbm_gbs=6800.0, source="fallback")


def profile_traffic(kernel: str, workload_key: str, precision: str):
    """DRAM bytes per launch of the step kernel from the committed ncu summary
    profiles/<kernel>_<workload>_<precision>.md, if it was taken on the current kernel
    source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload_key}_{precision}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch_%s:\s*([0-9.eE+]+)" % precision, text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_hash():
        return None
    return float(m_bytes.group(1))


def workload(name: str):
    wl = json.load(open(os.path.join(ROOT, "tests", "golden", "workloads.json")))
    from paper_2212_10680_gb300 import inputs
    if name == "droplet1024":
        b = wl["binary"]
        n = 1024
        rho = inputs.with_noise(inputs.droplet(b["slab"]["rt_vapour"], b["slab"]["rt_liquid"], n, n, 200.0, 4.0),
                                0.01, 2)
        return dict(name="binary PR droplet R=200, 1024x1024 periodic D2Q9", mixture=b["mixture"], rho=rho,
                    nx=n, ny=n, tau=1.0, stencil="isotropic", precision="fp32")
    if name == "ternary4096":
        t = wl["ternary"]
        n = 4096
        rho = inputs.with_noise(inputs.slab(t["slab"]["rt_vapour"], t["slab"]["rt_liquid"], n, n, 0.5, 4.0), 0.01, 3)
        return dict(name="ternary PR flat slab, 4096x4096 periodic D2Q9", mixture=t["mixture"], rho=rho,
                    nx=n, ny=n, tau=1.0, stencil="isotropic", precision="fp32")
    raise SystemExit(f"unknown workload {name}")


def sample_field(w: dict, s: int) -> np.ndarray:
    """A scaled-down s x s lattice of the workload's initial-field recipe."""
    from paper_2212_10680_gb300 import inputs
    wl = json.load(open(os.path.join(ROOT, "tests", "golden", "workloads.json")))
    if w["nx"] == 1024:
        b = wl["binary"]["slab"]
        return inputs.with_noise(inputs.droplet(b["rt_vapour"], b["rt_liquid"], s, s, 50.0, 4.0), 0.01, 2)
    t = wl["ternary"]["slab"]
    return inputs.with_noise(inputs.slab(t["rt_vapour"], t["rt_liquid"], s, s, 0.5, 4.0), 0.01, 3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self) -> dict:
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["unsampled"], samples=0)
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))


def cpu_oracle_rate(w: dict, max_seconds: float = 15.0):
    """The FP64 oracle as it stands, on the host, on full-lattice steps of the same workload
    (a bounded sample: as many steps as fit in about max_seconds, at least one)."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import lbm
    from oracle.eos import Mixture
    d = w["mixture"]
    n = len(d["Tc"])
    mix = Mixture(d["eos"], d["R"], d["T"], Tc=d["Tc"], Pc=d["Pc"], omega=d["omega"], M=d["M"], kappa=d["kappa"],
                  kij=np.asarray(d["kij"]).reshape(n, n))
    lat = lbm.Lattice(tau=w["tau"], stencil=w["stencil"], velocity_force="lagged")
    full = w["nx"] * w["ny"] <= 1024 * 1024
    rho = w["rho"] if full else sample_field(w, 256)
    ny_s, nx_s = rho.shape[1:]
    g, F = lbm.init_at_rest(rho)
    steps, t0 = 0, time.perf_counter()
    while True:
        g, F = lbm.step(g, mix, lat, F)
        steps += 1
        el = time.perf_counter() - t0
        if el >= max_seconds or steps >= 50:
            break
    units = n * nx_s * ny_s * steps
    what = (f"{steps} full-lattice FP64 oracle steps of the {nx_s}x{ny_s} workload" if full else
            f"{steps} FP64 oracle steps of a {nx_s}x{ny_s} lattice of the same mixture and initial-field recipe")
    return dict(value=units / el / 1e9, unit="component-GLUPS", cores=1, kind="oracle",
                sample=f"{what} ({el:.1f} s, numpy, one thread)")


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import lbm
    from oracle.eos import Mixture
    d = w["mixture"]
    n = len(d["Tc"])
    mix = Mixture(d["eos"], d["R"], d["T"], Tc=d["Tc"], Pc=d["Pc"], omega=d["omega"], M=d["M"], kappa=d["kappa"],
                  kij=np.asarray(d["kij"]).reshape(n, n))
    lat = lbm.Lattice(tau=w["tau"], stencil=w["stencil"], velocity_force="lagged")
    # bounded sample: each step advances a 256 x 256 lattice of the same mixture and
    # initial-field recipe (droplet radius scaled to 50), so K steps take seconds
    s = 256
    rho = sample_field(w, s)
    g, F = lbm.init_at_rest(rho)
    for _ in range(args.warmup):
        g, F = lbm.step(g, mix, lat, F)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g, F = lbm.step(g, mix, lat, F)
    el = time.perf_counter() - t0
    value = n * s * s * args.steps / el / 1e9
    line = dict(impl="reference", metric="component-GLUPS", value=value, unit="component-GLUPS", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * el / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=w["name"], nx=w["nx"], ny=w["ny"], n_components=n, tau=w["tau"],
                            stencil=w["stencil"], precision="fp64 (oracle)"),
                cpu_baseline=dict(value=value, unit="component-GLUPS", cores=1, kind="oracle",
                                  sample=f"{args.steps} FP64 oracle steps of a {s}x{s} lattice of the workload "
                                         f"after {args.warmup} warm-up steps (numpy, one thread)"),
                e2e=dict(value=value, unit="component-GLUPS", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def run_ours(args, w, rank, world, dist):
    import torch
    from paper_2212_10680_gb300 import fmlbm

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    prec = args.precision or w["precision"]
    n = len(w["mixture"]["Tc"])
    nx, ny = w["nx"], w["ny"]
    nodes = nx * ny
    lat = fmlbm.Lattice(fmlbm.mixture_from_dict(w["mixture"]), nx, ny, w["tau"], w["stencil"], prec, "lagged",
                        stream=stream.cuda_stream)
    if args.tile_y:
        fmlbm.fmlbm_set_tile_height(lat.h, args.tile_y)
    if args.variant:
        fmlbm.fmlbm_set_step_variant(lat.h, args.variant)
    variant = fmlbm.fmlbm_get_step_variant(lat.h)
    rho_dev = torch.from_numpy(w["rho"]).to(dev)
    fmlbm.fmlbm_init_device(lat.h, rho_dev.data_ptr())
    lat.step(args.warmup)
    lat.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            flush.zero_()                       # evict the previous step's data from L2 (untimed)
            ev[k][0].record(stream)
            fmlbm.fmlbm_step(lat.h, 1)
            ev[k][1].record(stream)
        barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    lat.synchronize()
    total_s = sum(ms) / 1e3
    if dist is not None:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    units = n * nodes * args.steps * world
    value = units / total_s / 1e9
    per_launch_s = total_s / args.steps
    algo = ALGO_BYTES[prec] * n * nodes
    peak = measured_peaks()
    achieved = algo / per_launch_s / 1e9
    kernel_name = "fused_step_tma" if variant == "tma" else "fused_step"
    traffic = profile_traffic(kernel_name, args.workload, prec)

    # end to end through the public API with host buffers: H2D of the initial field from
    # pinned memory, then per step one fused update and a D2H read of the step's
    # diagnostics (component masses, residual)
    rho_pinned = torch.from_numpy(w["rho"]).pin_memory()
    rho_np = rho_pinned.numpy()
    e2e_steps = args.steps
    barrier()
    t0 = time.perf_counter()
    fmlbm.fmlbm_init(lat.h, rho_np)
    for _ in range(e2e_steps):
        fmlbm.fmlbm_step(lat.h, 1)
        fmlbm.fmlbm_diagnostics(lat.h, n)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = n * nodes * e2e_steps * world / e2e_s / 1e9
    lat.close()

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(w, args.cpu_seconds)
    line = dict(
        metric="component-GLUPS", value=value, unit="component-GLUPS", n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=1e3 * total_s / args.steps, higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="f64" if prec == "fp64" else "f32",
        data="synthetic (seeded droplet/slab initial fields from oracle flash densities)",
        config=dict(workload=w["name"], nx=nx, ny=ny, n_components=n, tau=w["tau"], stencil=w["stencil"],
                    precision=prec, velocity_force="lagged", step_kernel=variant,
                    l2="flushed between timed steps (256 MB write)",
                    timing="CUDA events around each fused launch on the launching stream"),
        roofline=dict(bound="hbm", achieved=achieved, peak=peak["hbm_gbs"], unit="GB/s",
                      frac=achieved / peak["hbm_gbs"], traffic=traffic, peak_source=peak["source"],
                      algorithmic_bytes_per_component_node=ALGO_BYTES[prec],
                      kernel=kernel_name),
        cpu_baseline=cpu,
        e2e=dict(value=e2e_value, unit="component-GLUPS",
                 h2d_bytes_per_step=n * nodes * 8 / e2e_steps, d2h_bytes_per_step=(n + 2) * 8 + 16),
        gpu_launches=args.steps,
        clocks=clk.summary(),
    )
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="droplet1024")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--tile-y", type=int, default=0, help="override the fused step's tile height (8 or 16)")
    ap.add_argument("--variant", default=None, choices=["auto", "plain", "tma"], help="step kernel variant")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        w = workload(args.workload)
        run_reference(args, w, rank, world)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        td.init_process_group("nccl")
        dist = td
    w = workload(args.workload)
    run_ours(args, w, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
