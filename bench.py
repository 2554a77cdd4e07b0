"""Throughput benchmark of the fused lattice update (component-GLUPS).

Default workload: the binary PR vapour-liquid system in lattice units, a circular
liquid droplet of radius 200 in vapour on a periodic 1024 x 1024 D2Q9 lattice, FP32
storage and arithmetic, isotropic stencils, lagged velocity force, tau = 1.0, seeded
1% noise.  One "step" is one time step of the whole method (one fused kernel
launch).  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own independent lattice (weak scaling, no
data-path collective; a barrier and a max-reduction of the timings only); the batched
sweep splits its lattices and the serving run its requests between the ranks.
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

# per component-node update: one read and one write of the nine distributions
ALGO_BYTES = {"fp64": 144.0, "fp32": 72.0, "fp16dev": 40.0, "bf16dev": 40.0, "fp16dev_lnf64": 40.0,
              "bf16dev_lnf64": 40.0}
L2_FLUSH_BYTES = 256 << 20
KERNEL_SOURCES = ["paper_2212_10680_gb300/csrc/fmlbm_lanes.cuh", "paper_2212_10680_gb300/csrc/fmlbm_kernels.cuh",
                  "paper_2212_10680_gb300/csrc/fmlbm_pair.cuh", "paper_2212_10680_gb300/csrc/fmlbm_launch.cuh",
                  "paper_2212_10680_gb300/csrc/fmlbm_tma.cuh", "paper_2212_10680_gb300/csrc/fmlbm_multi.cuh"]


# ---- ranks (torchrun): independent problems are split, timings reduced; no data exchange ----

def shard(n_items: int, rank: int, world: int) -> range:
    """This rank's contiguous share of n_items independent problems (shares differ by at
    most one; together they cover every item once)."""
    return range(n_items * rank // world, n_items * (rank + 1) // world)


def round_robin(n_items: int, rank: int, world: int) -> list:
    """Items rank, rank + world, ...: an arrival stream thinned per rank (each share of a
    Poisson stream is again Poisson, at rate / world)."""
    return list(range(rank, n_items, world))


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over the ranks (every rank gets it); x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device) -> float:
    """The sum of x over the ranks (every rank gets it)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_lists(xs: list, dist) -> list:
    """Every rank's list, concatenated in rank order (every rank gets it)."""
    if dist is None:
        return list(xs)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, list(xs))
    return [x for p in parts for x in p]


def _code_only(src: str) -> str:
    """C++ source without comments and blank lines: editing a comment keeps the hash."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_hash() -> str:
    """Identifies the step kernel's code (comments excluded) that a committed profile
    describes; a profile with another hash gives no traffic figure."""
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p)) as f:
            h.update(_code_only(f.read()).encode())
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


def workload(name: str, size: int = 0):
    """A bench workload; size > 0 scales its lattice to size x size (profiling captures)."""
    wl = json.load(open(os.path.join(ROOT, "tests", "golden", "workloads.json")))
    from paper_2212_10680_gb300 import inputs
    if name == "droplet1024":
        b = wl["binary"]
        n = size or 1024
        radius = 200.0 * n / 1024
        rho = inputs.with_noise(inputs.droplet(b["slab"]["rt_vapour"], b["slab"]["rt_liquid"], n, n, radius, 4.0),
                                0.01, 2)
        return dict(name=f"binary PR droplet R={radius:g}, {n}x{n} periodic D2Q9", mixture=b["mixture"], rho=rho,
                    nx=n, ny=n, tau=1.0, stencil="isotropic", precision="fp32")
    if name == "ternary4096":
        t = wl["ternary"]
        n = size or 4096
        rho = inputs.with_noise(inputs.slab(t["slab"]["rt_vapour"], t["slab"]["rt_liquid"], n, n, 0.5, 4.0), 0.01, 3)
        return dict(name=f"ternary PR flat slab, {n}x{n} periodic D2Q9", mixture=t["mixture"], rho=rho,
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

    def wait_running(self, timeout: float = 10.0):
        """Return once the sampler has printed its first sample: nvidia-smi's start-up then no
        longer overlaps the timed work that follows, while the sampling still covers it."""
        self.wait_samples(1, timeout)

    def wait_samples(self, n: int, timeout: float = 2.0):
        """Wait until at least n samples have arrived (a sample after the timed work brackets it)."""
        t0 = time.perf_counter()
        while self.proc and len(self.lines) < n and time.perf_counter() - t0 < timeout:
            time.sleep(0.005)

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


def _device_steps(fmlbm, torch, w, prec, steps, warmup, stream, dev, variant=None, autotune=True, flush=None,
                  dist=None, tile_y=0):
    """K single-step launches of one lattice of workload w timed with CUDA events on the
    launching stream (L2 flushed between them, untimed), after the warm-up (and the
    autotuner's trial steps, which are real steps).  Returns the per-step times and the
    kernel choice; the lattice is closed."""
    n = len(w["mixture"]["Tc"])
    lat = fmlbm.Lattice(fmlbm.mixture_from_dict(w["mixture"]), w["nx"], w["ny"], w["tau"], w["stencil"], prec,
                        "lagged", stream=stream.cuda_stream)
    if tile_y:
        fmlbm.fmlbm_set_tile_height(lat.h, tile_y)
    rho_dev = torch.from_numpy(w["rho"]).to(dev)
    fmlbm.fmlbm_init_device(lat.h, rho_dev.data_ptr())
    tuned = None
    if variant:
        fmlbm.fmlbm_set_step_variant(lat.h, variant)
    elif autotune:
        v, ty, ms = fmlbm.fmlbm_autotune(lat.h, 5)
        tuned = dict(variant=v, tile_y=ty, ms_per_step=ms)
    chosen = fmlbm.fmlbm_get_step_variant(lat.h)
    lat.synchronize()
    del rho_dev
    if flush is None:
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    with ClockSampler(dev.index) as clk:
        clk.wait_running()
        # the warm-up steps (untimed) right before the timed ones, each after the same L2 flush,
        # so that the first timed step does not follow an idle device
        for _ in range(warmup):
            flush.zero_()
            flush.sum()
            fmlbm.fmlbm_step(lat.h, 1)
        barrier()
        n_before = len(clk.lines)
        for k in range(steps):
            # evict the previous step's data from L2 (untimed): write a buffer twice the L2
            # size, then read it, so that the lines left in L2 are clean and none is the step's
            # (after a write alone the timed step would also pay the write-back of 129 MB of
            # the flush buffer's dirty lines, traffic that is not the step's)
            flush.zero_()
            flush.sum()
            ev[k][0].record(stream)
            fmlbm.fmlbm_step(lat.h, 1)
            ev[k][1].record(stream)
        barrier()
        clk.wait_samples(n_before + 1)
    ms = [a.elapsed_time(b) for a, b in ev]
    lat.synchronize()
    lat.close()
    return dict(ms=ms, variant=chosen, tuned=tuned, clocks=clk.summary(), n=n, nodes=w["nx"] * w["ny"])


def _e2e_rate(fmlbm, torch, w, prec, steps, stream, dev, dist=None):
    """The same metric end to end through the C ABI with host buffers: fmlbm_init from pinned
    host memory, then fmlbm_step_diagnostics for all the steps (each step computes the masses
    and residual of the state it reads, and each step's row, with the error latch, is copied to
    the host and read there, three steps behind); every step's result reaches the host inside
    the timed region."""
    n = len(w["mixture"]["Tc"])
    lat = fmlbm.Lattice(fmlbm.mixture_from_dict(w["mixture"]), w["nx"], w["ny"], w["tau"], w["stencil"], prec,
                        "lagged", stream=stream.cuda_stream)
    rho_np = torch.from_numpy(w["rho"]).pin_memory().numpy()
    # warm-up (untimed): the same calls once, so that the timed run starts on a busy device
    # with the library's first-call costs paid
    fmlbm.fmlbm_init(lat.h, rho_np)
    fmlbm.fmlbm_step_diagnostics(lat.h, 3, n)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fmlbm.fmlbm_init(lat.h, rho_np)
    fmlbm.fmlbm_step_diagnostics(lat.h, steps, n)
    torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - t0, dist, dev)
    lat.close()
    world = dist.get_world_size() if dist is not None else 1
    nodes = w["nx"] * w["ny"]
    return dict(value=n * nodes * steps * world / el / 1e9, unit="component-GLUPS", steps=steps,
                h2d_bytes_per_step=n * nodes * 8 / steps, d2h_bytes_per_step=64)


def _oracle_worker(args):
    """One process: the FP64 oracle as it stands on a sample lattice of a workload, for about
    `seconds`; returns component-node updates and elapsed seconds."""
    wname, size, seconds = args
    w = workload(wname)
    from oracle import lbm
    from oracle.eos import Mixture
    d = w["mixture"]
    n = len(d["Tc"])
    mix = Mixture(d["eos"], d["R"], d["T"], Tc=d["Tc"], Pc=d["Pc"], omega=d["omega"], M=d["M"], kappa=d["kappa"],
                  kij=np.asarray(d["kij"]).reshape(n, n))
    lat = lbm.Lattice(tau=w["tau"], stencil=w["stencil"], velocity_force="lagged")
    rho = sample_field(w, size)
    g, F = lbm.init_at_rest(rho)
    steps, t0 = 0, time.perf_counter()
    while True:
        g, F = lbm.step(g, mix, lat, F)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return n * size * size * steps, time.perf_counter() - t0, steps


def cpu_oracle_all_cores(wname: str, seconds: float = 8.0, size: int = 256):
    """The oracle on every host core: one independent sample lattice per core (a pool of
    spawned processes; the oracle itself is single-threaded numpy), aggregate rate."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores, initializer=_pool_init) as pool:
        res = pool.map(_oracle_worker, [(wname, size, seconds)] * cores)
    units = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return dict(value=units / el / 1e9, unit="component-GLUPS", cores=cores, kind="oracle",
                sample=f"{cores} processes, each {min(r[2] for r in res)}-{max(r[2] for r in res)} FP64 oracle steps "
                       f"of its own {size}x{size} lattice of the workload's mixture and initial-field recipe "
                       f"({el:.1f} s, numpy, one thread each)")


def _pool_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))


def small_binary_fp64(fmlbm, torch, stream, dev, gpu_steps=2000, oracle_steps=20):
    """The small parity configuration (64 x 64 binary slab, FP64, tau 1): GPU and oracle
    milliseconds per step on the same lattice (the GPU run is latency-bound: 4,096 nodes)."""
    from paper_2212_10680_gb300 import inputs
    wl = json.load(open(os.path.join(ROOT, "tests", "golden", "workloads.json")))["binary"]
    rho = inputs.with_noise(inputs.slab(wl["slab"]["rt_vapour"], wl["slab"]["rt_liquid"], 64, 64, 0.5, 4.0), 0.01, 1)
    lat = fmlbm.Lattice(fmlbm.mixture_from_dict(wl["mixture"]), 64, 64, 1.0, "isotropic", "fp64", "lagged",
                        stream=stream.cuda_stream)
    lat.init(rho)
    lat.step(10)
    lat.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(gpu_steps)
    e1.record(stream)
    lat.synchronize()
    gpu_ms = e0.elapsed_time(e1) / gpu_steps
    lat.close()
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import lbm
    from oracle.eos import Mixture
    d = wl["mixture"]
    mix = Mixture(d["eos"], d["R"], d["T"], Tc=d["Tc"], Pc=d["Pc"], omega=d["omega"], M=d["M"], kappa=d["kappa"],
                  kij=np.asarray(d["kij"]).reshape(2, 2))
    g, F = lbm.init_at_rest(rho)
    olat = lbm.Lattice(tau=1.0, stencil="isotropic", velocity_force="lagged")
    t0 = time.perf_counter()
    for _ in range(oracle_steps):
        g, F = lbm.step(g, mix, olat, F)
    oracle_ms = 1e3 * (time.perf_counter() - t0) / oracle_steps
    return dict(workload="binary PR flat slab 64x64, FP64, tau 1, isotropic, lagged", gpu_ms_per_step=gpu_ms,
                gpu_steps=gpu_steps, oracle_ms_per_step=oracle_ms, oracle_steps=oracle_steps,
                note="GPU: launch-bound (4,096 nodes per step); oracle: numpy, one thread")


def ternary_forms(fmlbm, torch, stream, dev, steps, warmup, flush):
    """The 4096 x 4096 ternary slab in every storage form: component-GLUPS and the fraction of
    the measured HBM bandwidth by each form's own algorithmic bytes."""
    w = workload("ternary4096")
    peak = measured_peaks()
    out = {}
    for prec in ("fp32", "fp16dev", "bf16dev", "bf16dev_lnf64"):
        k = max(3, steps // 2) if prec.endswith("lnf64") else steps
        r = _device_steps(fmlbm, torch, w, prec, k, warmup, stream, dev, variant="plain", flush=flush)
        per = sum(r["ms"]) / 1e3 / k
        achieved = ALGO_BYTES[prec] * r["n"] * r["nodes"] / per / 1e9
        out[prec] = dict(value=r["n"] * r["nodes"] / per / 1e9, unit="component-GLUPS", ms_per_step=1e3 * per,
                         steps=k, roofline=dict(bound="hbm", achieved=achieved, peak=peak["hbm_gbs"], unit="GB/s",
                                                frac=achieved / peak["hbm_gbs"],
                                                traffic=profile_traffic("fused_step", "ternary4096", prec),
                                                algorithmic_bytes_per_component_node=ALGO_BYTES[prec]),
                         clocks=r["clocks"])
    return dict(workload=w["name"] + ", tau 1, isotropic, lagged, plain step", forms=out)


def temporal_blocking(fmlbm, torch, stream, dev, flush, reps=10, k=20):
    """The binary droplet workload advanced K steps per fmlbm_step call, by single-step launches
    (plain) and by one multi-step launch (temporal blocking): ms per step of each, L2 flushed
    before every timed call.  The two give bit-identical states."""
    w = workload("droplet1024")
    out = {}
    for variant in ("plain", "multi"):
        lat = fmlbm.Lattice(fmlbm.mixture_from_dict(w["mixture"]), w["nx"], w["ny"], w["tau"], w["stencil"], "fp32",
                            "lagged", stream=stream.cuda_stream)
        rho_dev = torch.from_numpy(w["rho"]).to(dev)
        fmlbm.fmlbm_init_device(lat.h, rho_dev.data_ptr())
        fmlbm.fmlbm_set_step_variant(lat.h, variant)
        lat.step(2 * k)
        lat.synchronize()
        ms = []
        for _ in range(reps):
            flush.zero_()
            flush.sum()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fmlbm.fmlbm_step(lat.h, k)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1) / k)
        lat.synchronize()
        lat.close()
        per = sum(ms) / len(ms)
        out[variant] = dict(ms_per_step=per, value=2 * w["nx"] * w["ny"] / (per * 1e-3) / 1e9, unit="component-GLUPS")
    return dict(workload=w["name"] + f", FP32, {k} steps per call", steps_per_call=k, reps=reps, **out)


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
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    r = _device_steps(fmlbm, torch, w, prec, args.steps, args.warmup, stream, dev, variant=args.variant,
                      flush=flush, dist=dist, tile_y=args.tile_y)
    ms, variant, tuned = r["ms"], r["variant"], r["tuned"]
    total_s = max_over_ranks(sum(ms) / 1e3, dist, dev)
    units = n * nodes * args.steps * world
    value = units / total_s / 1e9
    per_launch_s = total_s / args.steps
    algo = ALGO_BYTES[prec] * n * nodes
    peak = measured_peaks()
    achieved = algo / per_launch_s / 1e9
    kernel_name = {"tma": "fused_step_tma", "tma_tile": "fused_step_tma", "pair": "fused_step_pair"}.get(variant,
                                                                                                     "fused_step")
    # the committed counters describe the workload at its own size only
    traffic = None if args.size else profile_traffic(kernel_name, args.workload, prec)
    e2e = _e2e_rate(fmlbm, torch, w, prec, args.steps, stream, dev, dist)
    e2e_long = _e2e_rate(fmlbm, torch, w, prec, max(args.steps, args.e2e_steps), stream, dev, dist)

    configs = None
    if world == 1 and not args.no_configs and args.workload == "droplet1024":
        configs = dict(small_binary_fp64=small_binary_fp64(fmlbm, torch, stream, dev),
                       ternary_4096=ternary_forms(fmlbm, torch, stream, dev, max(10, min(args.steps, 20)),
                                                  max(3, args.warmup), flush),
                       temporal_blocking=temporal_blocking(fmlbm, torch, stream, dev, flush))
        del flush
        torch.cuda.empty_cache()
        configs["batch_sweep"] = run_batch(args, rank, world, dist, summary=True)
        # two offered loads: about 0.7 of the batching servers' capacity (the plain FIFO loop,
        # about 1.9 requests/s on these requests, is overloaded there), and one below the FIFO
        # loop's capacity, where both keep up
        configs["serving"] = run_serve(args, rank, world, dist, summary=True)
        configs["serving_low_load"] = run_serve(_summary_args(args, summary_rate=args.summary_rate_low), rank,
                                                world, dist, summary=True)

    if rank != 0:
        return
    cpu = cpu_all = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(w, args.cpu_seconds)
        cpu_all = cpu_oracle_all_cores(args.workload, seconds=args.cpu_seconds / 2)
        cpu["all_cores"] = cpu_all
    line = dict(
        metric="component-GLUPS", value=value, unit="component-GLUPS", n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=1e3 * total_s / args.steps, higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="f64" if prec == "fp64" else "f32",
        data="synthetic (seeded droplet/slab initial fields from oracle flash densities)",
        config=dict(workload=w["name"], nx=nx, ny=ny, n_components=n, tau=w["tau"], stencil=w["stencil"],
                    precision=prec, velocity_force="lagged", step_kernel=variant, autotune=tuned,
                    l2="flushed between timed steps (256 MB write, then read: clean lines, none of the step's)",
                    e2e="fmlbm_init from pinned host memory, then fmlbm_step_diagnostics: every step's masses, "
                        "residual and error latch copied to the host",
                    timing="CUDA events around each fused launch on the launching stream",
                    step_ms_spread=dict(median=statistics.median(ms), min=min(ms), max=max(ms))),
        roofline=dict(bound="hbm", achieved=achieved, peak=peak["hbm_gbs"], unit="GB/s",
                      frac=achieved / peak["hbm_gbs"], traffic=traffic, peak_source=peak["source"],
                      algorithmic_bytes_per_component_node=ALGO_BYTES[prec],
                      kernel=kernel_name),
        cpu_baseline=cpu,
        e2e=dict(value=e2e["value"], unit=e2e["unit"], h2d_bytes_per_step=e2e["h2d_bytes_per_step"],
                 d2h_bytes_per_step=e2e["d2h_bytes_per_step"]),
        e2e_amortized=dict(e2e_long, note="the same loop over more steps: the one-time fmlbm_init (16.8 MB from "
                                          "pinned host memory) spread over them"),
        gpu_launches=args.steps,
        clocks=r["clocks"],
        configs=configs,
        host=dict(nproc=os.cpu_count()),
    )
    print(json.dumps(line), flush=True)


def _stats_pct(values, q):
    return float(np.percentile(np.asarray(values), q)) if len(values) else None


def _summary_args(args, **over):
    """A copy of the command-line arguments with the given fields replaced."""
    a = argparse.Namespace(**vars(args))
    for k, v in over.items():
        setattr(a, k, v)
    return a


def _phase_dev(liquid, vapour, st):
    """Largest relative deviation of a retired lattice's two phases (molar densities) from the
    flash state it started from (stored in tests/golden/workloads.json; the equilibrium of the
    lattice sits at a slightly shifted pressure, Section V.A, so this is a check of scale)."""
    dl = np.abs(np.asarray(liquid) / np.asarray(st["rt_liquid"]) - 1.0)
    dv = np.abs(np.asarray(vapour) / np.asarray(st["rt_vapour"]) - 1.0)
    return float(max(dl.max(), dv.max()))


# The first feed of the stored sweep (z1 = 0.05 + 0.9 k / 255) the batched sweep uses: the
# unperturbed slabs of the feeds below z1 = 0.11 leave the EOS domain within a few hundred
# steps on wide lattices (FP64 and FP32 alike), so the sweep spans z1 = 0.12 .. 0.95.
SWEEP_FIRST = 20


def run_batch(args, rank, world, dist=None, summary=False):
    """Batched P-x sweep: independent binary lattices (side 4 x U{16..max_side / 4}, feeds z1 swept
    0.12..0.95 at fixed T), one persistent multi-lattice step per time step, graph-captured
    chunks, per-lattice retirement; against the same lattices run one after another with
    single-lattice handles and the same retirement rule.  Each lattice starts as Section V.B
    starts an envelope point: the flat interface of Eq. eqInit (W = 4) between the flash phases
    at S_V = 0.5, unperturbed.  A lattice retires when its phase measure (the mean of ln rho_i
    over the nodes, per component) changes by less than tol over a check interval
    (FMLBM_CRITERION_PHASE); the density residual does not settle, because the slab keeps a
    rigid sloshing motion that nothing damps in a periodic box.  Under torchrun each rank takes
    a contiguous share of the lattices (the total is fixed: strong scaling)."""
    if summary:
        # a short sweep for the main benchmark line: 32 of the recipe's feeds on lattices of
        # side 64..192
        args = _summary_args(args, batch_lattices=32, batch_max_side=192, max_steps=args.max_steps,
                             check_every=500, tol=args.tol, precision=None)
    import torch
    from paper_2212_10680_gb300 import fmlbm, inputs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = json.load(open(os.path.join(ROOT, "tests", "golden", "workloads.json")))
    mixd = wl["binary"]["mixture"]
    n = len(mixd["Tc"])
    nlat = args.batch_lattices
    rng = np.random.default_rng(4)
    # sides are multiples of 4, so that the interface centres of Eq. eqInit (n_x / 4 and
    # 3 n_x / 4) sit on nodes, as in the paper's set-ups (n_x = 200, 400); with the centres
    # between nodes the transient of the low-z1 feeds leaves the EOS domain on wide lattices
    sides = 4 * rng.integers(16, args.batch_max_side // 4 + 1, nlat)
    mine = list(shard(nlat, rank, world))
    fields, states = {}, {}
    for k in mine:
        st = wl["binary_sweep"][SWEEP_FIRST + int(round(k * (255 - SWEEP_FIRST) / max(nlat - 1, 1)))]
        L = int(sides[k])
        states[k] = st
        fields[k] = inputs.slab(st["rt_vapour"], st["rt_liquid"], L, L, 0.5, 4.0)
    mix = fmlbm.mixture_from_dict(mixd)
    prec = args.precision or "fp32"

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ty = blocks = None
    units, status_mine, steps_mine, dev_mine, failed_mine = 0, [], [], [], []
    b = fmlbm.fmlbm_batch_create(n, prec, max(len(mine), 1))
    fmlbm.fmlbm_batch_set_criterion(b, args.criterion)
    for k in mine:
        L = int(sides[k])
        fmlbm.fmlbm_batch_add(b, mix, fmlbm.make_lattice(L, L, 1.0, "isotropic", prec), fields[k])
    if mine:
        ty, blocks, ms_tune = fmlbm.fmlbm_batch_autotune(b, 3)
        # the autotuner's trial steps are real steps; count them in the work
        tuned_steps = [fmlbm.fmlbm_batch_slot_info(b, j)[0] for j in range(len(mine))]
    barrier()
    t0 = time.perf_counter()
    if mine:
        steps, res, st = fmlbm.fmlbm_batch_run(b, len(mine), args.max_steps, args.check_every, args.tol)
        torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    if mine:
        units = sum(n * int(sides[k]) ** 2 * (int(steps[j]) - tuned_steps[j]) for j, k in enumerate(mine))
        status_mine = [int(v) for v in st]
        steps_mine = [int(v) for v in steps]
        failed_mine = [[k, round(states[k]["z"][0], 4), int(sides[k]), fmlbm.STATUS[status_mine[j]], steps_mine[j]]
                       for j, k in enumerate(mine) if status_mine[j] != 0]
        # the answer of a sample of the retired solves against the flash they started from
        for j, k in enumerate(mine):
            if status_mine[j] == 0 and j % max(1, len(mine) // 8) == 0:
                liq, vap = fmlbm.fmlbm_batch_phases(b, j, n)
                dev_mine.append(_phase_dev(liq, vap, states[k]))
    fmlbm.fmlbm_batch_destroy(b)
    t_batch = max_over_ranks(t_batch, dist, dev)
    units = sum_over_ranks(units, dist, dev)
    statuses = np.array(gather_lists(status_mine, dist), dtype=np.int64)
    steps_all = np.array(gather_lists(steps_mine, dist), dtype=np.int64)
    devs = gather_lists(dev_mine, dist)
    failed = gather_lists(failed_mine, dist)
    max_steps_done = int(steps_all.max()) if steps_all.size else 0

    # the plain per-lattice loop: one handle at a time, the same check interval and
    # retirement rule (the phase measure of fmlbm_phase_measure, or the residual)
    seq_units, seq_status, seq_steps = 0, [], []
    barrier()
    t0 = time.perf_counter()
    for j, k in enumerate(mine):
        L = int(sides[k])
        lat = fmlbm.Lattice(mix, L, L, 1.0, "isotropic", prec, "lagged")
        lat.init(fields[k])
        # the steps the batch autotuner took before the batch's first check, so that both
        # check the same states
        done, status = tuned_steps[j], 0
        try:
            lat.step(done)
            lam = lat.phase_measure() if args.criterion == "phase" else None
            lat.diagnostics()
            while done < args.max_steps:
                lat.step(args.check_every)
                done += args.check_every
                if args.criterion == "phase":
                    now = lat.phase_measure()
                    measure = float(np.max(np.abs(now - lam)))
                    lam = now
                else:
                    measure = lat.diagnostics()[1]
                if measure < args.tol:
                    break
            else:
                status = fmlbm.E_NOT_CONVERGED
        except fmlbm.FmlbmError as e:
            status = e.status
        seq_units += n * L * L * (done - tuned_steps[j])
        seq_status.append(status)
        seq_steps.append(done)
        lat.close()
    torch.cuda.synchronize()
    t_seq = max_over_ranks(time.perf_counter() - t0, dist, dev)
    seq_units = sum_over_ranks(seq_units, dist, dev)
    seq_steps_all = np.array(gather_lists(seq_steps, dist), dtype=np.int64)
    counts = {fmlbm.STATUS[int(v)]: int((statuses == v).sum()) for v in np.unique(statuses)}
    ok = statuses == 0
    line = dict(
        metric="batched VLE solves/sec", value=nlat / t_batch, unit="solves/s", n_gpus=world,
        steps=max_steps_done, warmup=3, ms_per_step=None, higher_is_better=True, scaling="strong",
        vs_baseline=None, dtype="f64" if prec == "fp64" else "f32", data="synthetic",
        config=dict(workload=f"batched P-x sweep: {nlat} binary PR lattices, side 4 U{{16..{args.batch_max_side // 4}}}, "
                             f"z1 0.12..0.95, flat slab of Eq. eqInit (W 4, unperturbed), tau 1.0",
                    precision=prec, max_steps=args.max_steps, check_every=args.check_every, tol=args.tol,
                    criterion=args.criterion, autotune=dict(tile_y=ty, blocks=blocks)),
        aggregate_glups=units / t_batch / 1e9, seconds=t_batch, statuses=counts,
        retired_ok_fraction=float(ok.mean()) if statuses.size else None,
        not_ok=dict(fields=["lattice", "z1", "side", "status", "steps"], rows=failed),
        steps_to_retire=dict(median=int(np.median(steps_all[ok])) if ok.any() else None,
                             max=int(steps_all[ok].max()) if ok.any() else None),
        phase_vs_start_flash=dict(sample=len(devs), max_rel=max(devs) if devs else None,
                                  median_rel=float(np.median(devs)) if devs else None),
        sequential=dict(value=nlat / t_seq, unit="solves/s", seconds=t_seq, aggregate_glups=seq_units / t_seq / 1e9,
                        kind="plain per-lattice loop, same check interval and retirement rule",
                        same_retirement_step=int((seq_steps_all == steps_all).sum()) if seq_steps_all.size ==
                        steps_all.size else None),
        speedup_vs_sequential=t_seq / t_batch,
    )
    if summary:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)


def _downsample(points: list, k: int) -> list:
    """At most k of the (t, value) points, evenly spaced in index, first and last kept;
    rounded for the JSON line."""
    if len(points) > k:
        idx = sorted({round(j * (len(points) - 1) / (k - 1)) for j in range(k)})
        points = [points[j] for j in idx]
    return [[round(t, 3), int(v)] for t, v in points]


def run_serve(args, rank, world, dist=None, summary=False):
    """Serving: Poisson arrivals of binary and ternary VLE requests (templates with random T
    and feed, side 4 x U{16..max_side / 4}); continuous batching servers, one per component count;
    against a FIFO loop that runs one request at a time with a single-lattice handle and the
    same retirement rule.  Each request starts from the unperturbed flat interface of Eq.
    eqInit between its flash phases and retires at the convergence criterion (by default the
    phase-measure change over a check interval below tol).  Under torchrun rank r serves
    requests r, r + N, ... (the same arrival stream, thinned)."""
    if summary:
        # a short serving run for the main benchmark line, at an offered load below the
        # batching server's capacity: 48 requests, sides up to 192
        args = _summary_args(args, requests=48, rate=args.summary_rate, max_side=192, check_every=500)
    import threading as th
    import torch
    from paper_2212_10680_gb300 import fmlbm, inputs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = json.load(open(os.path.join(ROOT, "tests", "golden", "workloads.json")))
    temps = [t for t in wl["serve_templates"] if "slab" in t]
    rng = np.random.default_rng(5)
    R = args.requests
    gaps = rng.exponential(1.0 / args.rate, R)
    arrive = np.cumsum(gaps) - gaps[0]
    mine = set(round_robin(R, rank, world))
    reqs = {}
    for k in range(R):
        t = temps[int(rng.integers(0, len(temps)))]
        side = 4 * int(rng.integers(16, args.max_side // 4 + 1))     # interface centres on nodes
        if k not in mine:
            continue
        rho = inputs.slab(t["slab"]["rt_vapour"], t["slab"]["rt_liquid"], side, side, 0.5, 4.0)
        reqs[k] = dict(k=k, n=len(t["mixture"]["Tc"]), mix=fmlbm.mixture_from_dict(t["mixture"]), side=side,
                       rho=rho, t=float(arrive[k]))
    if dist is not None:
        dist.barrier()
    prec = "fp32"
    servers = {nc: fmlbm.fmlbm_server_create(nc, prec, args.slots, args.check_every, args.tol, args.max_steps,
                                             int(args.budget_gb * (1 << 30)), criterion=args.criterion)
               for nc in (2, 3)}
    results = []
    timeline = []          # (seconds, device bytes admitted over both servers), every >= 50 ms

    def sample():
        now = time.perf_counter() - t0
        if not timeline or now - timeline[-1][0] >= 0.05:
            timeline.append((now, sum(fmlbm.fmlbm_server_stats(s)["bytes"] for s in servers.values())))

    t0 = time.perf_counter()
    for r in reqs.values():
        wait = r["t"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        fmlbm.fmlbm_server_submit(servers[r["n"]], r["mix"], fmlbm.make_lattice(r["side"], r["side"], 1.0,
                                                                                 "isotropic", prec), r["rho"], tag=r["k"])
        for s in servers.values():
            results += fmlbm.fmlbm_server_poll(s)
        sample()
    while len(results) < len(reqs):
        for s in servers.values():
            results += fmlbm.fmlbm_server_poll(s)
        sample()
        time.sleep(0.002)
    wall = max_over_ranks(time.perf_counter() - t0, dist, dev)
    busy = {nc: sum_over_ranks(fmlbm.fmlbm_server_stats(s)["busy"], dist, dev) / world for nc, s in servers.items()}
    for s in servers.values():
        fmlbm.fmlbm_server_destroy(s)
    lat_s = gather_lists([r["t_done"] - r["t_submit"] for r in results], dist)
    units = sum_over_ranks(sum(reqs[r["tag"]]["n"] * reqs[r["tag"]]["side"] ** 2 * r["steps"] for r in results),
                           dist, dev)
    status_all = gather_lists([r["status"] for r in results], dist)

    # FIFO baseline: the same arrivals, one request at a time through a single-lattice handle,
    # the same check interval and retirement rule
    seq_lat, seq_status = [], []
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for r in reqs.values():
        wait = r["t"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        lat = fmlbm.Lattice(r["mix"], r["side"], r["side"], 1.0, "isotropic", prec, "lagged")
        lat.init(r["rho"])
        done, status = 0, 0
        try:
            lat.diagnostics()
            lam = lat.phase_measure() if args.criterion == "phase" else None
            while True:
                lat.step(args.check_every)
                done += args.check_every
                if args.criterion == "phase":
                    now = lat.phase_measure()
                    measure = float(np.max(np.abs(now - lam)))
                    lam = now
                else:
                    measure = lat.diagnostics()[1]
                if measure < args.tol:
                    break
                if done >= args.max_steps:
                    status = fmlbm.E_NOT_CONVERGED
                    break
        except fmlbm.FmlbmError as e:
            status = e.status
        lat.close()
        seq_lat.append(time.perf_counter() - t0 - r["t"])
        seq_status.append(status)
    seq_wall = max_over_ranks(time.perf_counter() - t0, dist, dev)
    seq_lat = gather_lists(seq_lat, dist)
    seq_status = gather_lists(seq_status, dist)
    counts, seq_counts = {}, {}
    for s_ in status_all:
        counts[fmlbm.STATUS[s_]] = counts.get(fmlbm.STATUS[s_], 0) + 1
    for s_ in seq_status:
        seq_counts[fmlbm.STATUS[s_]] = seq_counts.get(fmlbm.STATUS[s_], 0) + 1

    line = dict(
        metric="served VLE solves/sec", value=R / wall, unit="solves/s", n_gpus=world, steps=args.max_steps,
        warmup=0, ms_per_step=None, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic", config=dict(
            workload=f"Poisson arrivals ({args.rate}/s) of {R} binary/ternary PR VLE requests, side "
                     f"4 U{{16..{args.max_side // 4}}}, T U[0.80,0.92] Tc1 (binary) / U[0.85,0.92] Tc1 (ternary), "
                     f"flat slab of Eq. eqInit (W 4, unperturbed)",
            slots=args.slots, chunk_steps=args.check_every, tol=args.tol, criterion=args.criterion,
            max_steps=args.max_steps, hbm_budget_gb=args.budget_gb),
        retired_ok_fraction=counts.get("FMLBM_OK", 0) / max(len(status_all), 1),
        p50_s=_stats_pct(lat_s, 50), p99_s=_stats_pct(lat_s, 99), aggregate_glups=units / wall / 1e9,
        gpu_busy_fraction={str(k): v / wall for k, v in busy.items()}, statuses=counts, seconds=wall,
        admitted_bytes=dict(max=max((b for _, b in timeline), default=0), budget=int(args.budget_gb * (1 << 30)),
                            timeline=_downsample(timeline, 40), note="rank 0's servers, sampled every >= 50 ms"),
        fifo_baseline=dict(value=R / seq_wall, unit="solves/s", p50_s=_stats_pct(seq_lat, 50),
                           p99_s=_stats_pct(seq_lat, 99), seconds=seq_wall, statuses=seq_counts),
    )
    if summary:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="droplet1024")
    ap.add_argument("--size", type=int, default=0, help="scale the workload's lattice to size x size (profiling)")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--tile-y", type=int, default=0, help="override the fused step's tile height (8 or 16)")
    ap.add_argument("--variant", default=None, choices=["auto", "plain", "tma", "tma_tile", "pair", "multi"], help="step kernel variant")
    ap.add_argument("--batch-lattices", type=int, default=256)
    ap.add_argument("--batch-max-side", type=int, default=512)
    ap.add_argument("--max-steps", type=int, default=300000)
    ap.add_argument("--check-every", type=int, default=500)
    ap.add_argument("--tol", type=float, default=2e-6,
                    help="retirement threshold of the convergence measure over one check interval")
    ap.add_argument("--criterion", default="phase", choices=["phase", "residual"])
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--max-side", type=int, default=1024)
    ap.add_argument("--slots", type=int, default=256)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--e2e-steps", type=int, default=500, help="steps of the amortized end-to-end figure")
    ap.add_argument("--no-configs", action="store_true", help="only the headline workload (no per-config objects)")
    ap.add_argument("--summary-rate", type=float, default=7.0, help="offered load (req/s) of the serving summary")
    ap.add_argument("--summary-rate-low", type=float, default=1.5,
                    help="offered load (req/s) of the second serving summary (below the FIFO loop's capacity)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        w = workload(args.workload, args.size)
        run_reference(args, w, rank, world)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        td.init_process_group("nccl")
        dist = td
    if args.workload == "batch256":
        run_batch(args, rank, world, dist)
    elif args.workload == "serve":
        run_serve(args, rank, world, dist)
    else:
        w = workload(args.workload, args.size)
        run_ours(args, w, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
