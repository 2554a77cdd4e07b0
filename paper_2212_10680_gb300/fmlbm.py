"""Thin ctypes binding of libfmlbm.so (the C ABI in include/fmlbm.h).

Only argument marshalling lives here: every step of the lattice update runs in the
library's CUDA kernels.  The functions carry the C names; each raises FmlbmError on
a non-zero status.  If the shared library is missing, importing this module fails
loudly; there is no CPU fallback.

Host arrays are numpy float64, C order, with the layouts documented in fmlbm.h:
fields [N][ny][nx], vectors [2][ny][nx], distributions [N][9][ny][nx].
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

MAX_COMPONENTS = 4
_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfmlbm.so")

EOS = {"pr": 0, "srk": 1, "vdw": 2}
STENCIL = {"isotropic": 0, "central": 1}
PRECISION = {"fp64": 0, "fp32": 1, "fp16dev": 2, "bf16dev": 3, "fp16dev_lnf64": 4, "bf16dev_lnf64": 5}
VELOCITY_FORCE = {"lagged": 0, "current": 1}
FORMULATION = {"well_balanced": 0, "standard": 1}
STATUS = {0: "FMLBM_OK", 1: "FMLBM_E_INVALID_ARG", 2: "FMLBM_E_OOM", 3: "FMLBM_E_CUDA",
          4: "FMLBM_E_NONPHYSICAL", 5: "FMLBM_E_TIMEOUT", 6: "FMLBM_E_BUSY", 7: "FMLBM_E_NOT_CONVERGED",
          8: "FMLBM_E_UNSUPPORTED"}
E_NONPHYSICAL = 4
E_TIMEOUT = 5
E_NOT_CONVERGED = 7
E_BUSY = 6
E_UNSUPPORTED = 8


class FmlbmError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        super().__init__(f"{where}: {STATUS.get(status, status)} {message}".strip())
        self.status = status


class fmlbm_mixture(ctypes.Structure):
    _fields_ = [("n_components", ctypes.c_int32), ("eos", ctypes.c_int32), ("R", ctypes.c_double),
                ("T", ctypes.c_double), ("Tc", ctypes.c_double * MAX_COMPONENTS),
                ("Pc", ctypes.c_double * MAX_COMPONENTS), ("omega", ctypes.c_double * MAX_COMPONENTS),
                ("M", ctypes.c_double * MAX_COMPONENTS), ("kappa", ctypes.c_double * MAX_COMPONENTS),
                ("kij", ctypes.c_double * (MAX_COMPONENTS * MAX_COMPONENTS))]


class fmlbm_lattice(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("tau", ctypes.c_double),
                ("stencil", ctypes.c_int32), ("precision", ctypes.c_int32), ("velocity_force", ctypes.c_int32),
                ("formulation", ctypes.c_int32)]


class fmlbm_server_config(ctypes.Structure):
    _fields_ = [("n_components", ctypes.c_int32), ("precision", ctypes.c_int32), ("max_slots", ctypes.c_int32),
                ("chunk_steps", ctypes.c_int32), ("tol", ctypes.c_double), ("max_steps", ctypes.c_int64),
                ("hbm_budget_bytes", ctypes.c_size_t), ("queue_capacity", ctypes.c_int32),
                ("criterion", ctypes.c_int32)]


class fmlbm_request(ctypes.Structure):
    _fields_ = [("mixture", fmlbm_mixture), ("lattice", fmlbm_lattice), ("rho", ctypes.POINTER(ctypes.c_double)),
                ("rho_out", ctypes.POINTER(ctypes.c_double)), ("tag", ctypes.c_uint64)]


class fmlbm_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("n_components", ctypes.c_int32), ("steps", ctypes.c_int64), ("residual", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("rho_liquid", ctypes.c_double * MAX_COMPONENTS), ("rho_vapour", ctypes.c_double * MAX_COMPONENTS)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libfmlbm.so is not built ({_LIB_PATH}); run "
                          "`python -m paper_2212_10680_gb300.build` first")
    lib = ctypes.CDLL(_LIB_PATH)
    H = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "fmlbm_create": ([ctypes.POINTER(fmlbm_mixture), ctypes.POINTER(fmlbm_lattice), ctypes.c_void_p,
                          ctypes.POINTER(H)], ctypes.c_int),
        "fmlbm_create_with_buffers": ([ctypes.POINTER(fmlbm_mixture), ctypes.POINTER(fmlbm_lattice), ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(H)], ctypes.c_int),
        "fmlbm_buffer_sizes": ([ctypes.c_int32, ctypes.POINTER(fmlbm_lattice), ctypes.POINTER(ctypes.c_size_t),
                                ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "fmlbm_init": ([H, dp], ctypes.c_int),
        "fmlbm_init_device": ([H, ctypes.c_void_p], ctypes.c_int),
        "fmlbm_step": ([H, ctypes.c_int64], ctypes.c_int),
        "fmlbm_moments": ([H, dp, dp, dp], ctypes.c_int),
        "fmlbm_get_distributions": ([H, dp, dp], ctypes.c_int),
        "fmlbm_set_distributions": ([H, dp, dp], ctypes.c_int),
        "fmlbm_diagnostics": ([H, dp, dp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "fmlbm_phase_measure": ([H, dp], ctypes.c_int),
        "fmlbm_step_diagnostics": ([H, ctypes.c_int64, dp, dp], ctypes.c_int),
        "fmlbm_error_node": ([H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "fmlbm_state_size": ([H, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "fmlbm_get_state": ([H, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
        "fmlbm_set_state": ([H, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
        "fmlbm_synchronize": ([H], ctypes.c_int),
        "fmlbm_set_tile_height": ([H, ctypes.c_int32], ctypes.c_int),
        "fmlbm_set_step_variant": ([H, ctypes.c_int32], ctypes.c_int),
        "fmlbm_get_step_variant": ([H, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "fmlbm_set_wait_limit": ([H, ctypes.c_int64], ctypes.c_int),
        "fmlbm_autotune": ([H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), dp],
                           ctypes.c_int),
        "fmlbm_lattice_bytes": ([ctypes.c_int32, ctypes.POINTER(fmlbm_lattice), ctypes.POINTER(ctypes.c_size_t)],
                                ctypes.c_int),
        "fmlbm_diagnostics_noalloc": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
        "fmlbm_diagnostics_async": ([H, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "fmlbm_diagnostics_wait": ([H, ctypes.c_int64, dp, dp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "fmlbm_destroy": ([H], None),
        "fmlbm_batch_create": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(H)],
                               ctypes.c_int),
        "fmlbm_batch_add": ([H, ctypes.POINTER(fmlbm_mixture), ctypes.POINTER(fmlbm_lattice), dp,
                             ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "fmlbm_batch_remove": ([H, ctypes.c_int32], ctypes.c_int),
        "fmlbm_batch_set_active": ([H, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
        "fmlbm_batch_step": ([H, ctypes.c_int64], ctypes.c_int),
        "fmlbm_batch_check": ([H], ctypes.c_int),
        "fmlbm_batch_run": ([H, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(ctypes.c_int64), dp,
                             ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "fmlbm_batch_slot_info": ([H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), dp,
                                   ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "fmlbm_batch_moments": ([H, ctypes.c_int32, dp, dp, dp], ctypes.c_int),
        "fmlbm_batch_set_criterion": ([H, ctypes.c_int32], ctypes.c_int),
        "fmlbm_batch_slot_phase_change": ([H, ctypes.c_int32, dp], ctypes.c_int),
        "fmlbm_batch_phases": ([H, ctypes.c_int32, dp, dp], ctypes.c_int),
        "fmlbm_batch_get_distributions": ([H, ctypes.c_int32, dp, dp], ctypes.c_int),
        "fmlbm_batch_autotune": ([H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                  dp], ctypes.c_int),
        "fmlbm_batch_bytes": ([H, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "fmlbm_batch_last_error": ([H], ctypes.c_char_p),
        "fmlbm_batch_destroy": ([H], None),
        "fmlbm_batch_run_chunk": ([H, ctypes.c_int32], ctypes.c_int),
        "fmlbm_server_create": ([ctypes.POINTER(fmlbm_server_config), ctypes.POINTER(H)], ctypes.c_int),
        "fmlbm_server_submit": ([H, ctypes.POINTER(fmlbm_request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "fmlbm_server_poll": ([H, ctypes.POINTER(fmlbm_result), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)],
                              ctypes.c_int),
        "fmlbm_server_stats": ([H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_size_t), dp, dp], ctypes.c_int),
        "fmlbm_server_destroy": ([H], None),
        "fmlbm_status_str": ([ctypes.c_int], ctypes.c_char_p),
        "fmlbm_last_error": ([H], ctypes.c_char_p),
        "fmlbm_version": ([], ctypes.c_char_p),
        "fmlbm_decomp_slab_rows": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "fmlbm_decomp_create": ([ctypes.POINTER(fmlbm_mixture), ctypes.POINTER(fmlbm_lattice), ctypes.c_int32,
                                 ctypes.c_void_p, ctypes.POINTER(H)], ctypes.c_int),
        "fmlbm_decomp_init": ([H, dp], ctypes.c_int),
        "fmlbm_decomp_step": ([H, ctypes.c_int64], ctypes.c_int),
        "fmlbm_decomp_get_distributions": ([H, dp, dp], ctypes.c_int),
        "fmlbm_decomp_last_error": ([H], ctypes.c_char_p),
        "fmlbm_decomp_destroy": ([H], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


LIB = _load()


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(status: int, where: str, h=None):
    if status != 0:
        msg = LIB.fmlbm_last_error(h).decode() if h else ""
        raise FmlbmError(status, where, msg)


def make_mixture(eos: str, R: float, T: float, Tc: Sequence[float], Pc: Sequence[float], omega: Sequence[float],
                 M: Sequence[float] = None, kappa: Sequence[float] = None, kij=None) -> fmlbm_mixture:
    n = len(Tc)
    m = fmlbm_mixture()
    m.n_components = n
    m.eos = EOS[eos.lower()]
    m.R, m.T = R, T
    M = [1.0] * n if M is None else M
    kappa = [0.0] * n if kappa is None else kappa
    kij = np.zeros((n, n)) if kij is None else np.asarray(kij, dtype=np.float64).reshape(n, n)
    for i in range(n):
        m.Tc[i], m.Pc[i], m.omega[i], m.M[i], m.kappa[i] = Tc[i], Pc[i], omega[i], M[i], kappa[i]
        for j in range(n):
            m.kij[i * MAX_COMPONENTS + j] = kij[i, j]
    return m


def mixture_from_dict(d: dict) -> fmlbm_mixture:
    return make_mixture(d["eos"], d["R"], d["T"], d["Tc"], d["Pc"], d["omega"], d.get("M"), d.get("kappa"),
                        d.get("kij"))


def make_lattice(nx: int, ny: int, tau: float, stencil: str = "isotropic", precision: str = "fp32",
                 velocity_force: str = "lagged", formulation: str = "well_balanced") -> fmlbm_lattice:
    L = fmlbm_lattice()
    L.nx, L.ny, L.tau = nx, ny, tau
    L.stencil = STENCIL[stencil]
    L.precision = PRECISION[precision]
    L.velocity_force = VELOCITY_FORCE[velocity_force]
    L.formulation = FORMULATION[formulation]
    return L


# ---- the C entry points, one wrapper each ----

def fmlbm_create(mixture: fmlbm_mixture, lattice: fmlbm_lattice, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(LIB.fmlbm_create(ctypes.byref(mixture), ctypes.byref(lattice), ctypes.c_void_p(stream or None),
                            ctypes.byref(h)), "fmlbm_create")
    return h


def fmlbm_buffer_sizes(n_components: int, lattice: fmlbm_lattice):
    """(g_bytes, g0_bytes, force_bytes) of each caller-provided buffer."""
    s = [ctypes.c_size_t() for _ in range(3)]
    _check(LIB.fmlbm_buffer_sizes(n_components, ctypes.byref(lattice), *[ctypes.byref(x) for x in s]),
           "fmlbm_buffer_sizes")
    return tuple(x.value for x in s)


def fmlbm_create_with_buffers(mixture: fmlbm_mixture, lattice: fmlbm_lattice, g, g0, force,
                              stream: int = 0) -> ctypes.c_void_p:
    """g, force: two device addresses each (e.g. tensor.data_ptr()); g0: two addresses for the
    deviation forms, else None.  The caller keeps ownership of the buffers."""
    pair = ctypes.c_void_p * 2
    h = ctypes.c_void_p()
    _check(LIB.fmlbm_create_with_buffers(ctypes.byref(mixture), ctypes.byref(lattice), ctypes.c_void_p(stream or None),
                                         pair(*g), pair(*g0) if g0 else None, pair(*force), ctypes.byref(h)),
           "fmlbm_create_with_buffers")
    return h


def fmlbm_init(h, rho: np.ndarray):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    _check(LIB.fmlbm_init(h, _ptr(rho)), "fmlbm_init", h)


def fmlbm_init_device(h, rho_device_ptr: int):
    _check(LIB.fmlbm_init_device(h, ctypes.c_void_p(rho_device_ptr)), "fmlbm_init_device", h)


def fmlbm_step(h, nsteps: int):
    _check(LIB.fmlbm_step(h, ctypes.c_int64(nsteps)), "fmlbm_step", h)


def fmlbm_moments(h, rho: np.ndarray = None, u: np.ndarray = None, lnf: np.ndarray = None):
    _check(LIB.fmlbm_moments(h, _ptr(rho), _ptr(u), _ptr(lnf)), "fmlbm_moments", h)


def fmlbm_get_distributions(h, g: np.ndarray = None, force: np.ndarray = None):
    _check(LIB.fmlbm_get_distributions(h, _ptr(g), _ptr(force)), "fmlbm_get_distributions", h)


def fmlbm_set_distributions(h, g: np.ndarray, force: np.ndarray = None):
    g = np.ascontiguousarray(g, dtype=np.float64)
    force = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    _check(LIB.fmlbm_set_distributions(h, _ptr(g), _ptr(force)), "fmlbm_set_distributions", h)


def fmlbm_diagnostics(h, n_components: int):
    mass = np.empty(n_components)
    res = ctypes.c_double()
    step = ctypes.c_int64()
    st = LIB.fmlbm_diagnostics(h, _ptr(mass), ctypes.byref(res), ctypes.byref(step))
    _check(st, "fmlbm_diagnostics", h)
    return mass, res.value, step.value


def fmlbm_diagnostics_async(h) -> int:
    """Ticket for the diagnostics of the current state (computed inside the next step)."""
    t = ctypes.c_int64()
    _check(LIB.fmlbm_diagnostics_async(h, ctypes.byref(t)), "fmlbm_diagnostics_async", h)
    return t.value


def fmlbm_step_diagnostics(h, nsteps: int, n_components: int):
    """nsteps steps with every step's diagnostics: masses [nsteps][N], residuals [nsteps]."""
    mass = np.empty((max(nsteps, 0), n_components))
    res = np.empty(max(nsteps, 0))
    _check(LIB.fmlbm_step_diagnostics(h, nsteps, _ptr(mass), _ptr(res)), "fmlbm_step_diagnostics", h)
    return mass, res


def fmlbm_diagnostics_wait(h, ticket: int, n_components: int):
    mass = np.empty(n_components)
    res = ctypes.c_double()
    step = ctypes.c_int64()
    st = LIB.fmlbm_diagnostics_wait(h, ticket, _ptr(mass), ctypes.byref(res), ctypes.byref(step))
    _check(st, "fmlbm_diagnostics_wait", h)
    return mass, res.value, step.value


def fmlbm_phase_measure(h, n_components: int) -> np.ndarray:
    """lambda_i = mean over the nodes of ln rho_i, per component."""
    lam = np.empty(n_components)
    _check(LIB.fmlbm_phase_measure(h, _ptr(lam)), "fmlbm_phase_measure", h)
    return lam


def fmlbm_error_node(h):
    c, x, y = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(LIB.fmlbm_error_node(h, ctypes.byref(c), ctypes.byref(x), ctypes.byref(y)), "fmlbm_error_node", h)
    return c.value, x.value, y.value


def fmlbm_state_size(h) -> int:
    n = ctypes.c_size_t()
    _check(LIB.fmlbm_state_size(h, ctypes.byref(n)), "fmlbm_state_size", h)
    return n.value


def fmlbm_get_state(h) -> bytes:
    n = fmlbm_state_size(h)
    buf = ctypes.create_string_buffer(n)
    _check(LIB.fmlbm_get_state(h, buf, n), "fmlbm_get_state", h)
    return buf.raw


def fmlbm_set_state(h, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(LIB.fmlbm_set_state(h, buf, len(state)), "fmlbm_set_state", h)


def fmlbm_set_tile_height(h, tile_y: int):
    _check(LIB.fmlbm_set_tile_height(h, tile_y), "fmlbm_set_tile_height", h)


VARIANT = {"auto": 0, "plain": 1, "tma": 2, "tma_tile": 3, "pair": 4, "multi": 5}
CRITERION = {"residual": 0, "phase": 1}


def fmlbm_set_step_variant(h, variant: str):
    _check(LIB.fmlbm_set_step_variant(h, VARIANT[variant]), "fmlbm_set_step_variant", h)


def fmlbm_get_step_variant(h) -> str:
    v = ctypes.c_int32()
    _check(LIB.fmlbm_get_step_variant(h, ctypes.byref(v)), "fmlbm_get_step_variant", h)
    return {1: "plain", 2: "tma", 3: "tma_tile", 4: "pair", 5: "multi"}[v.value]


def fmlbm_set_wait_limit(h, polls: int):
    _check(LIB.fmlbm_set_wait_limit(h, polls), "fmlbm_set_wait_limit", h)


def fmlbm_autotune(h, steps_per_trial: int = 5):
    v, ty, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(LIB.fmlbm_autotune(h, steps_per_trial, ctypes.byref(v), ctypes.byref(ty), ctypes.byref(ms)),
           "fmlbm_autotune", h)
    return {1: "plain", 2: "tma", 3: "tma_tile", 4: "pair", 5: "multi"}[v.value], ty.value, ms.value


def fmlbm_synchronize(h):
    _check(LIB.fmlbm_synchronize(h), "fmlbm_synchronize", h)


def fmlbm_lattice_bytes(n_components: int, lattice: fmlbm_lattice) -> int:
    n = ctypes.c_size_t()
    _check(LIB.fmlbm_lattice_bytes(n_components, ctypes.byref(lattice), ctypes.byref(n)), "fmlbm_lattice_bytes")
    return n.value


def fmlbm_diagnostics_noalloc(n_components: int, nx: int, ny: int, precision: str, g_device: int,
                              g0_device: int, rho_prev_device: int, have_prev: bool, out_device: int,
                              stream: int = 0):
    """Device pointers in, device results out; allocates nothing (see fmlbm.h)."""
    _check(LIB.fmlbm_diagnostics_noalloc(n_components, nx, ny, PRECISION[precision], ctypes.c_void_p(g_device),
                                         ctypes.c_void_p(g0_device or None), ctypes.c_void_p(rho_prev_device),
                                         int(bool(have_prev)), ctypes.c_void_p(out_device),
                                         ctypes.c_void_p(stream or None)), "fmlbm_diagnostics_noalloc")


def fmlbm_destroy(h):
    LIB.fmlbm_destroy(h)


def fmlbm_version() -> str:
    return LIB.fmlbm_version().decode()


def _bcheck(status: int, where: str, b=None):
    if status != 0:
        msg = LIB.fmlbm_batch_last_error(b).decode() if b else ""
        raise FmlbmError(status, where, msg)


def fmlbm_batch_create(n_components: int, precision: str, capacity: int, stream: int = 0):
    b = ctypes.c_void_p()
    _bcheck(LIB.fmlbm_batch_create(n_components, PRECISION[precision], capacity, ctypes.c_void_p(stream or None),
                                   ctypes.byref(b)), "fmlbm_batch_create")
    return b


def fmlbm_batch_add(b, mixture: fmlbm_mixture, lattice: fmlbm_lattice, rho: np.ndarray) -> int:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    slot = ctypes.c_int32()
    _bcheck(LIB.fmlbm_batch_add(b, ctypes.byref(mixture), ctypes.byref(lattice), _ptr(rho), ctypes.byref(slot)),
            "fmlbm_batch_add", b)
    return slot.value


def fmlbm_batch_remove(b, slot: int):
    _bcheck(LIB.fmlbm_batch_remove(b, slot), "fmlbm_batch_remove", b)


def fmlbm_batch_set_active(b, slot: int, active: bool):
    _bcheck(LIB.fmlbm_batch_set_active(b, slot, int(bool(active))), "fmlbm_batch_set_active", b)


def fmlbm_batch_step(b, nsteps: int):
    _bcheck(LIB.fmlbm_batch_step(b, ctypes.c_int64(nsteps)), "fmlbm_batch_step", b)


def fmlbm_batch_check(b):
    _bcheck(LIB.fmlbm_batch_check(b), "fmlbm_batch_check", b)


def fmlbm_batch_run(b, capacity: int, max_steps: int, check_every: int, tol: float):
    steps = np.zeros(capacity, dtype=np.int64)
    res = np.zeros(capacity)
    st = np.zeros(capacity, dtype=np.int32)
    _bcheck(LIB.fmlbm_batch_run(b, ctypes.c_int64(max_steps), check_every, tol,
                                steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(res),
                                st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "fmlbm_batch_run", b)
    return steps, res, st


def fmlbm_batch_slot_info(b, slot: int):
    steps, res, st, act = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32()
    _bcheck(LIB.fmlbm_batch_slot_info(b, slot, ctypes.byref(steps), ctypes.byref(res), ctypes.byref(st),
                                      ctypes.byref(act)), "fmlbm_batch_slot_info", b)
    return steps.value, res.value, st.value, bool(act.value)


def fmlbm_batch_set_criterion(b, criterion: str):
    _bcheck(LIB.fmlbm_batch_set_criterion(b, CRITERION[criterion]), "fmlbm_batch_set_criterion", b)


def fmlbm_batch_slot_phase_change(b, slot: int) -> float:
    v = ctypes.c_double()
    _bcheck(LIB.fmlbm_batch_slot_phase_change(b, slot, ctypes.byref(v)), "fmlbm_batch_slot_phase_change", b)
    return v.value


def fmlbm_batch_moments(b, slot: int, rho=None, u=None, lnf=None):
    _bcheck(LIB.fmlbm_batch_moments(b, slot, _ptr(rho), _ptr(u), _ptr(lnf)), "fmlbm_batch_moments", b)


def fmlbm_batch_phases(b, slot: int, n_components: int):
    """(rho~ at the densest node, rho~ at the least dense node), molar densities."""
    liq, vap = np.empty(n_components), np.empty(n_components)
    _bcheck(LIB.fmlbm_batch_phases(b, slot, _ptr(liq), _ptr(vap)), "fmlbm_batch_phases", b)
    return liq, vap


def fmlbm_batch_get_distributions(b, slot: int, g=None, force=None):
    _bcheck(LIB.fmlbm_batch_get_distributions(b, slot, _ptr(g), _ptr(force)), "fmlbm_batch_get_distributions", b)


def fmlbm_batch_autotune(b, steps_per_trial: int = 5):
    ty, blocks, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _bcheck(LIB.fmlbm_batch_autotune(b, steps_per_trial, ctypes.byref(ty), ctypes.byref(blocks), ctypes.byref(ms)),
            "fmlbm_batch_autotune", b)
    return ty.value, blocks.value, ms.value


def fmlbm_batch_bytes(b) -> int:
    n = ctypes.c_size_t()
    _bcheck(LIB.fmlbm_batch_bytes(b, ctypes.byref(n)), "fmlbm_batch_bytes", b)
    return n.value


def fmlbm_batch_destroy(b):
    LIB.fmlbm_batch_destroy(b)


def fmlbm_batch_run_chunk(b, steps: int):
    _bcheck(LIB.fmlbm_batch_run_chunk(b, steps), "fmlbm_batch_run_chunk", b)


def fmlbm_server_create(n_components: int, precision: str, max_slots: int, chunk_steps: int, tol: float,
                        max_steps: int, hbm_budget_bytes: int, queue_capacity: int = 4096,
                        criterion: str = "residual"):
    cfg = fmlbm_server_config(n_components, PRECISION[precision], max_slots, chunk_steps, tol, max_steps,
                              hbm_budget_bytes, queue_capacity, CRITERION[criterion])
    s = ctypes.c_void_p()
    _check(LIB.fmlbm_server_create(ctypes.byref(cfg), ctypes.byref(s)), "fmlbm_server_create")
    return s


def fmlbm_server_submit(s, mixture: fmlbm_mixture, lattice: fmlbm_lattice, rho: np.ndarray, rho_out=None,
                        tag: int = 0) -> int:
    """Queues a solve; returns its id.  rho is copied; rho_out (if given) must stay alive until
    the result has been polled."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    req = fmlbm_request(mixture, lattice, _ptr(rho), _ptr(rho_out), tag)
    rid = ctypes.c_uint64()
    _check(LIB.fmlbm_server_submit(s, ctypes.byref(req), ctypes.byref(rid)), "fmlbm_server_submit")
    return rid.value


def fmlbm_server_poll(s, capacity: int = 1024):
    out = (fmlbm_result * capacity)()
    n = ctypes.c_int32()
    _check(LIB.fmlbm_server_poll(s, out, capacity, ctypes.byref(n)), "fmlbm_server_poll")
    return [dict(id=r.id, tag=r.tag, status=r.status, steps=r.steps, residual=r.residual, t_submit=r.t_submit,
                 t_admit=r.t_admit, t_done=r.t_done, rho_liquid=list(r.rho_liquid[:r.n_components]),
                 rho_vapour=list(r.rho_vapour[:r.n_components])) for r in out[:n.value]]


def fmlbm_server_stats(s):
    q, r, b, busy, now = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t(), ctypes.c_double(), ctypes.c_double()
    _check(LIB.fmlbm_server_stats(s, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b), ctypes.byref(busy),
                                  ctypes.byref(now)), "fmlbm_server_stats")
    return dict(queued=q.value, running=r.value, bytes=b.value, busy=busy.value, now=now.value)


def fmlbm_server_destroy(s):
    LIB.fmlbm_server_destroy(s)


class Lattice:
    """One lattice on the current CUDA device; a convenience owner of a handle."""

    def __init__(self, mixture: fmlbm_mixture, nx: int, ny: int, tau: float, stencil: str = "isotropic",
                 precision: str = "fp32", velocity_force: str = "lagged", stream: int = 0,
                 formulation: str = "well_balanced", buffers: Optional[dict] = None):
        """buffers: {"g": (a0, a1), "g0": (a0, a1) or None, "force": (a0, a1)}, device addresses of
        caller-owned storage (fmlbm_create_with_buffers); None: the handle allocates its own."""
        self.n = mixture.n_components
        self.nx, self.ny = nx, ny
        lat = make_lattice(nx, ny, tau, stencil, precision, velocity_force, formulation)
        if buffers is None:
            self.h = fmlbm_create(mixture, lat, stream)
        else:
            self.h = fmlbm_create_with_buffers(mixture, lat, buffers["g"], buffers.get("g0"), buffers["force"], stream)

    def init(self, rho: np.ndarray):
        fmlbm_init(self.h, rho)

    def step(self, n: int = 1):
        fmlbm_step(self.h, n)

    def moments(self):
        rho = np.empty((self.n, self.ny, self.nx))
        u = np.empty((2, self.ny, self.nx))
        lnf = np.empty((self.n, self.ny, self.nx))
        fmlbm_moments(self.h, rho, u, lnf)
        return rho, u, lnf

    def distributions(self):
        g = np.empty((self.n, 9, self.ny, self.nx))
        F = np.empty((2, self.ny, self.nx))
        fmlbm_get_distributions(self.h, g, F)
        return g, F

    def set_distributions(self, g, F=None):
        fmlbm_set_distributions(self.h, g, F)

    def diagnostics(self):
        return fmlbm_diagnostics(self.h, self.n)

    def phase_measure(self):
        return fmlbm_phase_measure(self.h, self.n)

    def synchronize(self):
        fmlbm_synchronize(self.h)

    def close(self):
        if self.h:
            fmlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- domain decomposition of one lattice into y-slabs (fmlbm.h: fmlbm_decomp_*) ----

def fmlbm_decomp_slab_rows(ny: int, nslabs: int, slab: int):
    """(first row, row count) of the global lattice that slab `slab` owns; needs no GPU."""
    y0, rows = ctypes.c_int32(), ctypes.c_int32()
    _check(LIB.fmlbm_decomp_slab_rows(ny, nslabs, slab, ctypes.byref(y0), ctypes.byref(rows)),
           "fmlbm_decomp_slab_rows")
    return y0.value, rows.value


def _dcheck(status: int, where: str, d=None):
    if status != 0:
        msg = LIB.fmlbm_decomp_last_error(d).decode() if d else ""
        raise FmlbmError(status, where, msg)


class Decomposition:
    """One lattice split into nslabs y-slabs with ghost rows exchanged after every step."""

    def __init__(self, mixture: fmlbm_mixture, nx: int, ny: int, tau: float, nslabs: int, stencil: str = "isotropic",
                 precision: str = "fp32", velocity_force: str = "lagged", stream: int = 0):
        self.n, self.nx, self.ny = mixture.n_components, nx, ny
        lat = make_lattice(nx, ny, tau, stencil, precision, velocity_force)
        self.d = ctypes.c_void_p()
        _dcheck(LIB.fmlbm_decomp_create(ctypes.byref(mixture), ctypes.byref(lat), nslabs, ctypes.c_void_p(stream or None),
                                        ctypes.byref(self.d)), "fmlbm_decomp_create")

    def init(self, rho: np.ndarray):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        _dcheck(LIB.fmlbm_decomp_init(self.d, rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                "fmlbm_decomp_init", self.d)

    def step(self, n: int = 1):
        _dcheck(LIB.fmlbm_decomp_step(self.d, n), "fmlbm_decomp_step", self.d)

    def distributions(self):
        g = np.empty((self.n, 9, self.ny, self.nx))
        F = np.empty((2, self.ny, self.nx))
        dp_ = ctypes.POINTER(ctypes.c_double)
        _dcheck(LIB.fmlbm_decomp_get_distributions(self.d, g.ctypes.data_as(dp_), F.ctypes.data_as(dp_)),
                "fmlbm_decomp_get_distributions", self.d)
        return g, F

    def close(self):
        if self.d:
            LIB.fmlbm_decomp_destroy(self.d)
            self.d = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
