"""Seeded synthetic inputs: initial density fields for the lattice.

This module holds no arithmetic of the lattice Boltzmann method itself.  It builds
the initial component mass-density fields rho_i(x, y, t=0) that both the CUDA path
and the test oracle start from:

* ``slab``     -- the flat-interface tanh profile of Eq. eqInit (a liquid slab in the
                  middle of the x-range, vapour outside, uniform along y);
* ``droplet``  -- the tanh profile of Eq. eqInit2D (an elliptical liquid droplet in
                  vapour; h = 1 gives a circle);
* ``uniform_noise`` / ``with_noise`` -- multiplicative noise rho_i <- rho_i (1 + a xi),
  xi uniform in [-1, 1), from a counter-based splitmix64 generator keyed by
  (seed, lattice id, component) and counted by the node index, so that any
  sub-block of a lattice can be regenerated independently and identically.

Arrays have shape (N, ny, nx), float64, C order (component-major, then rows).
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """Steele, Lea & Flood's SplitMix64 finaliser applied to x + golden gamma (wrapping uint64)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform_noise(seed: int, lattice: int, comp: int, n: int) -> np.ndarray:
    """n draws of xi ~ U[-1, 1) for (seed, lattice, comp), node k uses counter k."""
    key = splitmix64(np.uint64(seed) ^ splitmix64(np.uint64(lattice) ^ splitmix64(np.uint64(comp))))
    with np.errstate(over="ignore"):
        bits = splitmix64(key + np.arange(n, dtype=np.uint64))
    u = (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)  # [0, 1)
    return 2.0 * u - 1.0


def with_noise(rho: np.ndarray, amplitude: float, seed: int, lattice: int = 0) -> np.ndarray:
    """rho_i(x) (1 + amplitude xi_i(x)), independent per component and node."""
    rho = np.asarray(rho, dtype=np.float64)
    out = np.empty_like(rho)
    n = rho[0].size
    for i in range(rho.shape[0]):
        xi = uniform_noise(seed, lattice, i, n).reshape(rho.shape[1:])
        out[i] = rho[i] * (1.0 + amplitude * xi)
    return out


def slab(rho_v, rho_l, nx: int, ny: int, S_V: float = 0.5, W: float = 4.0) -> np.ndarray:
    """Eq. eqInit: rho_i(x) = rho_V + (rho_L - rho_V)/2 [tanh(2(x - S_V n_x/2)/W)
    - tanh(2(x - (1 - S_V/2) n_x)/W)], the same on every row."""
    rho_v = np.asarray(rho_v, dtype=np.float64)
    rho_l = np.asarray(rho_l, dtype=np.float64)
    x = np.arange(nx, dtype=np.float64)
    prof = np.tanh(2.0 * (x - 0.5 * S_V * nx) / W) - np.tanh(2.0 * (x - (1.0 - 0.5 * S_V) * nx) / W)
    out = rho_v[:, None] + 0.5 * (rho_l - rho_v)[:, None] * prof[None, :]
    return np.repeat(out[:, None, :], ny, axis=1).copy()


def droplet(rho_v, rho_l, nx: int, ny: int, R0: float, W: float = 4.0, h: float = 1.0,
            xc: float = None, yc: float = None) -> np.ndarray:
    """Eq. eqInit2D: rho_i = (rho_L + rho_V)/2 - (rho_L - rho_V)/2 tanh(2[sqrt((x-xc)^2 +
    (y-yc)^2/h^2) - R0]/W), centred at (nx/2, ny/2) unless given."""
    rho_v = np.asarray(rho_v, dtype=np.float64)
    rho_l = np.asarray(rho_l, dtype=np.float64)
    xc = nx / 2.0 if xc is None else xc
    yc = ny / 2.0 if yc is None else yc
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2 / (h * h))
    t = np.tanh(2.0 * (r - R0) / W)
    return 0.5 * (rho_l + rho_v)[:, None, None] - 0.5 * (rho_l - rho_v)[:, None, None] * t[None]
