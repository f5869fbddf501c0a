"""Seeded synthetic initial fields for the CTU lattice Boltzmann step.

This module is shared by the FP64 oracle tests and the CUDA path.  It holds
no arithmetic of the method itself: it only draws random numbers and lays
out initial density / velocity fields (rho, ux, uy) of the shapes the paper
runs.  Each side builds its own f = f^eq(rho, u) from these fields.

Random numbers: a splitmix64 counter generator (Steele, Lea & Flood, 2014,
"Fast splittable pseudorandom number generators") feeds the Box-Muller
transform in FP64.  Both are written out below so that the stream is fixed
by the seed alone, independent of numpy's generators.

Layout of every field: row-major [Ly][Lx], node (i, j) at x = i*ds, y = j*ds.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive outputs of splitmix64 started from state `seed` (uint64)."""
    idx = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in (0, 1]: the top 53 bits of splitmix64, plus one ulp."""
    z = splitmix64(seed, n)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal doubles from Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def noisy_uniform(Lx: int, Ly: int, rho0: float, amp: float, seed: int):
    """rho = rho0 * (1 + amp * N(0,1)), u = 0: the quiescent-liquid and the
    spinodal-decomposition starts (rho0 = a coexistence or the critical density)."""
    rho = rho0 * (1.0 + amp * normal(seed, Lx * Ly)).reshape(Ly, Lx)
    z = np.zeros((Ly, Lx))
    return rho, z.copy(), z.copy()


def bubble(Lx: int, Ly: int, rho_out: float, rho_in: float, R: float, W: float,
           cx: float | None = None, cy: float | None = None):
    """Circular vapour seed of radius R nodes and tanh interface width W nodes,
    centred at (Lx/2, Ly/2) unless given:
        rho(r) = (rho_out + rho_in)/2 + (rho_out - rho_in)/2 * tanh((r - R)/W).
    W = 0 gives the sharp interface (rho_in for r < R, else rho_out)."""
    cx = Lx / 2.0 if cx is None else cx
    cy = Ly / 2.0 if cy is None else cy
    j, i = np.mgrid[0:Ly, 0:Lx].astype(np.float64)
    r = np.hypot(i - cx, j - cy)
    if W > 0:
        rho = 0.5 * (rho_out + rho_in) + 0.5 * (rho_out - rho_in) * np.tanh((r - R) / W)
    else:
        rho = np.where(r < R, rho_in, rho_out)
    z = np.zeros((Ly, Lx))
    return rho, z.copy(), z.copy()


def linear_shear(Lx: int, Ly: int, u_w: float) -> np.ndarray:
    """ux(j) = -u_w + 2 u_w (j + 1)/(Ly + 1): the linear profile that reaches
    -u_w on row -1 and +u_w on row Ly, where the wall ghost rows sit."""
    j = np.arange(Ly, dtype=np.float64)
    ux = -u_w + 2.0 * u_w * (j + 1.0) / (Ly + 1.0)
    return np.repeat(ux[:, None], Lx, axis=1)


def shear_wave(Lx: int, Ly: int, ds: float, U: float, kx: float, ky: float, rho0: float = 1.0):
    """Shear wave u_perp = U cos(k.x), u_par = 0 on a uniform density rho0.
    The perpendicular direction is k rotated by +90 degrees."""
    j, i = np.mgrid[0:Ly, 0:Lx].astype(np.float64)
    phase = kx * i * ds + ky * j * ds
    kn = np.hypot(kx, ky)
    ex, ey = -ky / kn, kx / kn
    amp = U * np.cos(phase)
    return np.full((Ly, Lx), rho0), amp * ex, amp * ey


def fourier_mode(Lx: int, Ly: int, base: float, amp: float, mx: int, my: int) -> np.ndarray:
    """base + amp * cos(2 pi (mx i / Lx + my j / Ly)) on the node grid."""
    j, i = np.mgrid[0:Ly, 0:Lx].astype(np.float64)
    return base + amp * np.cos(2.0 * np.pi * (mx * i / Lx + my * j / Ly))


def random_f(Lx: int, Ly: int, base: np.ndarray, amp: float, seed: int) -> np.ndarray:
    """A generic distribution array f[16][Ly][Lx] = base[k] * (1 + amp*N(0,1)),
    for tests of the advection stencil on rough data."""
    z = normal(seed, 16 * Lx * Ly).reshape(16, Ly, Lx)
    return np.asarray(base, dtype=np.float64)[:, None, None] * (1.0 + amp * z)
