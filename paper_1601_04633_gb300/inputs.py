"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the oracle.

This module holds no arithmetic of the lattice Boltzmann method: it only draws
random numbers and lays out workload descriptions. Both sides receive its
output as plain arrays, so they see bit-identical inputs.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw q of stream ``seed`` is the SplitMix64 output function applied
to ``seed + (q + 1) * 0x9E3779B97F4A7C15``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` 64-bit outputs of stream ``seed`` starting at counter ``offset``."""
    with np.errstate(over="ignore"):
        q = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + q * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each draw."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_noise(seed: int, shape, amplitude: float) -> np.ndarray:
    """Uniform noise in [-amplitude, amplitude), row-major over ``shape``."""
    n = int(np.prod(shape))
    return (2.0 * uniform01(seed, n) - 1.0).reshape(shape) * amplitude


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform of pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


@dataclass
class Cavity:
    """One side-heated square-cavity problem as the paper states it (Sec. 2)."""
    nx: int
    ny: int
    Ra: float
    Pr: float
    alpha: float = 0.1
    theta_hot: float = 0.5
    theta_cold: float = -0.5
    theta_init: float = 0.0
    noise_amp: float = 1e-6
    seed: int = 1
    theta_hot_profile: np.ndarray | None = field(default=None, repr=False)

    def theta0(self) -> np.ndarray:
        """Initial temperature field (ny, nx): theta_init plus seeded uniform noise."""
        t = np.full((self.ny, self.nx), float(self.theta_init))
        if self.noise_amp:
            t = t + uniform_noise(self.seed, (self.ny, self.nx), self.noise_amp)
        return t


# Workloads shaped like the paper's Ra/Pr sweep (Table 1) at the sizes used here.
def cavity_64() -> Cavity:
    """64x64, Ra = 1e4, Pr = 0.01 (the paper's Case 1 parameters)."""
    return Cavity(64, 64, 1e4, 0.01, seed=1)


def cavity_256_oscillatory() -> Cavity:
    """256x256, Ra = 1e5, Pr = 0.005 (oscillatory regime)."""
    return Cavity(256, 256, 1e5, 0.005, seed=2)


def cavity_128_adjoint() -> Cavity:
    """128x128, Ra = 1e5, Pr = 0.01 with a perturbed hot-wall profile 0.5 + 0.01 N(0,1)."""
    c = Cavity(128, 128, 1e5, 0.01, seed=4)
    c.theta_hot_profile = 0.5 + 0.01 * normal(4, 128)
    return c


def cavity_4096() -> Cavity:
    """4096x4096, Ra = 1e7, Pr = 0.001 (the large single cavity)."""
    return Cavity(4096, 4096, 1e7, 0.001, seed=5)


def batch_sweep(n: int = 64, seed: int = 3) -> list[Cavity]:
    """``n`` independent cavities: side from {128,192,256,384}, log10 Ra ~ U[4,6],
    Pr from {0.001,0.005,0.01}, alpha = 0.1, each with its own noise seed."""
    sides = (128, 192, 256, 384)
    prs = (0.001, 0.005, 0.01)
    u = uniform01(seed, 3 * n).reshape(n, 3)
    out = []
    for k in range(n):
        side = sides[min(int(u[k, 0] * 4), 3)]
        Ra = 10.0 ** (4.0 + 2.0 * u[k, 1])
        Pr = prs[min(int(u[k, 2] * 3), 2)]
        out.append(Cavity(side, side, Ra, Pr, seed=1000 * seed + k))
    return out
