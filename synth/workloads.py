"""Workload shapes: the five synthetic configurations the library is measured on.

Every workload uses the same physical box (units with c0 = 1): X = [-1,1]^2 x
[0.2, 1.0] and a data layer Y = [-1,1]^2 x [1.2, 1.6], with a plane incident
wave exp(-i k0 z).  Only grid sizes, frequencies, phantoms and noise differ.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .phantoms import gaussian_inclusions, random_gaussians, sphere_phantom

Z1, Z2, Z3, Z4 = 0.2, 1.0, 1.2, 1.6


@dataclass
class Workload:
    name: str
    n: int
    m: int
    m1: int
    omegas: np.ndarray
    deltas: tuple
    seed: int
    xi: np.ndarray = field(repr=False, default=None)
    z1: float = Z1
    z2: float = Z2
    z3: float = Z3
    z4: float = Z4

    @property
    def zy(self):
        if self.m1 == 1:
            return np.array([self.z3])
        return self.z3 + (self.z4 - self.z3) * np.arange(self.m1) / (self.m1 - 1)

    @property
    def voxel_freqs(self) -> int:
        return len(self.omegas) * self.n * self.n * self.m

    def noise(self, shape=None, stream=0):
        """Seeded complex Gaussian draw with the shape of W (n_omega, M1, N, N)."""
        rng = np.random.default_rng([self.seed, 1000 + stream])
        shape = shape or (len(self.omegas), self.m1, self.n, self.n)
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _c1():
    xi = gaussian_inclusions(32, 16, Z1, Z2, [(0.1, -0.2, 0.6)], [0.15], [0.05])
    return Workload("single-frequency 32x32x16, 8 data planes, k0=4pi, 1% noise",
                    32, 16, 8, np.array([4 * np.pi]), (0.01,), 0, xi)


def _c2():
    rng = np.random.default_rng(1)
    xi = random_gaussians(rng, 128, 64, Z1, Z2, 3, (0.05, 0.2), 0.1)
    return Workload("single-frequency 128x128x64, 32 data planes, k0=8pi, noise 0/1/5%",
                    128, 64, 32, np.array([8 * np.pi]), (0.0, 0.01, 0.05), 1, xi)


def _c3():
    rng = np.random.default_rng(2)
    om = np.sort(rng.uniform(2 * np.pi, 12 * np.pi, 8))
    xi = sphere_phantom(rng, 256, 64, Z1, Z2)
    return Workload("8 frequencies 256x256x64, 32 data planes, 1% noise",
                    256, 64, 32, om, (0.01,), 2, xi)


def _c5():
    rng = np.random.default_rng(4)
    xi = random_gaussians(rng, 128, 64, Z1, Z2, 3, (0.05, 0.2), 0.1)
    return Workload("4 frequencies 128x128x64, 32 data planes, 1% noise (derivatives)",
                    128, 64, 32, np.pi * np.array([4.0, 6.0, 8.0, 10.0]), (0.01,), 4, xi)


def batch_c4(count=64, seed=3):
    """64 independent problems of uneven size: grid from {64^2x16, 128^2x32,
    192^2x48, 256^2x64}, 1-8 frequencies U[2pi, 12pi], 4-32 data planes,
    random Gaussians, 1% noise; problem j draws from seed (seed, j)."""
    grids = [(64, 16), (128, 32), (192, 48), (256, 64)]
    out = []
    for j in range(count):
        rng = np.random.default_rng([seed, j])
        n, m = grids[rng.integers(0, 4)]
        n_om = int(rng.integers(1, 9))
        m1 = int(rng.integers(4, 33))
        om = np.sort(rng.uniform(2 * np.pi, 12 * np.pi, n_om))
        xi = random_gaussians(rng, n, m, Z1, Z2, 2, (0.05, 0.2), 0.1)
        out.append(Workload(f"batch problem {j}: {n}^2x{m}, {m1} planes, {n_om} freqs",
                            n, m, m1, om, (0.01,), 10_000 + j, xi))
    return out


WORKLOADS = {"c1": _c1, "c2": _c2, "c3": _c3, "c5": _c5}


def workload(name: str) -> Workload:
    return WORKLOADS[name]()
