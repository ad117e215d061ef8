"""Workload shapes: the five synthetic configurations the library is measured on.

Every workload uses the same physical box (units with c0 = 1): X = [-1,1]^2 x
[0.2, 1.0] and a data layer Y = [-1,1]^2 x [1.2, 1.6], with a plane incident
wave exp(-i k0 z).  Only grid sizes, frequencies, phantoms and noise differ.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .phantoms import gaussian_inclusions, random_gaussians, sphere_phantom, three_bumps

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


@dataclass
class PaperWorkload:
    """The geometry of the paper's own experiments (Sec. 5): X = [-10,10]^2 x [-0.5,1.5] on
    an N x N x M grid, data in the thick layer [6.01, 6.5] (Sec. 5.3) or the thin layer
    [6.01, 6.02] (Sec. 5.4) on M1 planes, 11 point sources (0, y_s, 6), y_s = -5..5,
    a_s = 1, the three-bump xi with A0 = 0.3, frequencies omega = k0 in {1, 2, 3}
    (c0 = 1), noise levels 0, 1e-7, 1e-5."""
    name: str
    n: int = 128
    m: int = 71
    m1: int = 71
    layer: str = "thick"
    omegas: tuple = (1.0, 2.0, 3.0)
    deltas: tuple = (0.0, 1e-7, 1e-5)
    a0: float = 0.3
    period: float = 20.0
    x0: float = -10.0
    z1: float = -0.5
    z2: float = 1.5
    seed: int = 5

    @property
    def z3(self):
        return 6.01

    @property
    def z4(self):
        return 6.5 if self.layer == "thick" else 6.02

    @property
    def zy(self):
        if self.m1 == 1:
            return np.array([self.z3])
        return self.z3 + (self.z4 - self.z3) * np.arange(self.m1) / (self.m1 - 1)

    @property
    def sources(self):
        return [(0.0, float(y), 6.0, 1.0) for y in range(-5, 6)]

    @property
    def xi(self):
        return three_bumps(self.n, self.m, self.z1, self.z2, self.period, self.x0, self.a0)

    @property
    def voxel_freqs(self) -> int:
        return len(self.omegas) * self.n * self.n * self.m

    def noise(self, stream=0):
        rng = np.random.default_rng([self.seed, 2000 + stream])
        shape = (len(self.omegas), self.m1, self.n, self.n)
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def paper_workload(layer="thick", n=128, m=71, m1=None):
    """Sec. 5.3 (thick layer, M1 = M = 71) or Sec. 5.4 (thin layer, M1 = 2) at N = 128."""
    if m1 is None:
        m1 = 71 if layer == "thick" else 2
    return PaperWorkload(f"paper geometry, {layer} layer: {n}^2 x {m}, {m1} data planes, 11 point sources, "
                         f"three bumps A0 = 0.3, omega 1, 2, 3", n=n, m=m, m1=m1, layer=layer)
