"""Discrete conventions of the oracle.  Test infrastructure: see ``oracle/__init__``.

The paper (Sec. 5, 'finite-difference method on uniform grids') fixes only that X
and Y are flat layers discretised on uniform N x N x M and N x N x M1 grids, and
that the horizontal Fourier transforms are done by FFT.  The readings used here:

* Horizontal grid: periodic box [x0, x0+L) x [x0, x0+L), nodes x_i = x0 + i*h,
  h = L/N, identical for X and Y (Sec. 5, both layers share the N x N grid).
* X planes: cell midpoints z'_l = z1 + (l + 1/2) h_z, h_z = (z2 - z1)/M, so the
  quadrature coefficient mu_kl of Sec. 5.2 is the midpoint weight h_z.
* Y planes: given explicitly (host array), normally z3 + k (z4 - z3)/(M1 - 1).
* Wavenumbers: nu = 2 pi m / L with m the signed DFT index (NumPy fftfreq order);
  arrays are laid out [..., y, x], nu1 pairs with x (last axis), nu2 with y.
* k_z = sqrt(k0^2 - |nu|^2) on the branch Im k_z >= 0 (evanescent modes decay,
  Sec. 1 radiation condition with G = -exp(i k0 rho)/(4 pi rho)).
* Grazing modes |nu| = k0 exactly (k_z = 0, where the Weyl kernel is singular)
  are decided in exact integer arithmetic plus a relative 1e-9 margin and are
  excluded: the kernel is set to 0 there in every operator.
* Kernel: ``kernel="weyl"`` takes the exact horizontal transform of G (kernel.weyl);
  ``kernel="sampled"`` takes the DFT of G sampled on the grid, the way Sec. 5 builds
  G~ "from the known values of G using the FFT" (kernel.sampled_green).  The
  sampled kernel is finite at |nu| = k0, so it excludes no mode.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GRAZING_RTOL = 1e-9


@dataclass(frozen=True)
class Geometry:
    """Grid of one problem.  n: horizontal points per axis (N); m: X planes (M);
    [z1, z2]: X slab; zy: Y plane heights (M1 values, all > z2); period/x0:
    horizontal box [x0, x0+period)^2."""

    n: int
    m: int
    z1: float
    z2: float
    zy: tuple = field(default_factory=tuple)
    period: float = 2.0
    x0: float = -1.0
    kernel: str = "weyl"

    @property
    def m1(self) -> int:
        return len(self.zy)

    @property
    def h(self) -> float:
        return self.period / self.n

    @property
    def hz(self) -> float:
        return (self.z2 - self.z1) / self.m

    def x_nodes(self) -> np.ndarray:
        return self.x0 + self.h * np.arange(self.n)

    def zx(self) -> np.ndarray:
        """X plane heights z'_l (midpoints)."""
        return self.z1 + (np.arange(self.m) + 0.5) * self.hz

    def zy_arr(self) -> np.ndarray:
        return np.asarray(self.zy, dtype=np.float64)


def layer_planes(z3: float, z4: float, m1: int) -> tuple:
    """Y plane heights z_k = z3 + k (z4 - z3)/(M1 - 1), endpoints included."""
    if m1 == 1:
        return (float(z3),)
    return tuple(float(v) for v in z3 + (z4 - z3) * np.arange(m1) / (m1 - 1))


def mode_indices(n: int) -> np.ndarray:
    """Signed DFT indices m in fftfreq order (0, 1, ..., N/2-1, -N/2, ..., -1)."""
    return np.rint(np.fft.fftfreq(n) * n).astype(np.int64)


def wavenumbers(g: Geometry):
    """(nu1, nu2) on the [y, x] grid: nu1 varies along x, nu2 along y."""
    m = mode_indices(g.n).astype(np.float64) * (2.0 * np.pi / g.period)
    nu1 = np.broadcast_to(m[None, :], (g.n, g.n))
    nu2 = np.broadcast_to(m[:, None], (g.n, g.n))
    return nu1, nu2


def grazing_mask(k0: float, g: Geometry) -> np.ndarray:
    """True where |nu| = k0 (k_z = 0): m1^2 + m2^2 = (k0 L / 2 pi)^2 within 1e-9
    (Weyl kernel only: the sampled kernel has no singular mode)."""
    if g.kernel == "sampled":
        return np.zeros((g.n, g.n), dtype=bool)
    mi = mode_indices(g.n)
    msq = (mi[None, :] ** 2 + mi[:, None] ** 2).astype(np.float64)
    s2 = (k0 * g.period / (2.0 * np.pi)) ** 2
    return np.abs(msq - s2) <= GRAZING_RTOL * s2


def kz(k0, g: Geometry) -> np.ndarray:
    """k_z = sqrt(k0^2 - |nu|^2), principal root with Im k_z >= 0.

    For real k0 this is real and positive for |nu| < k0 and i*sqrt(|nu|^2 - k0^2)
    for |nu| > k0.  Complex k0 (a damped medium, used only by a test of the
    kernel) takes the root with non-negative imaginary part.
    """
    nu1, nu2 = wavenumbers(g)
    q = np.asarray(k0, dtype=np.complex128) ** 2 - (nu1 ** 2 + nu2 ** 2)
    r = np.sqrt(q.astype(np.complex128))
    return np.where(r.imag < 0, -r, r)
