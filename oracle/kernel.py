"""Horizontal Fourier transform of the Green function.  Test infrastructure.

Two forms, selected by ``Geometry.kernel``:

Sec. 1 defines G(rho) = -exp(i k0 rho)/(4 pi rho); Sec. 2 (eq. 5) needs its 2D
Fourier transform in (x, y) at fixed z - z'.  The paper obtains it by FFT of
sampled G (Sec. 5): ``sampled_green`` below.  The default is the exact transform
(Weyl's plane-wave expansion of a spherical wave):

    K_nu(dz) = -i exp(i k_z |dz|) / (2 k_z),   k_z = sqrt(k0^2 - |nu|^2), Im k_z >= 0.

It depends on nu only through |nu|, so the sign convention of the transform
(Sec. 2 prints exp(+i(Omega1 x + Omega1 y)), read as Omega2 y) does not matter.
The tests pin this formula against a direct numerical Hankel transform of G.
"""
from __future__ import annotations

import numpy as np


def weyl(kz, dz):
    """K_nu(dz) for arrays kz (complex) and dz (real), broadcast together."""
    kz = np.asarray(kz, dtype=np.complex128)
    return -1j * np.exp(1j * kz * np.abs(dz)) / (2.0 * kz)


def green(k0, rho):
    """G(rho) = -exp(i k0 rho) / (4 pi rho) (Sec. 1)."""
    return -np.exp(1j * k0 * rho) / (4.0 * np.pi * rho)


def self_cell(k0, h, hz):
    """Integral of G over one grid cell (h x h x hz), taken over the ball of the same
    volume, radius a = (3 h^2 hz / (4 pi))^(1/3), where G is integrable but cannot be
    sampled (rho = 0):
        int_{|x|<a} G dV = -int_0^a rho exp(i k0 rho) d rho = (1 - (1 - i k0 a) e^{i k0 a}) / k0^2.
    For |k0 a| <= 1 the difference cancels; there the same value is summed from its
    power series, (1 - (1 - i x) e^{i x}) / k0^2 = a^2 sum_{n>=2} (n-1) i^n x^(n-2) / n!
    with x = k0 a (the n = 2 term is the static value -a^2/2)."""
    a = (3.0 * h * h * hz / (4.0 * np.pi)) ** (1.0 / 3.0)
    x = k0 * a
    if abs(x) > 1.0:
        return (1.0 - (1.0 - 1j * x) * np.exp(1j * x)) / k0 ** 2
    s, fact = 0.0, 2.0
    for n in range(2, 40):
        s += (n - 1) * (1j ** n) * x ** (n - 2) / fact
        fact *= n + 1
    return a * a * s


def sampled_green(k0, n, period, dz, hz=None):
    """K~_nu(dz) for every wavenumber of the N x N grid and every dz (Sec. 5: the
    discrete analogue of G~ computed from the values of G by the FFT):

        K~_nu(dz) = h^2 sum_{i,j} G(sqrt(x_i^2 + y_j^2 + dz^2)) exp(-i (nu1 x_i + nu2 y_j)),

    over the offsets of the periodic cell, x_i = i h for i < N/2 and (i - N) h
    otherwise (the horizontal convolution with G restricted to one period, then
    periodised), h = L/N.  At dz = 0 the term rho = 0 is replaced by the cell integral
    of G divided by hz (``self_cell``), so that hz K~ carries the integral over the
    cell (hz: the X plane spacing; required when dz holds 0).
    Returns [len(dz), N, N] complex in the [y, x] fftfreq order of the grid."""
    h = period / n
    idx = np.arange(n)
    off = np.where(idx < n // 2, idx, idx - n) * h
    r2 = off[:, None] ** 2 + off[None, :] ** 2          # [y, x]
    dz = np.atleast_1d(np.asarray(dz, dtype=np.float64))
    out = np.empty((dz.size, n, n), dtype=np.complex128)
    for j, d in enumerate(dz):
        rho = np.sqrt(r2 + d * d)
        with np.errstate(divide="ignore", invalid="ignore"):
            gs = h * h * green(k0, rho)
        if d == 0.0:
            if hz is None:
                raise ValueError("dz = 0 needs the plane spacing hz for the self-cell term")
            gs[0, 0] = self_cell(k0, h, hz) / hz
        out[j] = np.fft.fft2(gs)
    return out
