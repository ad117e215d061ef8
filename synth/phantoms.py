"""Phantom coefficient fields xi(x) and seeded noise draws (no method arithmetic).

Grid placement matches the library's conventions: horizontal nodes
x_i = x0 + i L/N on a periodic box, X planes at cell midpoints
z'_l = z1 + (l + 1/2)(z2 - z1)/M.  Arrays are [M, N, N] = [z, y, x].
"""
from __future__ import annotations

import numpy as np


def grid_points(n, m, z1, z2, period=2.0, x0=-1.0):
    """(X, Y, Z) node coordinates, each [M, N, N]."""
    xs = x0 + period * np.arange(n) / n
    zs = z1 + (np.arange(m) + 0.5) * (z2 - z1) / m
    Z, Y, X = np.meshgrid(zs, xs, xs, indexing="ij")
    return X, Y, Z


def gaussian_inclusions(n, m, z1, z2, centres, sigmas, peaks, period=2.0, x0=-1.0):
    """xi = sum_j p_j exp(-|x - c_j|^2 / (2 sigma_j^2))."""
    X, Y, Z = grid_points(n, m, z1, z2, period, x0)
    xi = np.zeros_like(X)
    for (cx, cy, cz), s, p in zip(centres, sigmas, peaks):
        r2 = (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2
        xi += p * np.exp(-r2 / (2.0 * s * s))
    return xi


def random_gaussians(rng, n, m, z1, z2, count=3, width=(0.05, 0.2), peak=0.1,
                     period=2.0, x0=-1.0):
    """`count` Gaussians with centres uniform inside the X box (kept one width
    from the horizontal edges), widths U[width], peaks +-peak with random sign."""
    sig = rng.uniform(width[0], width[1], count)
    cx = rng.uniform(x0 + sig, x0 + period - sig)
    cy = rng.uniform(x0 + sig, x0 + period - sig)
    cz = rng.uniform(z1, z2, count)
    pk = peak * rng.choice([-1.0, 1.0], count)
    return gaussian_inclusions(n, m, z1, z2, list(zip(cx, cy, cz)), sig, pk, period, x0)


def sphere_phantom(rng, n, m, z1, z2, count=3, radii=(0.1, 0.3), contrast=(0.02, 0.15),
                   background=0.01, cutoff=0.2, period=2.0, x0=-1.0):
    """Piecewise-constant spheres plus a smooth random background: white
    N(0, background^2) noise low-pass filtered by a Gaussian of width `cutoff`
    (periodic in x, y), rescaled to standard deviation `background`."""
    X, Y, Z = grid_points(n, m, z1, z2, period, x0)
    xi = np.zeros_like(X)
    r = rng.uniform(radii[0], radii[1], count)
    cx = rng.uniform(x0 + r, x0 + period - r)
    cy = rng.uniform(x0 + r, x0 + period - r)
    cz = rng.uniform(z1, z2, count)
    cv = rng.uniform(contrast[0], contrast[1], count)
    for j in range(count):
        inside = (X - cx[j]) ** 2 + (Y - cy[j]) ** 2 + (Z - cz[j]) ** 2 <= r[j] ** 2
        xi[inside] = cv[j]
    if background > 0:
        h = period / n
        hz = (z2 - z1) / m
        white = rng.standard_normal(X.shape)
        fx = np.fft.fftfreq(n, d=h)
        fz = np.fft.fftfreq(m, d=hz)
        FZ, FY, FX = np.meshgrid(fz, fx, fx, indexing="ij")
        filt = np.exp(-2.0 * (np.pi * cutoff) ** 2 * (FX ** 2 + FY ** 2 + FZ ** 2))
        smooth = np.real(np.fft.ifftn(np.fft.fftn(white) * filt))
        sd = smooth.std()
        if sd > 0:
            xi += background * smooth / sd
    return xi


def noise_direction(rng, shape):
    """Complex noise draw with iid N(0,1) real and imaginary parts."""
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def three_bumps(n, m, z1, z2, period, x0, a0=0.3):
    """The model solution of Sec. 5: A0 [(1 - rho1^2/0.4^2)_+ + 2 (1 - rho2^2/0.25^2)_+
    + 2.5 (1 - rho3^2/0.3^2)_+] with
      rho1^2 = (x-1)^2 + (y-2)^2 + (z-0.5)^2,
      rho2^2 = (x-4)^2 + (y+3)^2 + (z-0.5)^2 + 1.5 (y+3)(z-0.5),
      rho3^2 = (x+3)^2 + y^2 + (z-0.45)^2 - 1.5 y (z-0.45)."""
    X, Y, Z = grid_points(n, m, z1, z2, period, x0)
    r1 = (X - 1) ** 2 + (Y - 2) ** 2 + (Z - 0.5) ** 2
    r2 = (X - 4) ** 2 + (Y + 3) ** 2 + (Z - 0.5) ** 2 + 1.5 * (Y + 3) * (Z - 0.5)
    r3 = (X + 3) ** 2 + Y ** 2 + (Z - 0.45) ** 2 - 1.5 * Y * (Z - 0.45)
    pos = lambda a: np.maximum(a, 0.0)
    return a0 * (pos(1 - r1 / 0.4 ** 2) + 2 * pos(1 - r2 / 0.25 ** 2) + 2.5 * pos(1 - r3 / 0.3 ** 2))
