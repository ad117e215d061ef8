"""Horizontal Fourier transform of the Green function.  Test infrastructure.

Sec. 1 defines G(rho) = -exp(i k0 rho)/(4 pi rho); Sec. 2 (eq. 5) needs its 2D
Fourier transform in (x, y) at fixed z - z'.  The paper obtains it by FFT of
sampled G (Sec. 5); the oracle uses the exact transform (Weyl's plane-wave
expansion of a spherical wave):

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
