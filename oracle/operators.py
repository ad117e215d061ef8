"""Discrete operators of eq. (5).  Test infrastructure: see ``oracle/__init__``.

With the horizontal transform read as the DFT on the periodic N x N grid and the
z-integral as the midpoint rule (mu = h_z, Sec. 5.2), the two integrals of eq. (5)
become, for every wavenumber nu, matrices acting on the z-profile of the field:

  data operator  (X -> Y):  A_nu[k, l] = h_z K_nu(z_k - z'_l)     (M1 x M)   eq. (5) third line / eq. (8)
  interior op.   (X -> X):  T_nu[l, l'] = h_z K_nu(z'_l - z'_l')  (M x M)    eq. (5) first line / eq. (9)

and in real space W = ifft2( A_nu fft2(w) ), with fft2 unnormalised and ifft2
carrying 1/N^2 (the factors h^2 of the forward transform and 1/L^2 of the inverse
cancel because h N = L).  Here w = omega^2 xi u is the unknown of eq. (3) times
omega^2 (the paper's v = xi u).  Grazing modes carry K = 0.

Two independent forms are given: the FFT form used by the oracle, and an explicit
dense assembly from DFT sums (no FFT) for tiny grids, which the tests compare.
"""
from __future__ import annotations

import functools

import numpy as np

from .grid import Geometry, grazing_mask, kz as kz_of, mode_indices
from .kernel import sampled_green, weyl

_CHUNK_ELEMS = 1 << 23  # bound on the size of a per-mode matrix batch


def fft2(a):
    return np.fft.fft2(a, axes=(-2, -1))


def ifft2(a):
    return np.fft.ifft2(a, axes=(-2, -1))


def _row_chunks(g: Geometry, per_mode: int):
    rows = max(1, min(g.n, _CHUNK_ELEMS // max(1, per_mode * g.n)))
    for r0 in range(0, g.n, rows):
        yield slice(r0, min(g.n, r0 + rows))


@functools.lru_cache(maxsize=8)
def _sampled_table(k0, g: Geometry, dz_key):
    """K~_nu(dz) of kernel.sampled_green for the distinct dz of an operator: [n_dz, N, N]."""
    return sampled_green(k0, g.n, g.period, np.array(dz_key), g.hz)


def mode_matrices(k0, g: Geometry, zrow, zcol, rows=slice(None), interior=False):
    """h_z K_nu(zrow[k] - zcol[l]) for the modes in `rows` of the [y, x] grid:
    array [y, x, k, l], zero on grazing modes.  With the sampled kernel
    (Geometry.kernel == "sampled") K is kernel.sampled_green; for the interior
    operator (interior=True, zrow = zcol = the X planes) the offsets are taken as
    |l - l'| h_z exactly, so that equal offsets share one sampled transform."""
    if g.kernel == "sampled":
        if interior:
            li = np.arange(len(zrow))
            dz = np.abs(li[:, None] - li[None, :]) * g.hz
        else:
            dz = np.asarray(zrow)[:, None] - np.asarray(zcol)[None, :]
        uniq, inv = np.unique(dz, return_inverse=True)
        tab = _sampled_table(complex(k0), g, tuple(uniq.tolist()))[:, rows]   # [n_dz, y, x]
        mat = g.hz * tab[inv.reshape(dz.shape)]                              # [k, l, y, x]
        return np.ascontiguousarray(np.moveaxis(mat, (0, 1), (-2, -1)))
    kz = kz_of(k0, g)[rows]
    graz = grazing_mask(np.real(k0), g)[rows] if np.isrealobj(k0) else np.zeros_like(kz, bool)
    kz_safe = np.where(graz, 1.0, kz)
    dz = np.asarray(zrow)[:, None] - np.asarray(zcol)[None, :]
    mat = g.hz * weyl(kz_safe[..., None, None], dz[None, None])
    mat[graz] = 0.0
    return mat


def data_matrices(k0, g: Geometry, rows=slice(None)):
    """A_nu (eq. 8): [y, x, M1, M]."""
    return mode_matrices(k0, g, g.zy_arr(), g.zx(), rows)


def interior_matrices(k0, g: Geometry, rows=slice(None)):
    """T_nu (eq. 9): [y, x, M, M]."""
    return mode_matrices(k0, g, g.zx(), g.zx(), rows, interior=True)


def _apply(build, nout, w, k0, g):
    wt = fft2(np.asarray(w, dtype=np.complex128))
    out = np.zeros((nout, g.n, g.n), dtype=np.complex128)
    for rows in _row_chunks(g, nout * wt.shape[0]):
        mat = build(k0, g, rows)
        out[:, rows, :] = np.einsum("yxkl,lyx->kyx", mat, wt[:, rows, :])
    return out


def apply_data(w, k0, g: Geometry):
    """W on Y from w on X: eq. (5) third line in real space, [M1, N, N]."""
    return ifft2(_apply(data_matrices, g.m1, w, k0, g))


def apply_interior(w, k0, g: Geometry):
    """(integral over X of G w) on X: eq. (5) first line without U0, [M, N, N]."""
    return ifft2(_apply(interior_matrices, g.m, w, k0, g))


def dense_operator_explicit(k0, g: Geometry, zrow):
    """Explicit matrix of w -> ifft2(h_z K fft2 w) onto planes `zrow`, assembled
    from DFT sums (no FFT): entry [(k,iy,ix), (l,jy,jx)] =
    (1/N^2) sum_{m1,m2} exp(2 pi i (m1 (ix-jx) + m2 (iy-jy))/N) h_z K_m(zrow_k - z'_l).
    Only for tiny grids (size (len(zrow) N^2) x (M N^2))."""
    n = g.n
    mi = mode_indices(n)
    idx = np.arange(n)
    # phase[m, i, j] = exp(2 pi i m (i - j)/N), summed mode by mode below
    ph = np.exp(2j * np.pi * mi[:, None, None] * (idx[None, :, None] - idx[None, None, :]) / n)
    same = np.array_equal(np.asarray(zrow), g.zx())
    kmat = mode_matrices(k0, g, np.asarray(zrow), g.zx(), interior=same)  # [m2, m1, k, l] in grid order
    nr, nc = len(zrow), g.m
    op = np.zeros((nr, n, n, nc, n, n), dtype=np.complex128)
    for a2 in range(n):          # mode along y (array axis 0 of kmat)
        for a1 in range(n):      # mode along x
            kk = kmat[a2, a1]    # [k, l]
            if not np.any(kk):
                continue
            # [iy, jy] x [ix, jx] phases
            sp = ph[a2][:, None, :, None] * ph[a1][None, :, None, :]   # [iy, ix, jy, jx]
            op += kk[:, None, None, :, None, None] * sp[None, :, :, None, :, :]
    return op.reshape(nr * n * n, nc * n * n) / (n * n)
