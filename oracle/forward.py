"""Forward data generator (the direct problem).  Test infrastructure.

Not part of the inverse method, but needed to make data W: given xi on X and the
incident field u0, solve the first equation of system (2) for u on X,

    u = u0 + omega^2 Int_X G (xi u)          (eq. 2, first line; eq. 5 first line),

then W = omega^2 Int_X G (xi u) on Y (eq. 2, second line; eq. 7).  Three
independent solvers of the same discrete equation are given so that the tests can
compare them:

* ``fixed_point`` -- Algorithm 1 (eq. 6): U_{n+1} = U0 + omega^2 T_nu F[xi F^-1 U_n]
  per mode, stopped when ||U_n - U_{n-1}|| <= 1e-13 ||U0|| (stop rule of Sec. 5.1);
* ``gmres``       -- Krylov solve of (I - omega^2 T diag(xi)) u = u0 to the same
  relative tolerance (for scatterers where Algorithm 1 does not contract, which
  the paper allows: it converges 'at least for small omega', Sec. 3);
* ``dense``       -- LU of the explicitly assembled matrix (tiny grids only).

``born`` skips the solve (u = u0): single scattering.
The incident field is the plane wave u0 = exp(-i k0 z) of the workloads, or the field
of point sources (``incident_point_sources``, Sec. 5) passed as u0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .grid import Geometry, grazing_mask, kz as kz_of, wavenumbers
from .kernel import weyl
from .operators import (apply_data, apply_interior, dense_operator_explicit, fft2,
                        ifft2, interior_matrices, _row_chunks)

STOP_RTOL = 1e-13  # Sec. 5.1 stop rule of Algorithm 1


def incident_plane_wave(k0, g: Geometry) -> np.ndarray:
    """u0 = exp(-i k0 z) on the X planes, [M, N, N]."""
    col = np.exp(-1j * k0 * g.zx())
    return np.broadcast_to(col[:, None, None], (g.m, g.n, g.n)).astype(np.complex128)


def incident_point_sources(k0, g: Geometry, sources) -> np.ndarray:
    """u0 = sum_s a_s G(|x - x_s|) on the X planes for point sources (x, y, z, a) above X
    (Sec. 5: f = sum_s a_s delta(x - x_s)), in the horizontally periodic model: the
    Fourier coefficient of the periodised field at nu is (1/L^2) K_nu(z - z_s) a_s
    exp(-i nu.r_s), so the DFT of its samples on the grid x0 + i h is
        U~0_nu(z) = (N^2/L^2) sum_s a_s K_nu(z - z_s) exp(-i nu.(r_s - x0))
    (the modes beyond the grid's band are negligible for sources well above X);
    u0 = ifft2(U~0).  Grazing modes carry K = 0, as in every operator.  [M, N, N]."""
    kz = kz_of(k0, g)
    graz = grazing_mask(np.real(k0), g) if np.isrealobj(k0) else np.zeros(kz.shape, bool)
    kz_safe = np.where(graz, 1.0, kz)
    nu1, nu2 = wavenumbers(g)
    zx = g.zx()
    Ut0 = np.zeros((g.m, g.n, g.n), dtype=np.complex128)
    for (xs, ys, zs, a) in sources:
        phase = np.exp(-1j * (nu1 * (xs - g.x0) + nu2 * (ys - g.x0)))
        K = weyl(kz_safe[None], (zx - zs)[:, None, None])     # [M, y, x]
        Ut0 += a * K * phase[None]
    Ut0[:, graz] = 0.0
    return ifft2((g.n * g.n) / g.period ** 2 * Ut0)


def _fixed_point(xi, k0, omega, g, u0, max_iter):
    """Algorithm 1, steps 2-3, written per mode in matrix form (Sec. 3)."""
    Ut0 = fft2(u0)
    Ut = Ut0.copy()
    nrm0 = np.linalg.norm(Ut0)
    for it in range(1, max_iter + 1):
        Vt = fft2(xi * ifft2(Ut))                      # F_r[xi F^-1 U_n]
        Un = np.empty_like(Ut)
        for rows in _row_chunks(g, g.m * g.m):
            T = interior_matrices(k0, g, rows)
            Un[:, rows, :] = Ut0[:, rows, :] + omega ** 2 * np.einsum(
                "yxkl,lyx->kyx", T, Vt[:, rows, :])
        diff = np.linalg.norm(Un - Ut)
        Ut = Un
        if diff <= STOP_RTOL * nrm0:
            return ifft2(Ut), it
        if not np.isfinite(diff) or diff > 1e30 * nrm0:
            break
    raise RuntimeError("Algorithm 1 did not converge (scatterer too strong for the fixed point)")


def _gmres(xi, k0, omega, g, u0):
    shape = u0.shape
    size = u0.size

    def mv(x):
        u = x.reshape(shape)
        return (u - omega ** 2 * apply_interior(xi * u, k0, g)).ravel()

    op = spla.LinearOperator((size, size), matvec=mv, dtype=np.complex128)
    sol, info = spla.gmres(op, u0.ravel(), rtol=STOP_RTOL, atol=0.0, restart=200, maxiter=50)
    if info != 0:
        raise RuntimeError(f"GMRES did not reach {STOP_RTOL} (info={info})")
    return sol.reshape(shape)


def _dense(xi, k0, omega, g, u0):
    T = dense_operator_explicit(k0, g, g.zx())
    L = np.eye(T.shape[0], dtype=np.complex128) - omega ** 2 * T * xi.ravel()[None, :]
    return np.linalg.solve(L, u0.ravel()).reshape(u0.shape)


def total_field(xi, omega, g: Geometry, c0=1.0, method="gmres", max_iter=500, u0=None):
    """u on X solving u = u0 + omega^2 T(xi u) (first line of eq. 2); u0 the plane wave
    unless given ([M, N, N] on X)."""
    k0 = omega / c0
    u0 = incident_plane_wave(k0, g) if u0 is None else np.asarray(u0, dtype=np.complex128)
    xi = np.asarray(xi, dtype=np.float64)
    if method == "born":
        return u0.copy()
    if method == "fixed_point":
        return _fixed_point(xi, k0, omega, g, u0, max_iter)[0]
    if method == "gmres":
        return _gmres(xi, k0, omega, g, u0)
    if method == "dense":
        return _dense(xi, k0, omega, g, u0)
    raise ValueError(method)


def fixed_point_iterations(xi, omega, g: Geometry, c0=1.0, max_iter=500):
    """(u, number of Algorithm-1 iterations) -- the quantity of Fig. 2."""
    k0 = omega / c0
    return _fixed_point(np.asarray(xi, np.float64), k0, omega, g, incident_plane_wave(k0, g), max_iter)


def scattered_data(xi, u, omega, g: Geometry, c0=1.0):
    """W = omega^2 Int_X G (xi u) on the Y planes (second line of eq. 2), [M1, N, N]."""
    return omega ** 2 * apply_data(np.asarray(xi) * u, omega / c0, g)


def make_data(xi, omegas, g: Geometry, c0=1.0, method="gmres", u0s=None):
    """Exact data W[n_omega, M1, N, N] and total fields u[n_omega, M, N, N]; u0s: the
    incident field per frequency ([n_omega, M, N, N]) or None for the plane wave."""
    Ws, us = [], []
    for j, om in enumerate(omegas):
        u = total_field(xi, om, g, c0, method, u0=None if u0s is None else u0s[j])
        us.append(u)
        Ws.append(scattered_data(xi, u, om, g, c0))
    return np.stack(Ws), np.stack(us)


def add_noise(W, delta, direction):
    """W^delta = W + delta ||W|| n/||n|| per frequency (Sec. 5.1): the perturbation
    has L2 norm exactly delta ||W||.  `direction` is the seeded complex Gaussian
    draw (same shape as W), generated outside the oracle."""
    W = np.asarray(W, dtype=np.complex128)
    out = np.empty_like(W)
    for j in range(W.shape[0]):
        n = direction[j]
        out[j] = W[j] + delta * np.linalg.norm(W[j]) * n / np.linalg.norm(n)
    return out
