"""Derivatives of the reconstruction at a fixed regularisation parameter per
frequency.  Test infrastructure: see ``oracle/__init__``.

The differentiated map is Algorithm 2 (Sec. 4) with Tikhonov's method at a given
alpha_omega (no discrepancy search), as a function of the data and of
log alpha_omega:

    (W, log alpha) -> (xi, Phi),

    W~ = F[W_omega],  b = W~_nu,  A = A_nu = U diag(s) V*        (eq. 8, SVD)
    V~ = V diag(f) U* b,  f_j = s_j / (s_j^2 + alpha)             (normal solution)
    U~ = U~0 + omega^2 T_nu V~                                    (eq. 9)
    V = F^-1[V~],  u = F^-1[U~]
    xi = Re(sum_omega conj(u) V) / D,  D = sum_omega |u|^2         (step 3)
    Phi_omega = sum_nu ||A V~ - b||^2                             (discrepancy)

Modes whose V~ is zero by rule (grazing, or a matrix that underflowed) keep
V~ = 0 and contribute ||b||^2 to Phi.  Where D < eps_u^2 n_omega, xi = 0 and its
derivative is 0 (the guard's mask is held fixed).

Gradients use the real-pair convention: for a real L and complex z,
grad z = dL/dRe z + i dL/dIm z, so that dL = Re sum conj(grad z) dz.

Every formula below comes from the SVD of A (the derivative of
f_j = s_j/(s_j^2 + alpha) in alpha is -s_j/(s_j^2 + alpha)^2); the GPU path uses a
Cholesky factor of A A* + alpha I instead, so the two share no algebra.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .forward import incident_plane_wave
from .grid import Geometry, grazing_mask
from .operators import data_matrices, fft2, ifft2, interior_matrices


@dataclass
class Tape:
    omegas: np.ndarray
    g: Geometry
    alpha: np.ndarray        # [n_omega]
    eps_u: float
    svd: list                # per omega: (A, U, s, Vh, usable)
    b: np.ndarray            # [n_omega, N, N, M1]  W~ per mode
    resid: np.ndarray        # [n_omega, N, N, M1]  A V~ - b
    V: np.ndarray            # [n_omega, M, N, N]
    u: np.ndarray            # [n_omega, M, N, N]
    xi: np.ndarray           # [M, N, N]
    D: np.ndarray            # [M, N, N]
    guard: np.ndarray        # [M, N, N] bool
    phi: np.ndarray          # [n_omega]


def _modes(omega, k0, g):
    A = omega ** 2 * data_matrices(k0, g)                 # [y, x, M1, M]
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    usable = ~grazing_mask(k0, g) & (np.sum(s ** 2, axis=-1) > 0)
    return A, U, s, Vh, usable


def _interior_T(k0, g):
    return interior_matrices(k0, g)                       # [y, x, M, M]


def forward(W, omegas, g: Geometry, log_alpha, c0=1.0, eps_u=1e-8) -> Tape:
    W = np.asarray(W, dtype=np.complex128)
    omegas = np.atleast_1d(np.asarray(omegas, dtype=np.float64))
    alpha = np.exp(np.atleast_1d(np.asarray(log_alpha, dtype=np.float64)))
    svd, bs, rs, Vs, us, phis = [], [], [], [], [], []
    for j, om in enumerate(omegas):
        k0 = om / c0
        A, U, s, Vh, usable = _modes(om, k0, g)
        b = np.moveaxis(fft2(W[j]), 0, -1)                 # [y, x, M1]
        beta = np.einsum("yxkj,yxk->yxj", U.conj(), b)
        f = np.where(usable[..., None], s / (s ** 2 + alpha[j]), 0.0)
        vt = np.einsum("yxjl,yxj->yxl", Vh.conj(), f * beta)
        r = np.einsum("yxkl,yxl->yxk", A, vt) - b
        Vt = np.moveaxis(vt, -1, 0)
        Ut = fft2(incident_plane_wave(k0, g)) + om ** 2 * np.einsum("yxkl,lyx->kyx", _interior_T(k0, g), Vt)
        svd.append((A, U, s, Vh, usable))
        bs.append(b)
        rs.append(r)
        Vs.append(ifft2(Vt))
        us.append(ifft2(Ut))
        phis.append(np.sum(np.abs(r) ** 2))
    V, u = np.stack(Vs), np.stack(us)
    D = np.sum(np.abs(u) ** 2, axis=0)
    guard = D < eps_u ** 2 * len(omegas)
    xi = np.where(guard, 0.0, np.sum(np.real(np.conj(u) * V), axis=0) / np.where(guard, 1.0, D))
    return Tape(omegas, g, alpha, eps_u, svd, np.stack(bs), np.stack(rs), V, u, xi, D, guard, np.array(phis))


def vjp(t: Tape, grad_xi, grad_phi=None, c0=1.0):
    """(grad W [n_omega, M1, N, N] complex, grad log alpha [n_omega]) for
    L = <grad_xi, xi> + <grad_phi, Phi>."""
    g = t.g
    N2 = g.n * g.n
    gphi = np.zeros(len(t.omegas)) if grad_phi is None else np.asarray(grad_phi, dtype=np.float64)
    gx = np.where(t.guard, 0.0, np.asarray(grad_xi, dtype=np.float64)) / np.where(t.guard, 1.0, t.D)
    gW = np.zeros((len(t.omegas), g.m1, g.n, g.n), dtype=np.complex128)
    gla = np.zeros(len(t.omegas))
    for j, om in enumerate(t.omegas):
        A, U, s, Vh, usable = t.svd[j]
        a = t.alpha[j]
        # step 3 -> V, u;  F^-1 adjoint = F / N^2
        Vbar = gx * t.u[j]
        ubar = gx * (t.V[j] - 2.0 * t.xi * t.u[j])
        Vtb = fft2(Vbar) / N2
        Utb = fft2(ubar) / N2
        # eq. (9) adjoint: V~bar += omega^2 T^H U~bar
        T = _interior_T(om / c0, g)
        tv = np.moveaxis(Vtb, 0, -1) + om ** 2 * np.einsum("yxkl,kyx->yxl", T.conj(), Utb)   # [y, x, M]
        f = np.where(usable[..., None], s / (s ** 2 + a), 0.0)
        df = np.where(usable[..., None], -s / (s ** 2 + a) ** 2, 0.0)      # d f / d alpha
        beta = np.einsum("yxkj,yxk->yxj", U.conj(), t.b[j])
        Vt_t = np.einsum("yxjl,yxl->yxj", Vh, tv)                          # V* t
        bbar = np.einsum("yxkj,yxj->yxk", U, f * Vt_t)
        dalpha = np.sum(np.real(np.conj(Vt_t) * df * beta))
        # Phi = ||r||^2, r = A V~ - b:  grad_b = 2 gphi (M^H A^H - I) r,  M = V diag(f) U*
        r = t.resid[j]
        AHr = np.einsum("yxkl,yxk->yxl", A.conj(), r)
        MH_AHr = np.einsum("yxkj,yxj->yxk", U, f * np.einsum("yxjl,yxl->yxj", Vh, AHr))
        bbar = bbar + 2.0 * gphi[j] * (MH_AHr - r)
        # d Phi / d alpha = 2 Re r^H A dV~/dalpha,  dV~/dalpha = V diag(df) U* b
        dVt = np.einsum("yxjl,yxj->yxl", Vh.conj(), df * beta)
        dalpha += 2.0 * gphi[j] * np.sum(np.real(np.conj(AHr) * dVt))
        gla[j] = a * dalpha
        gW[j] = N2 * ifft2(np.moveaxis(bbar, -1, 0))                     # F adjoint = N^2 F^-1
    return gW, gla


def jvp(t: Tape, dW, dlog_alpha=None, c0=1.0):
    """(d xi [M, N, N], d Phi [n_omega]) along (dW, d log alpha)."""
    g = t.g
    dla = np.zeros(len(t.omegas)) if dlog_alpha is None else np.asarray(dlog_alpha, dtype=np.float64)
    dW = np.asarray(dW, dtype=np.complex128)
    num = np.zeros((g.m, g.n, g.n))
    dD = np.zeros((g.m, g.n, g.n))
    dphi = np.zeros(len(t.omegas))
    for j, om in enumerate(t.omegas):
        A, U, s, Vh, usable = t.svd[j]
        a = t.alpha[j]
        db = np.moveaxis(fft2(dW[j]), 0, -1)
        f = np.where(usable[..., None], s / (s ** 2 + a), 0.0)
        df = np.where(usable[..., None], -s / (s ** 2 + a) ** 2, 0.0)
        beta = np.einsum("yxkj,yxk->yxj", U.conj(), t.b[j])
        dbeta = np.einsum("yxkj,yxk->yxj", U.conj(), db)
        dvt = np.einsum("yxjl,yxj->yxl", Vh.conj(), f * dbeta + a * dla[j] * df * beta)
        dr = np.einsum("yxkl,yxl->yxk", A, dvt) - db
        dphi[j] = 2.0 * np.sum(np.real(np.conj(t.resid[j]) * dr))
        dVt = np.moveaxis(dvt, -1, 0)
        dUt = om ** 2 * np.einsum("yxkl,lyx->kyx", _interior_T(om / c0, g), dVt)
        dV, du = ifft2(dVt), ifft2(dUt)
        num += np.real(np.conj(du) * t.V[j] + np.conj(t.u[j]) * dV)
        dD += 2.0 * np.real(np.conj(t.u[j]) * du)
    dxi = np.where(t.guard, 0.0, (num - t.xi * dD) / np.where(t.guard, 1.0, t.D))
    return dxi, dphi


def discrepancy_target(W, delta, tau=2.0, delta_floor=1e-5):
    """N^2 delta_nu^2 per frequency: the total of the per-mode noise bounds of
    Sec. 4 (delta_nu = tau max(delta, delta_floor) ||W_omega||, one per mode)."""
    W = np.asarray(W)
    n2 = W.shape[-1] * W.shape[-2]
    return np.array([n2 * (tau * max(delta, delta_floor) * np.linalg.norm(Wj)) ** 2 for Wj in W])


def global_discrepancy_log_alpha(W, omegas, g: Geometry, target, c0=1.0, lo=-60.0, hi=20.0, iters=80):
    """log alpha_omega with Phi_omega(alpha) = target_omega, by bisection (Phi is
    increasing in alpha: each mode's residual grows with alpha)."""
    omegas = np.atleast_1d(np.asarray(omegas, dtype=np.float64))
    out = np.zeros(len(omegas))
    for j in range(len(omegas)):
        a, b = lo, hi
        for _ in range(iters):
            mid = 0.5 * (a + b)
            phi = forward(W[j:j + 1], omegas[j:j + 1], g, [mid], c0).phi[0]
            if phi > target[j]:
                b = mid
            else:
                a = mid
        out[j] = 0.5 * (a + b)
    return out
