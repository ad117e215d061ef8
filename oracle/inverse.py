"""Algorithm 2 (the inverse problem).  Test infrastructure: see ``oracle/__init__``.

Steps, in the paper's order (Sec. 4, Algorithm 2; Sec. 5.2):

1. W~ = F_r[W] on every Y plane (2D FFT).  For every wavenumber nu the discretised
   first-kind equation (8) is the SLAE  A_nu V~_nu = W~_nu  with
   A_nu[k, l] = omega^2 h_z K_nu(z_k - z'_l)  (M1 x M).  It is solved by a
   regularising algorithm giving the normal solution (Sec. 4 comment b):
   Tikhonov, V~ = (A*A + alpha I)^-1 A* b, written through the SVD
   A = U S V*:  V~ = V diag(s/(s^2 + alpha)) U* b.
   alpha is chosen per mode by the discrepancy principle ||A V~ - b|| = delta_nu,
   delta_nu = tau * max(delta, delta_floor) * ||W^delta_omega||_2 (the expected
   noise norm on one mode of the unnormalised DFT, by Parseval), with
     ||b|| <= delta_nu            -> V~ = 0  (alpha = infinity),
     phi(alpha_floor) >= delta_nu -> alpha = alpha_floor = alpha_rel * ||A||_F^2,
     otherwise the root of phi(alpha) = delta_nu, found by bisection in log(alpha).
   phi^2(alpha) = sum_j (alpha/(s_j^2+alpha))^2 |(U* b)_j|^2 + ||b - U U* b||^2.
   Option: truncated SVD instead of Tikhonov (the regularising algorithm Sec. 5
   reports as the best), V~ = sum_{j<r} (U* b)_j / s_j v_j with the truncation
   rank r chosen by the same discrepancy principle (`tsvd_filter`).
2. U~ = U~0 + omega^2 T_nu V~ with T_nu[l, l'] = h_z K_nu(z'_l - z'_l') (eq. 9),
   an explicit M x M matrix-vector product per mode (Sec. 5.2: 'matrix
   multiplication'); then V = F^-1[V~], u = F^-1[U~] on X.
3. xi from u xi = V: one frequency, xi = Re(V/u); several, the least-squares
   solution over omega, xi = Re(sum conj(u) V) / sum |u|^2 (Sec. 4 step 3,
   Sec. 5.2).  c = (c0^-2 - xi)^(-1/2) (Sec. 1, xi = c0^-2 - c^-2), NaN where
   xi >= c0^-2.  Where |u| is below eps_u (relative to the unit incident
   amplitude) xi is set to 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .forward import incident_plane_wave
from .grid import Geometry, grazing_mask
from .operators import data_matrices, fft2, ifft2, interior_matrices, _row_chunks

BISECT_ITERS = 200


@dataclass
class Options:
    tau: float = 2.0            # discrepancy safety factor (delta_nu is a high-probability bound)
    delta_floor: float = 1e-5   # delta_eff = max(delta, delta_floor)
    alpha_rel: float = 1e-6     # alpha_floor = alpha_rel * ||A_nu||_F^2
    eps_u: float = 1e-8         # |u| guard for step 3
    alpha_given: object = None  # per-frequency alpha (skips the discrepancy search)
    mode_rows: object = None    # (r0, r1): solve only wavenumber rows r0 <= row < r1, treating the
                                # others as zeroed -- a proportional work sample, for timing only
    regularizer: str = "tikhonov"  # or "tsvd": truncated SVD, rank by the discrepancy principle
    tsvd_rcut: float = 1e-8     # TSVD: singular values below tsvd_rcut * s_1 count as zero


@dataclass
class Result:
    xi: np.ndarray                      # [M, N, N] float64
    c: np.ndarray                       # [M, N, N] float64
    V: np.ndarray                       # [n_omega, M, N, N] complex
    u: np.ndarray                       # [n_omega, M, N, N] complex
    Vt: np.ndarray                      # [n_omega, M, N, N] mode space
    Ut: np.ndarray                      # [n_omega, M, N, N] mode space
    alpha: np.ndarray                   # [n_omega, N, N]; inf where inactive, nan grazing
    active: np.ndarray                  # [n_omega, N, N] bool
    delta_nu: np.ndarray                # [n_omega]
    counts: dict = field(default_factory=dict)


def discrepancy_sq(alpha, s2, beta2, perp2):
    """phi^2(alpha) for arrays broadcast over modes: s2 = s_j^2, beta2 = |U*b|_j^2."""
    a = np.asarray(alpha)[..., None]
    return np.sum((a / (s2 + a)) ** 2 * beta2, axis=-1) + perp2


def choose_alpha(s2, beta2, perp2, bnorm, delta_nu, alpha_rel):
    """Discrepancy-principle alpha for a batch of modes (all with ||b|| > delta_nu)."""
    tr = np.sum(s2, axis=-1)
    a_lo = alpha_rel * tr
    target = delta_nu ** 2
    floor_case = discrepancy_sq(a_lo, s2, beta2, perp2) >= target
    a_hi = np.maximum(tr * delta_nu / (bnorm - delta_nu), a_lo)
    lo, hi = np.log(a_lo), np.log(a_hi)
    for _ in range(BISECT_ITERS):
        mid = 0.5 * (lo + hi)
        above = discrepancy_sq(np.exp(mid), s2, beta2, perp2) >= target
        hi = np.where(above, mid, hi)
        lo = np.where(above, lo, mid)
    alpha = np.exp(0.5 * (lo + hi))
    return np.where(floor_case, a_lo, alpha), floor_case


def tsvd_filter(s, beta2, bnorm2, delta_nu, rcut):
    """Truncated SVD (Sec. 4, the regularising algorithm the paper found best): the
    filter 1/s_j for j < r and 0 beyond, r the smallest rank whose residual
    ||b||^2 - sum_{j<r} |beta_j|^2 is within delta_nu^2 (the discrepancy principle),
    counting only singular values above rcut s_1; the numerical rank if no rank is
    enough.  Returns (filter [..., K], r [...])."""
    num = s > rcut * s[..., :1]
    cum = np.cumsum(np.where(num, beta2, 0.0), axis=-1)
    ok = ((bnorm2[..., None] - cum) <= delta_nu ** 2) & num
    r = np.where(ok.any(axis=-1), ok.argmax(axis=-1) + 1, num.sum(axis=-1))
    j = np.arange(s.shape[-1])
    return np.where(j < r[..., None], 1.0 / np.where(num, s, 1.0), 0.0), r


def solve_modes(Wt, omega, k0, g: Geometry, delta_nu, opts: Options, alpha_fixed=None):
    """Step 1 for one frequency: V~[M, N, N] from W~[M1, N, N]; alpha[N, N]; active."""
    Vt = np.zeros((g.m, g.n, g.n), dtype=np.complex128)
    alpha = np.full((g.n, g.n), np.inf)
    graz = grazing_mask(k0, g)
    alpha[graz] = np.nan
    n_floor = 0
    for rows in _band(_row_chunks(g, g.m1 * g.m * 4), opts.mode_rows):
        A = omega ** 2 * data_matrices(k0, g, rows)           # [y, x, M1, M]
        b = np.moveaxis(Wt[:, rows, :], 0, -1)                 # [y, x, M1]
        bnorm = np.linalg.norm(b, axis=-1)
        U, s, Vh = np.linalg.svd(A, full_matrices=False)
        beta = np.einsum("yxkj,yxk->yxj", U.conj(), b)
        # ||P_perp b||^2 of phi^2, as the norm of the projection residual b - U U* b
        # itself: the difference of squares ||b||^2 - ||U* b||^2 would leave a rounding
        # error of order eps ||b||^2 in phi^2, which decides alpha once delta_nu^2 is
        # not far above it (the tiny noise levels of Sec. 5.3)
        perp2 = np.sum(np.abs(b - np.einsum("yxkj,yxj->yxk", U, beta)) ** 2, axis=-1)
        s2 = s ** 2
        # a mode whose matrix underflowed to zero carries no information: V~ = 0
        usable = ~graz[rows] & (np.sum(s ** 2, axis=-1) > 0)
        act = (bnorm > delta_nu) & usable
        if alpha_fixed is not None:
            act = usable
        a = np.full(bnorm.shape, np.inf)
        if opts.regularizer == "tsvd":
            f, _ = tsvd_filter(s, np.abs(beta) ** 2, bnorm ** 2, delta_nu, opts.tsvd_rcut)
            filt = np.where(act[..., None], f, 0.0)
            vt = np.einsum("yxjl,yxj->yxl", Vh.conj(), filt * beta)
            Vt[:, rows, :] = np.moveaxis(vt, -1, 0)
            sub = alpha[rows]
            sub[act] = 0.0  # no Tikhonov parameter: recorded as 0 on active modes
            alpha[rows] = sub
            continue
        if np.any(act):
            if alpha_fixed is not None:
                a[act] = alpha_fixed
            else:
                a[act], fl = choose_alpha(s2[act], np.abs(beta[act]) ** 2, perp2[act],
                                          bnorm[act], delta_nu, opts.alpha_rel)
                n_floor += int(np.sum(fl))
        filt = np.where(act[..., None], s / (s2 + np.where(act, a, 1.0)[..., None]), 0.0)
        vt = np.einsum("yxjl,yxj->yxl", Vh.conj(), filt * beta)
        Vt[:, rows, :] = np.moveaxis(vt, -1, 0)
        sub = alpha[rows]
        sub[act] = a[act]
        alpha[rows] = sub
    active = np.isfinite(alpha)
    return Vt, alpha, active, n_floor


def _band(chunks, band):
    for rows in chunks:
        if band is not None:
            rows = slice(max(rows.start, band[0]), min(rows.stop, band[1]))
            if rows.start >= rows.stop:
                continue
        yield rows


def interior_field(Vt, omega, k0, g: Geometry, band=None, u0=None):
    """Step 2 (eq. 9): U~ = U~0 + omega^2 T_nu V~ per mode, explicit matrix product;
    U~0 = F[u0], u0 the plane wave unless given."""
    Ut = fft2(incident_plane_wave(k0, g) if u0 is None else np.asarray(u0, dtype=np.complex128))
    for rows in _band(_row_chunks(g, g.m * g.m), band):
        T = interior_matrices(k0, g, rows)
        Ut[:, rows, :] += omega ** 2 * np.einsum("yxkl,lyx->kyx", T, Vt[:, rows, :])
    return Ut


def combine(V, u, eps_u=1e-8, c0=1.0):
    """Step 3: xi from u xi = V (least squares over frequencies), and c."""
    num = np.sum(np.real(np.conj(u) * V), axis=0)
    den = np.sum(np.abs(u) ** 2, axis=0)
    guard = den < eps_u ** 2 * u.shape[0]
    xi = np.where(guard, 0.0, num / np.where(guard, 1.0, den))
    ok = xi < c0 ** -2
    c = np.where(ok, 1.0 / np.sqrt(np.where(ok, c0 ** -2 - xi, 1.0)), np.nan)
    return xi, c, int(np.sum(guard)), int(np.sum(~ok))


def reconstruct(W, omegas, g: Geometry, delta, c0=1.0, opts: Options | None = None, u0s=None) -> Result:
    """Algorithm 2 on data W[n_omega, M1, N, N] at frequencies `omegas`; u0s: the incident
    field on X per frequency ([n_omega, M, N, N]), None for the plane wave."""
    opts = opts or Options()
    W = np.asarray(W, dtype=np.complex128)
    omegas = np.atleast_1d(np.asarray(omegas, dtype=np.float64))
    if W.shape != (len(omegas), g.m1, g.n, g.n):
        raise ValueError(f"W shape {W.shape} does not match geometry")
    Vs, us, Vts, Uts, alphas, acts, dnus = [], [], [], [], [], [], []
    counts = {"zeroed": 0, "grazing": 0, "alpha_floor": 0}
    for j, om in enumerate(omegas):
        k0 = om / c0
        Wt = fft2(W[j])
        dnu = opts.tau * max(delta, opts.delta_floor) * np.linalg.norm(W[j])
        afix = None if opts.alpha_given is None else float(np.atleast_1d(opts.alpha_given)[j])
        Vt, alpha, active, nfl = solve_modes(Wt, om, k0, g, dnu, opts, afix)
        Ut = interior_field(Vt, om, k0, g, opts.mode_rows, None if u0s is None else u0s[j])
        Vs.append(ifft2(Vt))
        us.append(ifft2(Ut))
        Vts.append(Vt)
        Uts.append(Ut)
        alphas.append(alpha)
        acts.append(active)
        dnus.append(dnu)
        counts["grazing"] += int(np.sum(np.isnan(alpha)))
        counts["zeroed"] += int(np.sum(np.isinf(alpha)))
        counts["alpha_floor"] += nfl
    V, u = np.stack(Vs), np.stack(us)
    xi, c, n_guard, n_nan = combine(V, u, opts.eps_u, c0)
    counts["u_guard"] = n_guard
    counts["nan_c"] = n_nan
    return Result(xi=xi, c=c, V=V, u=u, Vt=np.stack(Vts), Ut=np.stack(Uts),
                  alpha=np.stack(alphas), active=np.stack(acts),
                  delta_nu=np.array(dnus), counts=counts)
