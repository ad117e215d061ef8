"""Pins of the oracle's Algorithm 2 against facts fixed outside it.

* Rank-1 structure: with every data plane above X, K_nu(z_k - z'_l) factors as
  (-i/2k_z) e^{i k_z z_k} e^{-i k_z z'_l}, so A_nu = gamma a e^T exactly.  Then
  Tikhonov and the discrepancy root have closed forms, which the SVD-based
  oracle must reproduce (Sec. 4 comment b, Sec. 5.2).
* Discrepancy identity ||A V - b|| = delta_nu at the chosen alpha, monotonicity
  of phi, the push-through identity (primal == dual form).
* Step 2 (eq. 9): the explicit matrix product equals a zero-padded FFT
  convolution along z; given the generator's true V = xi u, steps 2-3 return the
  generator's u and the true xi.
* Step 3: one frequency == V/u; a duplicated frequency changes nothing; the
  combined xi is the real least-squares minimiser over frequencies.
* Exact recovery of a V in the row space of every A_nu (the normal solution).
"""
import numpy as np
import pytest

from oracle import forward, inverse
from oracle.grid import Geometry, grazing_mask, kz, layer_planes
from oracle.operators import data_matrices, fft2, ifft2, interior_matrices
from synth import workload


@pytest.fixture(scope="module")
def c1_case():
    w = workload("c1")
    g = Geometry(w.n, w.m, w.z1, w.z2, tuple(w.zy))
    W, u = forward.make_data(w.xi, w.omegas, g, method="gmres")
    Wd = forward.add_noise(W, 0.01, w.noise())
    return w, g, W, u, Wd


def _closed_form(A, b, delta_nu, k_z, om, g):
    """Rank-1 closed form of the Tikhonov/discrepancy solution of one mode."""
    zy, zx = g.zy_arr(), g.zx()
    gamma = om ** 2 * g.hz * (-1j / (2 * k_z))
    a = np.exp(1j * k_z * zy)
    e = np.exp(-1j * k_z * zx)
    s1sq = abs(gamma) ** 2 * np.vdot(a, a).real * np.vdot(e, e).real
    ahat = a / np.linalg.norm(a)
    proj = np.vdot(ahat, b)
    perp2 = np.vdot(b, b).real - abs(proj) ** 2
    t = np.sqrt(delta_nu ** 2 - perp2) / abs(proj)
    alpha = s1sq * t / (1 - t)
    V = np.conj(gamma) * np.vdot(a, b) / (s1sq + alpha) * np.conj(e)
    return V, alpha, s1sq


def test_data_matrix_is_rank_one(c1_case):
    w, g, *_ = c1_case
    A = data_matrices(w.omegas[0], g)
    s = np.linalg.svd(A, compute_uv=False)
    ok = s[..., 0] > 0
    assert np.all(s[..., 1][ok] <= 1e-13 * s[..., 0][ok])


def test_solve_matches_rank_one_closed_form(c1_case):
    w, g, W, u, Wd = c1_case
    om = w.omegas[0]
    opts = inverse.Options(tau=2.0)
    r = inverse.reconstruct(Wd, w.omegas, g, 0.01, opts=opts)
    A = om ** 2 * data_matrices(om, g)
    Wt = fft2(Wd[0])
    q = kz(om, g)
    iy, ix = np.nonzero(r.active[0])
    assert len(iy) > 20
    for a_, b_ in zip(iy, ix):
        V, alpha, s1 = _closed_form(A[a_, b_], Wt[:, a_, b_], r.delta_nu[0], q[a_, b_], om, g)
        assert abs(r.alpha[0, a_, b_] / alpha - 1) < 1e-9
        ref = r.Vt[0][:, a_, b_]
        assert np.linalg.norm(ref - V) <= 1e-12 * np.linalg.norm(V)


def test_discrepancy_holds_and_phi_monotone(c1_case):
    w, g, W, u, Wd = c1_case
    om = w.omegas[0]
    r = inverse.reconstruct(Wd, w.omegas, g, 0.01, opts=inverse.Options(tau=2.0))
    A = om ** 2 * data_matrices(om, g)
    Wt = fft2(Wd[0])
    iy, ix = np.nonzero(r.active[0])
    for a_, b_ in zip(iy, ix):
        Am, b = A[a_, b_], Wt[:, a_, b_]
        res = np.linalg.norm(Am @ r.Vt[0][:, a_, b_] - b)
        # the residual is formed by cancellation: its round-off is ~eps ||b||
        assert abs(res - r.delta_nu[0]) <= 1e-12 * r.delta_nu[0] + 1e-13 * np.linalg.norm(b)
        U, s, Vh = np.linalg.svd(Am, full_matrices=False)
        beta2 = np.abs(U.conj().T @ b) ** 2
        alphas = r.alpha[0, a_, b_] * np.logspace(-3, 3, 13)
        phi = [inverse.discrepancy_sq(al, s ** 2, beta2, 0.0) for al in alphas]
        assert np.all(np.diff(phi) > 0)
    # zeroed modes: ||b|| <= delta_nu
    zer = np.isinf(r.alpha[0])
    assert np.all(np.linalg.norm(Wt, axis=0)[zer] <= r.delta_nu[0])


def test_primal_equals_dual(c1_case):
    w, g, W, u, Wd = c1_case
    om = w.omegas[0]
    r = inverse.reconstruct(Wd, w.omegas, g, 0.01, opts=inverse.Options(tau=2.0))
    A = om ** 2 * data_matrices(om, g)
    Wt = fft2(Wd[0])
    iy, ix = np.nonzero(r.active[0])
    for a_, b_ in list(zip(iy, ix))[:30]:
        Am, b, al = A[a_, b_], Wt[:, a_, b_], r.alpha[0, a_, b_]
        primal = np.linalg.solve(Am.conj().T @ Am + al * np.eye(g.m), Am.conj().T @ b)
        dual = Am.conj().T @ np.linalg.solve(Am @ Am.conj().T + al * np.eye(g.m1), b)
        ref = r.Vt[0][:, a_, b_]
        assert np.linalg.norm(dual - ref) <= 1e-9 * np.linalg.norm(ref)
        assert np.linalg.norm(primal - ref) <= 1e-9 * np.linalg.norm(ref)


def test_interior_product_equals_zero_padded_fft_convolution():
    """T_nu V~ (explicit matrix) == linear convolution along z of V~ with the
    kernel samples h_z K(l h_z), |l| < M, done by FFT of length 2M."""
    g = Geometry(16, 12, 0.2, 1.0, layer_planes(1.2, 1.6, 4))
    om = 3 * np.pi
    rng = np.random.default_rng(5)
    Vt = rng.standard_normal((g.m, g.n, g.n)) + 1j * rng.standard_normal((g.m, g.n, g.n))
    Ut = inverse.interior_field(Vt, om, om, g) - fft2(forward.incident_plane_wave(om, g))
    q = kz(om, g)
    graz = grazing_mask(om, g)
    lags = np.arange(-(g.m - 1), g.m)
    ker = g.hz * (-1j * np.exp(1j * q[None] * np.abs(lags)[:, None, None] * g.hz)
                  / (2 * np.where(graz, 1.0, q))[None])
    ker[:, graz] = 0
    L = 2 * g.m
    kpad = np.zeros((L, g.n, g.n), complex)
    kpad[: g.m] = ker[g.m - 1:]          # lags 0..M-1
    kpad[L - (g.m - 1):] = ker[: g.m - 1]  # lags -(M-1)..-1
    vpad = np.zeros((L, g.n, g.n), complex)
    vpad[: g.m] = Vt
    conv = np.fft.ifft(np.fft.fft(kpad, axis=0) * np.fft.fft(vpad, axis=0), axis=0)[: g.m]
    ref = om ** 2 * conv
    assert np.linalg.norm(Ut - ref) / np.linalg.norm(ref) < 1e-13


def test_steps_2_3_exact_given_true_V(c1_case):
    """Given V = xi u from the forward solve, eq. (9) reproduces u and step 3
    returns xi_true on the support (paper, Sec. 4: scheme 1)-3) is exact)."""
    w, g, W, u, Wd = c1_case
    om = w.omegas[0]
    V = w.xi * u[0]
    Ut = inverse.interior_field(fft2(V), om, om, g)
    u_rec = ifft2(Ut)
    assert np.linalg.norm(u_rec - u[0]) / np.linalg.norm(u[0]) < 1e-11
    xi, c, ng, nn = inverse.combine(V[None], u_rec[None])
    assert np.max(np.abs(xi - w.xi)) < 1e-11 * np.max(np.abs(w.xi))
    assert ng == 0 and nn == 0
    assert np.allclose(c, 1 / np.sqrt(1 - w.xi), rtol=1e-11)


def test_combine_single_duplicate_and_least_squares():
    rng = np.random.default_rng(7)
    shp = (3, 4, 5)
    u = rng.standard_normal((3,) + shp) + 1j * rng.standard_normal((3,) + shp)
    V = rng.standard_normal((3,) + shp) + 1j * rng.standard_normal((3,) + shp)
    xi1, *_ = inverse.combine(V[:1], u[:1])
    assert np.allclose(xi1, np.real(V[0] / u[0]), rtol=1e-14, atol=0)
    xi2, *_ = inverse.combine(np.concatenate([V[:1], V[:1]]), np.concatenate([u[:1], u[:1]]))
    assert np.allclose(xi2, xi1, rtol=1e-14, atol=0)
    xi3, *_ = inverse.combine(V, u)
    f = lambda x: np.sum(np.abs(u * x - V) ** 2, axis=0)
    for eps in (1e-3, -1e-3):
        assert np.all(f(xi3 + eps) > f(xi3))


def test_combine_guards():
    u = np.array([[[1.0 + 0j, 1e-12]]])
    V = np.array([[[2.0 + 0j, 1.0]]])
    xi, c, ng, nn = inverse.combine(V, u, eps_u=1e-8, c0=1.0)
    assert xi[0, 0] == 2.0 and xi[0, 1] == 0.0 and ng == 1
    assert np.isnan(c[0, 0]) and nn == 1
    assert c[0, 1] == 1.0


def test_exact_recovery_in_row_space():
    """A V~ lying in the row space of every A_nu (V~_nu proportional to
    conj(e^{-i k_z z'})) is the normal solution of its own data and comes back
    to round-off with a negligible alpha (Sec. 4 comment b)."""
    g = Geometry(16, 12, 0.2, 1.0, layer_planes(1.2, 1.6, 6))
    om = 2 * np.pi
    rng = np.random.default_rng(11)
    q = kz(om, g)
    graz = grazing_mask(om, g)
    coef = (rng.standard_normal((g.n, g.n)) + 1j * rng.standard_normal((g.n, g.n)))
    prof = np.conj(np.exp(-1j * q[None] * g.zx()[:, None, None]))
    prof = prof / np.linalg.norm(prof, axis=0)
    Vt = coef[None] * prof
    Vt[:, graz] = 0
    A = om ** 2 * data_matrices(om, g)
    Wt = np.einsum("yxkl,lyx->kyx", A, Vt)
    W = ifft2(Wt)[None]
    opts = inverse.Options(tau=1.0, delta_floor=0.0, alpha_rel=1e-14)
    r = inverse.reconstruct(W, [om], g, 0.0, opts=opts)
    assert np.linalg.norm(r.Vt[0] - Vt) / np.linalg.norm(Vt) < 1e-11


def test_zero_data_gives_zero():
    g = Geometry(8, 4, 0.2, 1.0, layer_planes(1.2, 1.6, 2))
    W = np.zeros((1, 2, 8, 8), complex)
    r = inverse.reconstruct(W, [np.pi], g, 0.01)
    assert np.all(r.Vt == 0) and np.all(r.xi == 0)
    assert r.counts["zeroed"] == 64 - r.counts["grazing"]


def test_tsvd_filter_is_the_smallest_rank_meeting_the_discrepancy():
    """Brute force over ranks on random full-rank matrices: the truncated solution of
    the smallest rank whose explicit residual is within delta."""
    rng = np.random.default_rng(5)
    for trial in range(20):
        A = rng.standard_normal((5, 7)) + 1j * rng.standard_normal((5, 7))
        b = rng.standard_normal(5) + 1j * rng.standard_normal(5)
        U, s, Vh = np.linalg.svd(A, full_matrices=False)
        beta = U.conj().T @ b
        res = [np.linalg.norm(A @ (Vh[:r].conj().T @ (beta[:r] / s[:r])) - b) for r in range(0, 6)]
        delta = rng.uniform(0.1, 1.0) * res[0]
        f, r = inverse.tsvd_filter(s[None], np.abs(beta[None]) ** 2, np.array([np.linalg.norm(b) ** 2]),
                                   delta, 1e-8)
        r_brute = next((k for k in range(1, 6) if res[k] <= delta), 5)
        assert int(r[0]) == r_brute
        x = Vh.conj().T @ (f[0] * beta)
        x_brute = Vh[:r_brute].conj().T @ (beta[:r_brute] / s[:r_brute])
        assert np.allclose(x, x_brute, rtol=1e-12, atol=0)


def test_tsvd_on_the_rank_one_kernel_is_the_pseudo_inverse(c1_case):
    """Every A_nu is rank one, so TSVD keeps one singular value on every active mode:
    V~ = pinv(A_nu) b (the library pseudo-inverse at the same cutoff)."""
    w, g, W, u, Wd = c1_case
    res = inverse.reconstruct(Wd, w.omegas, g, 0.01, opts=inverse.Options(regularizer="tsvd"))
    om = w.omegas[0]
    A = om ** 2 * data_matrices(om, g)
    Wt = fft2(Wd[0])
    idx = np.argwhere(res.active[0])
    assert len(idx) > 10
    for (i2, i1) in idx[:: max(1, len(idx) // 12)]:
        ref = np.linalg.pinv(A[i2, i1], rcond=1e-8) @ Wt[:, i2, i1]
        assert np.allclose(res.Vt[0][:, i2, i1], ref, rtol=1e-12, atol=1e-12 * np.linalg.norm(ref))
    assert np.all(np.isfinite(res.xi))


def test_alpha_floor_branch_on_a_hand_built_rank_one_mode():
    """choose_alpha's floor branch: a mode A = gamma a e^T (the Weyl factorisation,
    written out by hand) whose data has a component outside the range of A larger
    than delta_nu, so phi(alpha) >= ||P_perp b|| > delta_nu for every alpha and the
    rule (Sec. 4 comment b with the alpha floor) must return
    alpha = alpha_rel ||A||_F^2 = alpha_rel |gamma|^2 ||a||^2 ||e||^2, flagged as floor."""
    rng = np.random.default_rng(3)
    m1, m, hz, kzv = 5, 9, 0.05, 3.0 + 0.0j
    zk = 1.2 + 0.1 * np.arange(m1)
    zl = 0.2 + (np.arange(m) + 0.5) * hz
    gamma = -1j * hz / (2 * kzv)
    a = np.exp(1j * kzv * zk)
    e = np.exp(-1j * kzv * zl)
    A = gamma * np.outer(a, e)
    # b = A x + r with r orthogonal to a (the range of A), ||r|| = 3 delta_nu
    x = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    r = rng.standard_normal(m1) + 1j * rng.standard_normal(m1)
    r -= a * (a.conj() @ r) / (a.conj() @ a)
    dnu = 0.1 * np.linalg.norm(A @ x)
    r *= 3 * dnu / np.linalg.norm(r)
    b = A @ x + r
    U, s, Vh = np.linalg.svd(A)
    beta = U.conj().T @ b
    bn = np.linalg.norm(b)
    perp2 = max(bn ** 2 - np.sum(np.abs(beta[:len(s)]) ** 2), 0.0)
    alpha, floor = inverse.choose_alpha(s[None] ** 2, np.abs(beta[None, :len(s)]) ** 2, np.array([perp2]),
                                        np.array([bn]), dnu, 1e-6)
    expect = 1e-6 * abs(gamma) ** 2 * np.linalg.norm(a) ** 2 * np.linalg.norm(e) ** 2
    assert bool(floor[0])
    assert abs(alpha[0] / expect - 1) <= 1e-12
    # the same mode with the out-of-range part below delta_nu has an interior root
    r2 = r * (0.5 * dnu / np.linalg.norm(r))
    b2 = A @ x + r2
    beta2 = U.conj().T @ b2
    bn2 = np.linalg.norm(b2)
    perp22 = max(bn2 ** 2 - np.sum(np.abs(beta2[:len(s)]) ** 2), 0.0)
    alpha2, floor2 = inverse.choose_alpha(s[None] ** 2, np.abs(beta2[None, :len(s)]) ** 2, np.array([perp22]),
                                          np.array([bn2]), dnu, 1e-6)
    assert not bool(floor2[0]) and alpha2[0] > expect
