"""Pins of the oracle's derivatives of the fixed-alpha reconstruction.

* The JVP equals central finite differences of the oracle's forward map
  (h = 1e-6, FP64) along random complex directions of W and along log alpha.
* The VJP is the adjoint of the JVP: <J x, y> = <x, J^T y> (dot-product test),
  so with the finite-difference pin it is pinned too.
* Phi_omega equals the SVD closed form of the per-mode discrepancy
  (sum_j (alpha/(s_j^2+alpha))^2 |beta_j|^2 + ||P_perp b||^2, Sec. 4), reaches
  ||W~||^2 = N^2 ||W||^2 (Parseval) as alpha -> infinity and increases with alpha.
* The fixed-alpha forward map is the reconstruction of Algorithm 2 with the
  given alpha (the oracle's own reconstruct with alpha_given).
* The global-discrepancy log alpha found by bisection satisfies Phi = target.
"""
import numpy as np
import pytest

from oracle import adjoint, forward, inverse
from oracle.grid import Geometry
from synth import random_gaussians

FD_H = 1e-6


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(41)
    g = Geometry(12, 8, 0.2, 1.0, (1.2, 1.3, 1.45, 1.6))
    xi = random_gaussians(rng, g.n, g.m, 0.2, 1.0, 2, (0.15, 0.3), 0.1)
    om = np.array([4 * np.pi, 6 * np.pi])
    W, _ = forward.make_data(xi, om, g, method="gmres")
    Wd = forward.add_noise(W, 0.01, rng.standard_normal(W.shape) + 1j * rng.standard_normal(W.shape))
    # alpha a decade or two below the largest s^2 of each frequency
    la = []
    for o in om:
        s = np.linalg.svd(o ** 2 * adjoint.data_matrices(o, g), compute_uv=False)
        la.append(np.log(3e-2 * np.max(s[..., 0] ** 2)))
    return g, om, Wd, np.array(la), rng


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def test_forward_is_reconstruct_with_given_alpha(case):
    g, om, W, la, _ = case
    t = adjoint.forward(W, om, g, la)
    ref = inverse.reconstruct(W, om, g, 0.01, opts=inverse.Options(alpha_given=np.exp(la)))
    assert _rel(t.xi, ref.xi) < 1e-12


def test_phi_closed_form_and_limits(case):
    g, om, W, la, _ = case
    t = adjoint.forward(W, om, g, la)
    for j in range(len(om)):
        A, U, s, Vh, usable = t.svd[j]
        b = t.b[j]
        beta = np.einsum("yxkj,yxk->yxj", U.conj(), b)
        bb = np.sum(np.abs(b) ** 2, axis=-1)
        perp2 = np.maximum(bb - np.sum(np.abs(beta) ** 2, axis=-1), 0.0)
        phi2 = inverse.discrepancy_sq(np.full(bb.shape, t.alpha[j]), s ** 2, np.abs(beta) ** 2, perp2)
        closed = np.sum(np.where(usable, phi2, bb))
        assert abs(t.phi[j] - closed) <= 1e-12 * closed
    big = adjoint.forward(W, om, g, [60.0, 60.0]).phi
    parseval = np.array([g.n * g.n * np.linalg.norm(W[j]) ** 2 for j in range(len(om))])
    assert np.allclose(big, parseval, rtol=1e-12, atol=0)
    phis = [adjoint.forward(W, om, g, la + d).phi for d in (-4, -2, 0, 2, 4)]
    assert np.all(np.diff(np.array(phis), axis=0) > 0)


def test_jvp_matches_central_differences(case):
    g, om, W, la, rng = case
    t = adjoint.forward(W, om, g, la)
    for kind in ("re", "im", "alpha"):
        if kind == "alpha":
            dW = np.zeros_like(W)
            dla = rng.standard_normal(len(om))
        else:
            d = rng.standard_normal(W.shape) + 1j * rng.standard_normal(W.shape)
            d = d.real if kind == "re" else 1j * d.imag
            dW = d * np.linalg.norm(W) / np.linalg.norm(d)
            dla = np.zeros(len(om))
        dxi, dphi = adjoint.jvp(t, dW, dla)
        p = adjoint.forward(W + FD_H * dW, om, g, la + FD_H * dla)
        m = adjoint.forward(W - FD_H * dW, om, g, la - FD_H * dla)
        fd_xi = (p.xi - m.xi) / (2 * FD_H)
        fd_phi = (p.phi - m.phi) / (2 * FD_H)
        assert _rel(dxi, fd_xi) < 1e-6, kind
        assert _rel(dphi, fd_phi) < 1e-6, kind


def test_vjp_is_adjoint_of_jvp(case):
    g, om, W, la, rng = case
    t = adjoint.forward(W, om, g, la)
    dW = rng.standard_normal(W.shape) + 1j * rng.standard_normal(W.shape)
    dla = rng.standard_normal(len(om))
    gxi = rng.standard_normal(t.xi.shape)
    gphi = rng.standard_normal(len(om)) / np.abs(t.phi)
    dxi, dphi = adjoint.jvp(t, dW, dla)
    gW, gla = adjoint.vjp(t, gxi, gphi)
    lhs = np.sum(dxi * gxi) + np.sum(dphi * gphi)
    rhs = np.sum(np.real(np.conj(gW) * dW)) + np.sum(gla * dla)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.sum(np.abs(dxi * gxi)))


def test_global_discrepancy_root(case):
    g, om, W, _, _ = case
    target = adjoint.discrepancy_target(W, 0.01)
    la = adjoint.global_discrepancy_log_alpha(W, om, g, target)
    phi = adjoint.forward(W, om, g, la).phi
    assert np.allclose(phi, target, rtol=1e-9, atol=0)


def test_gauss_newton_tuning_reaches_the_global_discrepancy_root(case):
    """The host-side step rule of the alpha tuner, driven by the oracle's Phi and
    VJP, converges in 50 steps to the bisection root (1e-6 relative in alpha)."""
    from paper_1911_10487_gb300.diff import gauss_newton_step
    g, om, W, la0, _ = case
    target = adjoint.discrepancy_target(W, 0.01)
    root = adjoint.global_discrepancy_log_alpha(W, om, g, target)
    la = la0 + 6.0  # start far above the root
    for _ in range(50):
        t = adjoint.forward(W, om, g, la)
        r = t.phi / target - 1.0
        _, J = adjoint.vjp(t, np.zeros_like(t.xi), 1.0 / target)
        la = la + gauss_newton_step(r, J)
    assert np.all(np.abs(np.exp(la - root) - 1.0) < 1e-6)
