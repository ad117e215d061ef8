"""Pins of the sampled-G kernel (Geometry.kernel = "sampled"): G~ computed from the
values of G by the FFT, the construction Sec. 5 describes.

  * the FFT form equals the explicit DFT double sum of the sampled G (no FFT);
  * with a damped wavenumber it converges to the exact transform (the Weyl form,
    itself pinned by a Hankel quadrature in test_oracle_kernel_ops) as the period
    grows -- a wrong normalisation, sign or offset convention fails this;
  * the self-cell term (the ball integral of G) equals a numerical quadrature and
    has the static limit -a^2/2;
  * the X -> Y and X -> X operators built on it equal a brute-force periodic
    convolution sum over the grid in real space;
  * A_nu is numerically full rank with rapidly decaying singular values (Sec. 6),
    and the discrepancy principle still holds at the chosen alpha.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import forward, inverse
from oracle.grid import Geometry, layer_planes, mode_indices
from oracle.kernel import green, sampled_green, self_cell, weyl
from oracle.operators import apply_data, apply_interior, data_matrices, fft2


def _offsets(n, h):
    i = np.arange(n)
    return np.where(i < n // 2, i, i - n) * h


def test_fft_form_equals_explicit_dft_sum():
    n, L, k0, hz = 8, 2.0, 3.7, 0.05
    h = L / n
    off = _offsets(n, h)
    m = mode_indices(n)
    nu = 2 * np.pi * m / L
    for dz in (0.0, 0.07, 0.4):
        got = sampled_green(k0, n, L, [dz], hz)[0]
        ref = np.zeros((n, n), complex)
        for a2 in range(n):          # nu2 (y)
            for a1 in range(n):      # nu1 (x)
                s = 0.0
                for j in range(n):
                    for i in range(n):
                        rho = np.sqrt(off[i] ** 2 + off[j] ** 2 + dz ** 2)
                        gv = self_cell(k0, h, hz) / hz if rho == 0 else h * h * green(k0, rho)
                        s += gv * np.exp(-1j * (nu[a1] * off[i] + nu[a2] * off[j]))
                ref[a2, a1] = s
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_converges_to_the_weyl_form_with_damping():
    k0, dz = 4 * np.pi * (1 + 0.3j), 0.5
    errs = []
    for L, n in ((4.0, 128), (8.0, 256), (16.0, 512)):
        K = sampled_green(k0, n, L, [dz])[0]
        nu1 = 2 * np.pi * mode_indices(n) / L
        nu = np.sqrt(nu1[None, :] ** 2 + nu1[:, None] ** 2)
        kz = np.sqrt(k0 ** 2 - nu ** 2 + 0j)
        kz = np.where(kz.imag < 0, -kz, kz)
        Kw = weyl(kz, dz)
        sel = nu <= 20
        errs.append(np.max(np.abs(K[sel] - Kw[sel])) / np.max(np.abs(Kw[sel])))
    # truncation to one period costs ~exp(-Im k0 L/2): 1e-3, 4e-7, 1e-13
    assert errs[2] <= 1e-12
    assert errs[0] > errs[1] > errs[2]


def test_self_cell_is_the_ball_integral():
    for k0 in (0.5, 4 * np.pi, 8 * np.pi):
        h, hz = 1 / 16, 0.05
        a = (3 * h * h * hz / (4 * np.pi)) ** (1 / 3)
        re = integrate.quad(lambda r: -r * np.cos(k0 * r), 0, a, epsabs=0, epsrel=1e-13)[0]
        im = integrate.quad(lambda r: -r * np.sin(k0 * r), 0, a, epsabs=0, epsrel=1e-13)[0]
        got = self_cell(k0, h, hz)
        assert abs(got - (re + 1j * im)) <= 1e-10 * abs(got)
    # static limit: -int_0^a rho d rho = -a^2/2
    h, hz = 1e-3, 1e-3
    a = (3 * h * h * hz / (4 * np.pi)) ** (1 / 3)
    assert abs(self_cell(1e-3, h, hz) / (-a * a / 2) - 1) <= 1e-6


def _brute_convolution(w, g, k0, zout, interior):
    """sum over the periodic grid and the X planes of h^2 h_z G(|x - x'|) w(x'), offsets
    taken in one period (the nearest image), the rho = 0 term by the cell integral."""
    n, h, hz = g.n, g.h, g.hz
    zx = g.zx()
    out = np.zeros((len(zout), n, n), complex)
    for k, z in enumerate(zout):
        for l in range(g.m):
            dz = abs(k - l) * hz if interior else z - zx[l]
            for jy in range(n):
                for ix in range(n):
                    s = 0.0
                    for jy2 in range(n):
                        dy = ((jy - jy2) % n)
                        dy = (dy if dy < n // 2 else dy - n) * h
                        for ix2 in range(n):
                            dx = ((ix - ix2) % n)
                            dx = (dx if dx < n // 2 else dx - n) * h
                            rho = np.sqrt(dx * dx + dy * dy + dz * dz)
                            kern = self_cell(k0, h, hz) if rho == 0 else h * h * hz * green(k0, rho)
                            s += kern * w[l, jy2, ix2]
                    out[k, jy, ix] += s
    return out


def test_operators_equal_brute_force_convolution():
    g = Geometry(6, 3, 0.2, 0.5, layer_planes(0.6, 0.7, 2), period=1.5, x0=-0.75, kernel="sampled")
    rng = np.random.default_rng(2)
    w = rng.standard_normal((g.m, g.n, g.n)) + 1j * rng.standard_normal((g.m, g.n, g.n))
    k0 = 5.0
    Wd = apply_data(w, k0, g)
    ref = _brute_convolution(w, g, k0, g.zy_arr(), interior=False)
    assert np.max(np.abs(Wd - ref)) <= 1e-12 * np.max(np.abs(ref))
    Ui = apply_interior(w, k0, g)
    refi = _brute_convolution(w, g, k0, g.zx(), interior=True)
    assert np.max(np.abs(Ui - refi)) <= 1e-12 * np.max(np.abs(refi))


@pytest.fixture(scope="module")
def sampled_case():
    g = Geometry(24, 8, 0.2, 1.0, layer_planes(1.2, 1.6, 6), kernel="sampled")
    rng = np.random.default_rng(24)
    from synth import random_gaussians
    xi = random_gaussians(rng, g.n, g.m, g.z1, g.z2, 2, (0.1, 0.25), 0.05)
    om = [3 * np.pi]
    W, _ = forward.make_data(xi, om, g, method="born")
    W = forward.add_noise(W, 0.01, np.random.default_rng(5).standard_normal(W.shape)
                          + 1j * np.random.default_rng(6).standard_normal(W.shape))
    return g, om, W


def test_sampled_matrices_are_full_rank_with_fast_decay(sampled_case):
    g, om, _ = sampled_case
    A = om[0] ** 2 * data_matrices(om[0], g)     # [y, x, M1, M]
    s = np.linalg.svd(A, compute_uv=False)
    ratio = s[..., 1] / s[..., 0]
    # not rank one (the Weyl kernel gives <= 1e-13), but the second singular value is
    # already small: the rapid decay Sec. 6 reports
    assert np.median(ratio) > 1e-10
    assert np.max(ratio) < 0.5
    assert np.all(np.diff(s, axis=-1) <= 0)


def test_discrepancy_holds_with_the_sampled_kernel(sampled_case):
    g, om, W = sampled_case
    res = inverse.reconstruct(W, om, g, 0.01)
    assert res.counts["grazing"] == 0
    A = om[0] ** 2 * data_matrices(om[0], g)
    Wt = fft2(W[0])
    b = np.moveaxis(Wt, 0, -1)
    v = np.moveaxis(res.Vt[0], 0, -1)
    r = np.linalg.norm(np.einsum("yxkl,yxl->yxk", A, v) - b, axis=-1)
    act = res.active[0]
    tr = np.sum(np.abs(A) ** 2, axis=(-2, -1))
    interior = act & (res.alpha[0] > 1.000001e-6 * tr)
    assert interior.sum() > 10
    assert np.allclose(r[interior], res.delta_nu[0], rtol=1e-9)
