"""Pins of the oracle's kernel and discrete operators against facts fixed outside it.

* Weyl kernel (Sec. 2, eq. 5): direct numerical Hankel transform of
  G = -exp(i k0 rho)/(4 pi rho) (Sec. 1), with a slightly damped k0 so the
  integral converges absolutely.
* Midpoint quadrature in z (Sec. 5.2, mu = h_z): converges to the z-integral of
  eq. (5) computed by adaptive quadrature.
* FFT form of the operators == explicit DFT-sum assembly (no FFT) on tiny grids.
* Grazing modes, the k_z branch, mirror symmetry (the transform's sign is
  irrelevant, Sec. 2 typo reading).
"""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import operators
from oracle.grid import Geometry, grazing_mask, kz, layer_planes, wavenumbers
from oracle.kernel import weyl


def hankel_transform_G(k0, nu, z, R=120.0):
    """2 pi Int_0^R G(sqrt(rho^2+z^2)) J0(nu rho) rho d rho (the 2D Fourier
    transform of a radial function), by adaptive quadrature."""
    def f(rho, part):
        r = np.sqrt(rho * rho + z * z)
        val = -np.exp(1j * k0 * r) / (4 * np.pi * r) * special.j0(nu * rho) * rho * 2 * np.pi
        return val.real if part == 0 else val.imag
    kw = dict(limit=4000, epsabs=1e-13, epsrel=1e-11)
    return (integrate.quad(f, 0, R, args=(0,), **kw)[0]
            + 1j * integrate.quad(f, 0, R, args=(1,), **kw)[0])


@pytest.mark.parametrize("nu", [0.0, 5.0, 12.0, 20.0])
@pytest.mark.parametrize("z", [0.2, 0.5])
def test_weyl_matches_hankel_transform(nu, z):
    k0 = 4 * np.pi * (1 + 0.03j)
    q = np.sqrt(complex(k0 ** 2 - nu ** 2))
    q = q if q.imag >= 0 else -q
    ref = hankel_transform_G(k0, nu, z)
    got = weyl(q, z)
    assert abs(got - ref) / abs(ref) < 1e-8


def test_weyl_even_in_dz():
    q = np.array([3.0 + 0j, 0.0 + 4.0j])
    assert np.allclose(weyl(q, 0.3), weyl(q, -0.3), rtol=0, atol=0)


def _geom(n=8, m=8, m1=4):
    return Geometry(n, m, 0.2, 1.0, layer_planes(1.2, 1.6, m1))


def test_kz_branch_and_grazing_count():
    g = Geometry(32, 16, 0.2, 1.0, layer_planes(1.2, 1.6, 8))
    k0 = 4 * np.pi
    q = kz(k0, g)
    assert np.all(q.imag >= 0)
    nu1, nu2 = wavenumbers(g)
    prop = nu1 ** 2 + nu2 ** 2 < k0 ** 2
    assert np.all(q[prop].real > 0) and np.all(q[prop].imag == 0)
    assert np.all(q[~prop].real == 0)
    graz = grazing_mask(k0, g)
    # |m|^2 = (k0 L / 2 pi)^2 = 16 has the four integer solutions (+-4, 0), (0, +-4)
    assert graz.sum() == 4
    # propagating (|m| < 4) modes of a disc of radius 4: 45 lattice points
    assert int(np.sum(prop & ~graz)) == 45


def test_fft2_is_unnormalised_dft():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6))
    j = np.arange(6)
    F = np.exp(-2j * np.pi * np.outer(j, j) / 6)
    assert np.allclose(operators.fft2(a), F @ a @ F.T, rtol=0, atol=1e-12)


@pytest.mark.parametrize("k0", [4 * np.pi, 2.5])
def test_data_operator_fft_equals_explicit_dft_sums(k0):
    g = _geom()
    rng = np.random.default_rng(1)
    w = rng.standard_normal((g.m, g.n, g.n)) + 1j * rng.standard_normal((g.m, g.n, g.n))
    D = operators.dense_operator_explicit(k0, g, g.zy_arr())
    ref = (D @ w.ravel()).reshape(g.m1, g.n, g.n)
    got = operators.apply_data(w, k0, g)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


def test_interior_operator_fft_equals_explicit_dft_sums():
    g = _geom()
    k0 = 3.7
    rng = np.random.default_rng(2)
    w = rng.standard_normal((g.m, g.n, g.n)) + 1j * rng.standard_normal((g.m, g.n, g.n))
    D = operators.dense_operator_explicit(k0, g, g.zx())
    ref = (D @ w.ravel()).reshape(g.m, g.n, g.n)
    got = operators.apply_interior(w, k0, g)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


def test_operator_commutes_with_mirror():
    """K depends on |nu| only, so the operator commutes with x -> -x (on the
    periodic grid: index i -> -i mod N); the sign of the transform is irrelevant."""
    g = Geometry(16, 6, 0.2, 1.0, layer_planes(1.2, 1.6, 3))
    rng = np.random.default_rng(3)
    w = rng.standard_normal((g.m, g.n, g.n)) + 1j * rng.standard_normal((g.m, g.n, g.n))
    mir = lambda a: np.roll(a[..., ::-1], 1, axis=-1)
    k0 = 2 * np.pi
    a = mir(operators.apply_data(w, k0, g))
    b = operators.apply_data(mir(w), k0, g)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-13


def test_midpoint_rule_converges_to_z_integral():
    """For one mode and a smooth profile f(z'), sum_l h_z K(z_k - z'_l) f(z'_l)
    approaches Int_{z1}^{z2} K(z_k - z') f(z') dz' at the O(h_z^2) rate."""
    z1, z2, zk = 0.2, 1.0, 1.3
    q = 5.0 + 0j
    f = lambda z: np.cos(3 * z) + 0.5 * z
    fun = lambda z, p: (weyl(q, zk - z) * f(z)).real if p == 0 else (weyl(q, zk - z) * f(z)).imag
    ref = integrate.quad(fun, z1, z2, args=(0,))[0] + 1j * integrate.quad(fun, z1, z2, args=(1,))[0]
    errs = []
    for m in (20, 40, 80):
        g = Geometry(4, m, z1, z2, (zk,))
        zx = g.zx()
        errs.append(abs(np.sum(g.hz * weyl(q, zk - zx) * f(zx)) - ref))
    assert errs[2] < 1e-4 * abs(ref)
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5
