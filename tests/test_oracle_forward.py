"""Pins of the forward data generator and the noise model.

* Three independent solvers of the discrete first line of eq. (2) agree: dense LU
  of the explicitly assembled matrix (DFT sums, no FFT), GMRES with the FFT
  operator, and Algorithm 1 (eq. 6) with the Sec. 5.1 stop rule.
* Born limit: as xi -> 0, W / xi is linear (W(t xi)/t -> the Born data).
* Noise (Sec. 5.1): ||W^delta - W|| = delta ||W|| exactly, reproducible from the seed.
"""
import numpy as np
import pytest

from oracle import forward
from oracle.grid import Geometry, layer_planes
from synth import gaussian_inclusions, workload


def _tiny():
    g = Geometry(8, 8, 0.2, 1.0, layer_planes(1.2, 1.6, 4))
    xi = gaussian_inclusions(8, 8, 0.2, 1.0, [(0.1, -0.2, 0.6)], [0.3], [0.02])
    return g, xi


def test_three_solvers_agree_on_8cubed():
    g, xi = _tiny()
    om = 2 * np.pi
    ud = forward.total_field(xi, om, g, method="dense")
    ug = forward.total_field(xi, om, g, method="gmres")
    uf, it = forward.fixed_point_iterations(xi, om, g)
    assert np.linalg.norm(ug - ud) / np.linalg.norm(ud) < 1e-12
    assert np.linalg.norm(uf - ud) / np.linalg.norm(ud) < 1e-12
    assert it > 3
    # the solution satisfies u = u0 + omega^2 T(xi u)
    from oracle.operators import apply_interior
    res = ud - forward.incident_plane_wave(om, g) - om ** 2 * apply_interior(xi * ud, om, g)
    assert np.linalg.norm(res) / np.linalg.norm(ud) < 1e-12


def test_fixed_point_fails_loudly_when_not_contracting():
    g, xi = _tiny()
    with pytest.raises(RuntimeError):
        forward.fixed_point_iterations(200 * xi, 4 * np.pi, g, max_iter=200)


def test_born_limit_is_linear():
    g, xi = _tiny()
    om = 2 * np.pi
    Wb = forward.make_data(xi, [om], g, method="born")[0]
    for t, tol in ((1e-3, 5e-3), (1e-5, 5e-5)):
        Wt = forward.make_data(t * xi, [om], g, method="dense")[0] / t
        err = np.linalg.norm(Wt - Wb) / np.linalg.norm(Wb)
        assert err < tol


def test_noise_norm_exact_and_seeded():
    w = workload("c1")
    rng = np.random.default_rng(0)
    W = rng.standard_normal((1, w.m1, w.n, w.n)) + 1j * rng.standard_normal((1, w.m1, w.n, w.n))
    for d in (0.0, 0.01, 0.05):
        Wd = forward.add_noise(W, d, w.noise())
        assert abs(np.linalg.norm(Wd - W) - d * np.linalg.norm(W)) <= 1e-15 * np.linalg.norm(W) * 10
    assert np.array_equal(w.noise(), w.noise())
