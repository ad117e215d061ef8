"""Pins of the error measures: Delta_L2(z) of Sec. 5.3 (per X plane, the L2(xy)
norm of the error over that of the exact solution) on planted per-plane errors
whose value is known in advance, and rel_l2 on a hand-computed case."""
import numpy as np

from oracle.metrics import delta_l2_z, rel_l2


def test_delta_l2_z_recovers_planted_plane_errors():
    rng = np.random.default_rng(11)
    m, n = 7, 16
    exact = rng.standard_normal((m, n, n))
    exact[4] = 0.0  # a plane without scatterer: Delta undefined there
    planted = np.array([0.0, 1e-3, 0.5, 2.0, 0.3, 1e-7, 1.0])
    appr = exact.copy()
    for l in range(m):
        d = rng.standard_normal((n, n))
        d /= np.linalg.norm(d)
        appr[l] += planted[l] * (np.linalg.norm(exact[l]) if l != 4 else 1.0) * d
    got = delta_l2_z(appr, exact)
    ok = np.arange(m) != 4
    assert np.allclose(got[ok], planted[ok], rtol=1e-12, atol=1e-15)
    assert np.isnan(got[4])
    # one number per plane, independent of the other planes
    appr2 = appr.copy()
    appr2[2] = exact[2]
    got2 = delta_l2_z(appr2, exact)
    assert got2[2] == 0.0 and np.array_equal(got2[[0, 1, 3, 5, 6]], got[[0, 1, 3, 5, 6]])


def test_rel_l2_hand_case():
    a = np.array([3.0, 4.0, 0.0])
    b = np.array([0.0, 4.0, 0.0])
    assert rel_l2(a, b) == 3.0 / 4.0
    assert rel_l2(np.zeros(3), np.zeros(3)) == 0.0
