"""Pins of the point-source incident field (Sec. 5: sources f = sum a_s delta(x - x_s),
u0 = sum a_s G(|x - x_s|)) in the periodic model of the oracle.

With a damped wavenumber the periodised field is an absolutely convergent sum of
images, sum_s sum_n a_s G(|x - x_s - n L|), which a direct sum over a few hundred
images reproduces; the spectral form (DFT coefficients (N^2/L^2) K_nu e^{-i nu.(r_s - x0)})
must equal it at every grid point -- a wrong sign of the phase, a wrong grid origin
or a missing 1/L^2 fails this.  The field also satisfies the reciprocity / symmetry
of G (a source on the symmetry axis gives a mirror-symmetric field)."""
import numpy as np

from oracle.forward import incident_point_sources
from oracle.grid import Geometry, layer_planes
from oracle.kernel import green


def test_spectral_field_equals_image_sum_with_damping():
    g = Geometry(16, 3, -0.5, 0.1, layer_planes(1.0, 1.2, 2), period=4.0, x0=-2.0)
    k0 = 3.0 * (1 + 0.6j)  # damping makes the image sum converge: |G| ~ e^{-1.8 rho}
    sources = [(0.3, -0.7, 1.5, 1.0), (-1.1, 0.4, 1.8, -0.5)]
    u0 = incident_point_sources(k0, g, sources)
    xs = g.x_nodes()
    Z, Y, X = np.meshgrid(g.zx(), xs, xs, indexing="ij")
    ref = np.zeros_like(u0)
    R = 12  # images within 12 periods: e^{-1.8 * 48} is far below rounding
    for (sx, sy, sz, a) in sources:
        for nx in range(-R, R + 1):
            for ny in range(-R, R + 1):
                rho = np.sqrt((X - sx - nx * g.period) ** 2 + (Y - sy - ny * g.period) ** 2 + (Z - sz) ** 2)
                ref += a * green(k0, rho)
    # the spectral form drops the modes beyond the grid's band: e^{-|nu| dz} with
    # |nu| >= 2 pi (N/2)/L = 12.6 and dz >= 1.4
    assert np.max(np.abs(u0 - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_source_on_the_axis_gives_a_mirror_symmetric_field():
    g = Geometry(16, 4, -0.5, 1.5, layer_planes(6.01, 6.5, 3), period=20.0, x0=-10.0)
    u0 = incident_point_sources(2.0, g, [(0.0, 0.0, 6.0, 1.0)])
    # nodes x0 + i h are symmetric about 0 under i -> N - i (x = -10 is its own image)
    mirror = np.roll(u0[:, :, ::-1], 1, axis=2)
    assert np.max(np.abs(u0 - mirror)) <= 1e-12 * np.max(np.abs(u0))
