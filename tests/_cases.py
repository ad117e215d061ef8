"""Seeded cases shared by the GPU parity tests: data W from the oracle's forward
generator (CPU, FP64) plus seeded noise, and the oracle's reconstruction."""
from __future__ import annotations

import functools

import numpy as np

from oracle import forward, inverse
from oracle.grid import Geometry, layer_planes
from synth import gaussian_inclusions, random_gaussians, workload


def geometry(n, m, m1, z1=0.2, z2=1.0, z3=1.2, z4=1.6, period=2.0):
    return Geometry(n, m, z1, z2, layer_planes(z3, z4, m1), period)


@functools.lru_cache(maxsize=None)
def case(name: str, delta: float = 0.01, method: str = "gmres"):
    """(geometry, omegas, W_noisy, xi_true) for a named seeded case."""
    if name in ("c1", "c2", "c5"):
        w = workload(name)
        g = Geometry(w.n, w.m, w.z1, w.z2, tuple(w.zy))
        # the 128^2 x 64 workloads take single-scattering data (as the bench does): a
        # CPU full-scattering solve at that size takes many minutes
        W, _ = forward.make_data(w.xi, w.omegas, g, method="born" if w.n >= 128 else method)
        return g, np.array(w.omegas), forward.add_noise(W, delta, w.noise()), w.xi
    if name == "thin256":
        # the thin data layer of Sec. 5.4: two planes 0.01 apart (the paper's
        # [6.01, 6.02] above X), here 0.2 above the X box of the workloads
        g = geometry(256, 6, 2, z3=1.2, z4=1.21)
        om = [2 * np.pi, 3 * np.pi]
        rng = np.random.default_rng(256 * 1000 + 6)
        xi = random_gaussians(rng, 256, 6, g.z1, g.z2, 2, (0.1, 0.25), 0.05)
        W, _ = forward.make_data(xi, om, g, method="born")
        noise = np.random.default_rng(9).standard_normal(W.shape) + 1j * np.random.default_rng(10).standard_normal(W.shape)
        return g, np.array(om), forward.add_noise(W, delta, noise), xi
    # small ragged cases: (n, m, m1, omegas)
    spec = {
        "r12": (12, 5, 3, [3 * np.pi]),
        "r24": (24, 7, 5, [2 * np.pi, 4.5 * np.pi]),
        "r48": (48, 13, 9, [4 * np.pi, 6 * np.pi, 7 * np.pi]),
        "r96": (96, 24, 17, [5 * np.pi]),
        "r8": (8, 3, 1, [np.pi]),
        "r192": (192, 9, 4, [3 * np.pi]),
        "r256": (256, 6, 6, [2 * np.pi, 3 * np.pi]),
    }[name]
    n, m, m1, om = spec
    g = geometry(n, m, m1)
    rng = np.random.default_rng(n * 1000 + m)
    xi = random_gaussians(rng, n, m, g.z1, g.z2, 2, (0.1, 0.25), 0.05)
    W, _ = forward.make_data(xi, om, g, method="born" if n >= 96 else method)
    noise = np.random.default_rng(7).standard_normal(W.shape) + 1j * np.random.default_rng(8).standard_normal(W.shape)
    return g, np.array(om), forward.add_noise(W, delta, noise), xi


@functools.lru_cache(maxsize=None)
def oracle_result(name: str, delta: float = 0.01, **kw):
    g, om, W, _ = case(name, delta)
    return inverse.reconstruct(W, om, g, delta, opts=inverse.Options(**kw))
