"""The sampled-G kernel (Sec. 5: G~ computed from the values of G by the FFT; the
Geometry.kernel = "sampled" reading of the oracle) through the C ABI: a kernel plan
tabulates A_nu and the Toeplitz row of eq. (9) for every mode, and the dense
per-mode solve runs on it.  Unlike the Weyl kernel, A_nu is numerically full rank
(rapidly decaying singular values, Sec. 6), so the Lanczos model runs past two steps
and the mixed refinement's treatment of the complement is no longer exact.

Tolerances as for the Weyl kernel: xi rel. L2 <= 1e-10 (FS_FP64), <= 1e-5 (FS_MIXED);
identical active sets and alpha per mode <= 1e-7 (FP64)."""
import functools

import numpy as np
import pytest

from oracle import forward, inverse
from oracle.grid import Geometry as OGeom, layer_planes
from oracle.metrics import rel_l2
from synth import random_gaussians

pytestmark = pytest.mark.gpu

SPEC = {  # n, m, m1, omegas
    "s12": (12, 5, 3, [3 * np.pi]),
    "s24": (24, 7, 5, [2 * np.pi, 4.5 * np.pi]),
    "s32": (32, 16, 8, [4 * np.pi]),
    "s48": (48, 13, 9, [4 * np.pi, 6 * np.pi]),
    "s96": (96, 24, 17, [5 * np.pi]),
}


@functools.lru_cache(maxsize=None)
def sampled_case(name, delta=0.01):
    n, m, m1, om = SPEC[name]
    g = OGeom(n, m, 0.2, 1.0, layer_planes(1.2, 1.6, m1), kernel="sampled")
    rng = np.random.default_rng(n * 1000 + m + 7)
    xi = random_gaussians(rng, n, m, g.z1, g.z2, 2, (0.1, 0.25), 0.05)
    W, _ = forward.make_data(xi, om, g, method="born" if n >= 48 else "gmres")
    noise = np.random.default_rng(17).standard_normal(W.shape) + 1j * np.random.default_rng(18).standard_normal(W.shape)
    W = forward.add_noise(W, delta, noise)
    ref = inverse.reconstruct(W, om, g, delta)
    return g, np.array(om), W, ref


@pytest.fixture(scope="module")
def rc():
    import torch
    from paper_1911_10487_gb300 import build
    build.build()
    from paper_1911_10487_gb300 import Reconstructor
    r = Reconstructor(0)
    yield r
    torch.cuda.synchronize()
    r.close()


def _geom(g):
    from paper_1911_10487_gb300 import Geometry
    return Geometry(g.n, g.m, g.z1, g.z2, tuple(g.zy), g.period)


def run(rc, name, precision, delta=0.01, **opts):
    import torch
    from paper_1911_10487_gb300 import KernelPlan
    g, om, W, ref = sampled_case(name, delta)
    plan = KernelPlan(rc, _geom(g), list(om), precision)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(device=rc.device, dtype=dt)
    xi, c, alpha = rc.reconstruct(Wd, list(om), _geom(g), delta, precision=precision, want_alpha=True,
                                  kernel_plan=plan, **opts)
    torch.cuda.synchronize()
    rep = rc.report()
    plan.close()
    return xi.double().cpu().numpy(), alpha.cpu().numpy(), rep, ref


@pytest.mark.parametrize("name", list(SPEC))
def test_sampled_fp64_matches_oracle(rc, name):
    xi, alpha, rep, ref = run(rc, name, "fp64")
    err = rel_l2(xi, ref.xi)
    act = np.isfinite(alpha)
    same = np.array_equal(act, ref.active)
    ra = np.abs(alpha[ref.active] / ref.alpha[ref.active] - 1) if same and ref.active.any() else np.zeros(1)
    print(f"sampled {name} fp64: xi {err:.2e}, active {act.sum()}/{ref.active.sum()}, alpha {ra.max():.2e}, "
          f"floor {rep['n_alpha_floor']}/{ref.counts['alpha_floor']}")
    assert same
    assert err <= 1e-10
    assert ra.max() <= 1e-7
    assert rep["n_grazing"] == 0 and ref.counts["grazing"] == 0
    assert rep["n_alpha_floor"] == ref.counts["alpha_floor"]


@pytest.mark.parametrize("name", list(SPEC))
def test_sampled_mixed_matches_oracle(rc, name):
    xi, alpha, rep, ref = run(rc, name, "mixed")
    err = rel_l2(xi, ref.xi)
    act = np.isfinite(alpha)
    print(f"sampled {name} mixed: xi {err:.2e}, active {act.sum()}/{ref.active.sum()}, "
          f"fp64 route {rep['n_fp64_fallback']}, refine sweeps {rep['n_refine_iters']}")
    assert np.sum(act != ref.active) <= 2
    assert err <= 1e-5


def test_sampled_is_not_the_weyl_kernel(rc):
    """The same data reconstructed with the Weyl kernel differs: the plan is used."""
    import torch
    g, om, W, ref = sampled_case("s24")
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(rc.device)
    xi_w, _, _ = rc.reconstruct(Wd, list(om), _geom(g), 0.01)
    torch.cuda.synchronize()
    assert rel_l2(xi_w.cpu().numpy(), ref.xi) > 1e-3


def test_plan_checks(rc):
    import torch
    from paper_1911_10487_gb300 import FlatLayerError, KernelPlan
    g, om, W, ref = sampled_case("s12")
    plan = KernelPlan(rc, _geom(g), list(om), "fp64")
    D = g.m1 * g.m + g.m
    assert plan.nbytes == 16 * D * g.n * g.n * len(om) + 8 * g.n * g.n * len(om)
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(rc.device)
    with pytest.raises(FlatLayerError, match="FS_EINVAL"):  # other frequencies
        rc.reconstruct(Wd, [2 * np.pi], _geom(g), 0.01, kernel_plan=plan)
    with pytest.raises(FlatLayerError, match="FS_EINVAL"):  # other precision
        rc.reconstruct(Wd.to(torch.complex64), list(om), _geom(g), 0.01, precision="mixed", kernel_plan=plan)
    with pytest.raises(FlatLayerError, match="FS_EUNSUPPORTED"):  # rank-one form
        rc.reconstruct(Wd, list(om), _geom(g), 0.01, kernel_plan=plan, solve_form=1)
    with pytest.raises(FlatLayerError, match="FS_EUNSUPPORTED"):
        rc.reconstruct_batch([(Wd, list(om), _geom(g), 0.01)], "fp64", n_streams=1, kernel_plan=plan.handle)
    plan.close()
