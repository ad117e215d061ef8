"""The build's limits, through the C ABI against the oracle: the rank-one form at the
largest plane counts (M = M1 = 128), the dense form at its own (M = 64, M1 = 32), the
largest frequency list (n_omega = 64), and the first sizes beyond each limit, which
must be refused with FS_EUNSUPPORTED before any device work.  Tolerances as for every
result: xi rel. L2 <= 1e-10 (FS_FP64), <= 1e-5 (FS_MIXED), identical active sets."""
import functools

import numpy as np
import pytest

from _cases import geometry
from oracle import forward, inverse
from oracle.metrics import rel_l2
from synth import random_gaussians

pytestmark = pytest.mark.gpu


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


@functools.lru_cache(maxsize=None)
def limit_case(n, m, m1, n_omega):
    g = geometry(n, m, m1)
    rng = np.random.default_rng(n * 100000 + m * 1000 + m1 * 10 + n_omega)
    om = np.sort(rng.uniform(1.5 * np.pi, 4.0 * np.pi, n_omega))
    xi = random_gaussians(rng, n, m, g.z1, g.z2, 2, (0.15, 0.3), 0.05)
    W, _ = forward.make_data(xi, list(om), g, method="born")
    noise = np.random.default_rng(11).standard_normal(W.shape) + 1j * np.random.default_rng(12).standard_normal(W.shape)
    W = forward.add_noise(W, 0.01, noise)
    return g, om, W, inverse.reconstruct(W, list(om), g, 0.01)


def _geom(g):
    from paper_1911_10487_gb300 import Geometry
    return Geometry(g.n, g.m, g.z1, g.z2, tuple(g.zy), g.period)


def _run(rc, g, om, W, precision, **kw):
    import torch
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(rc.device, dt)
    xi, _, alpha = rc.reconstruct(Wd, list(om), _geom(g), 0.01, precision=precision, want_alpha=True, **kw)
    torch.cuda.synchronize()
    return xi.double().cpu().numpy(), np.isfinite(alpha.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape, form", [((12, 128, 128, 2), 1), ((8, 64, 32, 2), 0), ((8, 3, 2, 64), 0),
                                         ((8, 3, 2, 64), 1)])
def test_at_the_limits(rc, shape, form, precision):
    g, om, W, ref = limit_case(*shape)
    xi, act = _run(rc, g, om, W, precision, solve_form=form)
    err = rel_l2(xi, ref.xi)
    print(f"{shape} form {form} {precision}: xi {err:.2e}, active {act.sum()}")
    assert np.array_equal(act, ref.active)
    assert err <= (1e-10 if precision == "fp64" else 1e-5)


def test_first_sizes_beyond_the_limits_are_refused(rc):
    import torch
    from paper_1911_10487_gb300 import FlatLayerError
    from paper_1911_10487_gb300._abi import FS_EUNSUPPORTED
    for (n, m, m1, n_om, form) in ((8, 129, 2, 1, 1), (8, 3, 129, 1, 1), (8, 3, 2, 65, 1), (8, 65, 2, 1, 0),
                                   (8, 3, 33, 1, 0), (20, 3, 2, 1, 1)):
        g = geometry(n, m, m1)
        W = torch.zeros((n_om, m1, n, n), dtype=torch.complex128, device=rc.device)
        with pytest.raises(FlatLayerError) as ei:
            rc.reconstruct(W, [2.0 * np.pi] * n_om, _geom(g), 0.01, solve_form=form)
        assert ei.value.status == FS_EUNSUPPORTED, (n, m, m1, n_om, form)
