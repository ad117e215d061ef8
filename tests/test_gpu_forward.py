"""The full-scattering forward solve on the device (fs_forward: Algorithm 1, the fixed
point of eq. 6; restarted GMRES; Algorithm 1 with a GMRES fallback -- then the data of
eq. 7) against the oracle's own fixed point and GMRES (oracle/forward.py), through the
C ABI.

FP64: W and the total field u agree to 1e-10 (relative L2) and Algorithm 1 takes the
oracle's number of iterations per frequency (the same stopping rule, rtol = 1e-13, on
iterates that agree to ~1e-15); GMRES solutions agree to 1e-10 (1e-9 for a strong
scatterer, condition number ~10).  Mixed: 1e-5 at rtol = 1e-6 (the FP32 transforms'
rounding).
"""
import numpy as np
import pytest

from _cases import case
from oracle import forward
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu

NAMES = ["c1", "r12", "r24", "r48"]


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


def _run(rc, name, precision, **kw):  # kw: forward options (method, max_iter, rtol)
    import torch
    g, om, _, xi = case(name, 0.01)
    dt = torch.float64 if precision == "fp64" else torch.float32
    x = torch.from_numpy(np.ascontiguousarray(xi)).to(rc.device, dt)
    W, u, its = rc.forward(x, list(om), _geom(g), precision=precision, want_u=True, **kw)
    torch.cuda.synchronize()
    return g, om, xi, W.cpu().numpy(), u.cpu().numpy(), its


@pytest.mark.parametrize("name", NAMES)
def test_fixed_point_matches_oracle_fp64(rc, name):
    g, om, xi, W, u, its = _run(rc, name, "fp64")
    Wr, ur = forward.make_data(xi, om, g, method="fixed_point")
    ref_its = [forward.fixed_point_iterations(xi, o, g)[1] for o in om]
    ew, eu = rel_l2(W, Wr), rel_l2(u, ur)
    print(f"{name}: W {ew:.2e}, u {eu:.2e}, iterations gpu {its} oracle {ref_its}")
    assert ew <= 1e-10 and eu <= 1e-10
    assert its == ref_its


@pytest.mark.parametrize("name", ["c1", "r48"])
def test_fixed_point_mixed(rc, name):
    g, om, xi, W, u, its = _run(rc, name, "mixed")
    Wr, ur = forward.make_data(xi, om, g, method="fixed_point")
    ew, eu = rel_l2(W, Wr), rel_l2(u, ur)
    print(f"{name} mixed: W {ew:.2e}, u {eu:.2e}, iterations {its}")
    assert ew <= 1e-5 and eu <= 1e-5


def test_zero_iterations_is_born(rc):
    import torch
    g, om, _, xi = case("r24", 0.01)
    x = torch.from_numpy(np.ascontiguousarray(xi)).to(rc.device, torch.float64)
    W, u, its = rc.forward(x, list(om), _geom(g), max_iter=0, want_u=True)
    Wb = rc.forward_born(x, list(om), _geom(g))
    torch.cuda.synchronize()
    assert its == [0] * len(om)
    assert rel_l2(W.cpu().numpy(), Wb.cpu().numpy()) <= 1e-13
    u0 = np.stack([forward.incident_plane_wave(o, g) for o in om])
    assert rel_l2(u.cpu().numpy(), u0) <= 1e-14


def test_not_converged_is_reported(rc):
    """Too few iterations, and a scatterer too strong for the fixed point
    (omega^2 ||T xi|| > 1): FS_ENOCONV, raised on the host."""
    import torch
    from paper_1911_10487_gb300 import FlatLayerError
    g, om, _, xi = case("r24", 0.01)
    x = torch.from_numpy(np.ascontiguousarray(xi)).to(rc.device, torch.float64)
    with pytest.raises(FlatLayerError, match="FS_ENOCONV"):
        rc.forward(x, list(om), _geom(g), max_iter=2)
    with pytest.raises(FlatLayerError, match="FS_ENOCONV"):
        rc.forward(60.0 * x, list(om), _geom(g), max_iter=200)


@pytest.mark.parametrize("name", ["c1", "r24"])
def test_gmres_matches_oracle_fp64(rc, name):
    """FS_GMRES against the oracle's GMRES (both to a relative residual 1e-13)."""
    g, om, xi, W, u, its = _run(rc, name, "fp64", method="gmres")
    Wr, ur = forward.make_data(xi, om, g, method="gmres")
    ew, eu = rel_l2(W, Wr), rel_l2(u, ur)
    print(f"{name} gmres: W {ew:.2e}, u {eu:.2e}, operator applications {its}")
    assert ew <= 1e-10 and eu <= 1e-10


def test_gmres_mixed(rc):
    g, om, xi, W, u, its = _run(rc, "c1", "mixed", method="gmres")
    Wr, ur = forward.make_data(xi, om, g, method="gmres")
    assert rel_l2(W, Wr) <= 1e-5 and rel_l2(u, ur) <= 1e-5


def test_fixed_point_falls_back_to_gmres(rc):
    """20 xi on the 24^2 case: Algorithm 1 converges at the lower frequency and
    diverges at the upper one, where GMRES takes over; both match the oracle's GMRES."""
    import torch
    g, om, _, xi = case("r24", 0.01)
    xs = 20.0 * xi
    x = torch.from_numpy(np.ascontiguousarray(xs)).to(rc.device, torch.float64)
    with pytest.raises(Exception, match="FS_ENOCONV"):
        rc.forward(x, list(om), _geom(g), max_iter=200)
    W, u, its = rc.forward(x, list(om), _geom(g), max_iter=200, want_u=True, method="fixed_point_gmres")
    torch.cuda.synchronize()
    Wr, ur = forward.make_data(xs, om, g, method="gmres")
    ew, eu = rel_l2(W.cpu().numpy(), Wr), rel_l2(u.cpu().numpy(), ur)
    print(f"fallback: W {ew:.2e}, u {eu:.2e}, iterations {its}")
    assert its[0] == forward.fixed_point_iterations(xs, om[0], g)[1]
    assert ew <= 1e-9 and eu <= 1e-9
