"""The paper's own experiment (Sec. 5, 5.3, 5.4) through the C ABI against the oracle:
X = [-10,10]^2 x [-0.5,1.5] with M = 71 planes, data in the thick layer [6.01, 6.5]
on M1 = 71 planes or the thin layer [6.01, 6.02] on two, 11 point sources
(0, y_s, 6), the three-bump xi with A0 = 0.3, omega = 1, 2, 3, noise 0, 1e-7 and
1e-5 (delta_floor 1e-10, so that these levels stay distinct).  The horizontal grid
is N = 64 here (the bench runs N = 128) to keep the oracle to seconds.

M1 = 71 exceeds the dense form's limit (M1 <= 32), so the per-mode problem is solved
in the rank-one closed form (solve_form 1), exact for the Weyl kernel.  Checked: the
incident field of the sources (fs_incident_point_sources), the single-scattering
data with that field (fs_forward_born), and the reconstruction -- identical active
sets, alpha per mode, xi within fp64_tol (1e-10 down to delta = 1e-7, growing as
1/delta_eff below: the root's sensitivity to the data's rounding) in FP64, 1e-5 in the
mixed path at 1e-2 noise -- with its Delta_L2(z) (Sec. 5.3) printed beside the
oracle's."""
import functools

import numpy as np
import pytest

from oracle import forward, inverse
from oracle.grid import Geometry as OGeom
from oracle.metrics import delta_l2_z, rel_l2
from synth import paper_workload

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
N = 64
FLOOR = 1e-10


@functools.lru_cache(maxsize=None)
def paper_case(layer, delta):
    w = paper_workload(layer, n=N)
    g = OGeom(w.n, w.m, w.z1, w.z2, tuple(w.zy), period=w.period, x0=w.x0)
    u0s = np.stack([forward.incident_point_sources(om, g, w.sources) for om in w.omegas])
    W, _ = forward.make_data(w.xi, w.omegas, g, method="born", u0s=u0s)
    W = forward.add_noise(W, delta, w.noise()) if delta > 0 else W
    ref = inverse.reconstruct(W, w.omegas, g, delta, opts=inverse.Options(delta_floor=FLOOR), u0s=u0s)
    return w, g, u0s, W, ref


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


def _geom(w):
    from paper_1911_10487_gb300 import Geometry
    return Geometry(w.n, w.m, w.z1, w.z2, tuple(w.zy), w.period)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_incident_field_and_born_data(rc, precision):
    import torch
    w, g, u0s, W, _ = paper_case("thick", 0.0)
    u0 = rc.incident_point_sources(w.sources, list(w.omegas), _geom(w), precision=precision)
    torch.cuda.synchronize()
    e_u = rel_l2(u0.cpu().numpy(), u0s)
    rdt = torch.float64 if precision == "fp64" else torch.float32
    xi = torch.from_numpy(np.ascontiguousarray(w.xi)).to(rc.device, rdt)
    Wg = rc.forward_born(xi, list(w.omegas), _geom(w), precision=precision, incident=u0)
    torch.cuda.synchronize()
    e_w = rel_l2(Wg.cpu().numpy(), W)
    print(f"paper geometry {precision}: incident field {e_u:.2e}, Born data {e_w:.2e}")
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert e_u <= tol and e_w <= tol


def run(rc, layer, delta, precision):
    import torch
    w, g, u0s, W, ref = paper_case(layer, delta)
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    u0 = torch.from_numpy(u0s).to(rc.device, cdt)
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(rc.device, cdt)
    xi, c, alpha = rc.reconstruct(Wd, list(w.omegas), _geom(w), delta, precision=precision, want_alpha=True,
                                  solve_form=1, incident=u0, delta_floor=FLOOR)
    torch.cuda.synchronize()
    return w, ref, xi.double().cpu().numpy(), alpha.cpu().numpy(), rc.report()


def fp64_tol(delta, factor=1.0):
    """The FP64 agreement two correct implementations can reach on these data: the two
    sides' transforms of W differ by about u = 1e-16 ||W|| per mode, and the discrepancy
    root turns a data change into a relative change of alpha of order u ||W|| / delta_nu
    (phi^2 - delta_nu^2 is fixed to within ||P_perp b|| Delta b ~ delta_nu Delta b), which
    moves V~ by at most that: xi to max(1e-10, 1e-17 / delta_eff), delta_eff =
    max(delta, 1e-10).  The thin layer's per-mode problems are conditioned ten times
    worse (factor 10)."""
    return factor * max(1e-10, 1e-17 / max(delta, FLOOR))


@pytest.mark.parametrize("delta", [0.0, 1e-7, 1e-5])
def test_thick_layer_fp64(rc, delta):
    w, ref, xi, alpha, rep = run(rc, "thick", delta, "fp64")
    err = rel_l2(xi, ref.xi)
    act = np.isfinite(alpha)
    assert np.array_equal(act, ref.active)
    ra = np.abs(alpha[act] / ref.alpha[act] - 1)
    dz, dz_ref = delta_l2_z(xi, w.xi), delta_l2_z(ref.xi, w.xi)
    print(f"thick delta={delta}: xi {err:.2e}, alpha {ra.max():.2e}, active {act.sum()}, floor {rep['n_alpha_floor']}; "
          f"Delta_L2(z) min/median/max {np.nanmin(dz):.3f}/{np.nanmedian(dz):.3f}/{np.nanmax(dz):.3f} "
          f"(oracle {np.nanmin(dz_ref):.3f}/{np.nanmedian(dz_ref):.3f}/{np.nanmax(dz_ref):.3f})")
    assert err <= fp64_tol(delta)
    # alpha near its floor on the strong modes is fixed only loosely at the smallest
    # noise level (phi is flat in alpha there), as in test_gpu_parity
    assert ra.max() <= (1e-3 if delta == 0 else 1e-6)
    assert rep["n_alpha_floor"] == ref.counts["alpha_floor"]
    assert rep["n_grazing"] == ref.counts["grazing"]


@pytest.mark.parametrize("delta", [1e-2, 1e-5])
def test_thick_layer_mixed(rc, delta):
    """The mixed path transforms complex64 data in FP32 (relative rounding ~1e-7 per
    mode); the discrepancy root amplifies that by ||b|| / delta_nu, so the mixed path
    meets its 1e-5 bound where the noise level is well above the FP32 rounding
    (delta = 1e-2 asserted) and not at the paper's 1e-5 (printed: the FP64 path is the
    one for those data)."""
    w, ref, xi, alpha, rep = run(rc, "thick", delta, "mixed")
    err = rel_l2(xi, ref.xi)
    print(f"thick mixed delta={delta}: xi {err:.2e}, active {np.isfinite(alpha).sum()}/{ref.active.sum()}")
    if delta >= 1e-2:
        assert err <= 1e-5


@pytest.mark.parametrize("delta", [0.0, 1e-7])
def test_thin_layer_fp64(rc, delta):
    """Sec. 5.4.  As for the thin layer of test_gpu_parity_c2, xi is compared in the weight
    of its least-squares denominator (near the zeros of u it is fixed only to rounding)."""
    w, ref, xi, alpha, rep = run(rc, "thin", delta, "fp64")
    act = np.isfinite(alpha)
    assert np.array_equal(act, ref.active)
    den = np.sum(np.abs(ref.u) ** 2, axis=0)
    werr = np.linalg.norm((xi - ref.xi) * den) / np.linalg.norm(ref.xi * den)
    dz = delta_l2_z(xi, w.xi)
    print(f"thin delta={delta}: weighted xi {werr:.2e}, unweighted {rel_l2(xi, ref.xi):.2e}, active {act.sum()}; "
          f"Delta_L2(z) median {np.nanmedian(dz):.3f}")
    assert werr <= fp64_tol(delta, 10.0)


def test_dense_form_rejects_the_thick_layer(rc):
    import torch
    from paper_1911_10487_gb300 import FlatLayerError
    w, _, _, W, _ = paper_case("thick", 0.0)
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(rc.device)
    with pytest.raises(FlatLayerError, match="FS_EUNSUPPORTED"):
        rc.reconstruct(Wd, list(w.omegas), _geom(w), 0.0)


@pytest.mark.parametrize("method", ["fixed_point_gmres", "gmres"])
def test_full_scattering_data_with_point_sources(rc, method):
    """Algorithm 1 (with the GMRES fallback where the fixed point does not contract) and
    GMRES on u = u0 + omega^2 T(xi u) with the point-source incident field of the paper
    geometry (Sec. 5.1 generates its data this way), against the oracle's GMRES with the
    same field, at N = 24 (the strong three-bump scatterer)."""
    import torch
    w = paper_workload("thick", n=24, m=12, m1=6)
    g = OGeom(w.n, w.m, w.z1, w.z2, tuple(w.zy), period=w.period, x0=w.x0)
    om = list(w.omegas)
    u0s = np.stack([forward.incident_point_sources(o, g, w.sources) for o in om])
    Wref, uref = forward.make_data(w.xi, om, g, method="gmres", u0s=u0s)
    u0 = torch.from_numpy(u0s).to(rc.device)
    xi = torch.from_numpy(np.ascontiguousarray(w.xi)).to(rc.device)
    Wg, ug, its = rc.forward(xi, om, _geom(w), method=method, want_u=True, incident=u0)
    torch.cuda.synchronize()
    ew, eu = rel_l2(Wg.cpu().numpy(), Wref), rel_l2(ug.cpu().numpy(), uref)
    print(f"point sources, {method}: W {ew:.2e}, u {eu:.2e}, iterations {its}")
    assert ew <= 1e-10 and eu <= 1e-10
