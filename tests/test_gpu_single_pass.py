"""The single-pass (thread-block cluster) transforms of the mixed path against the
two-pass forms, through the C ABI:
  forward_single_pass  the 2D transform of W (Algorithm 2, step 1) by a cluster per data
                       plane, rows and columns exchanged in distributed shared memory;
  inverse_single_pass  the inverse transforms and the recovery of xi (steps 2 and 3) by
                       a cluster per X plane;
  fp64_sums            the least-squares sums of Sec. 5.2 in FP64 from the start (the
                       route the FP32 sums take where they overflow).
Every combination decides the same active modes and gives xi within FP32 rounding
(1e-6) of the two-pass form, over the sizes that select each cluster size (1, 2, 4 and 8
CTAs; N = 96, whose inverse stays two-pass, for the forward pass; at N = 192 and 256 both
passes stay two-pass and the options must change nothing), with the plane wave and with a
given incident field.  Also: the mixed path refuses noise levels
below its FP32 data resolution (FS_MIXED_MIN_NOISE)."""
import numpy as np
import pytest

from _cases import case
from oracle.metrics import rel_l2

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


def _geom(g):
    from paper_1911_10487_gb300 import Geometry
    return Geometry(g.n, g.m, g.z1, g.z2, tuple(g.zy), g.period)


def _run(rc, Wd, om, geom, delta, **kw):
    import torch
    xi, _, alpha = rc.reconstruct(Wd, list(om), geom, delta, precision="mixed", want_alpha=True, **kw)
    torch.cuda.synchronize()
    return xi.double().cpu().numpy(), np.isfinite(alpha.cpu().numpy()), rc.report()


@pytest.mark.parametrize("name", ["r8", "r12", "r24", "r48", "c1", "r96", "r192", "r256", "c2"])
def test_single_pass_transforms_match_two_pass(rc, name):
    import torch
    g, om, W, _ = case(name, 0.01)
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(device=rc.device, dtype=torch.complex64)
    x0, a0, r0 = _run(rc, Wd, om, _geom(g), 0.01, forward_single_pass=0, inverse_single_pass=0)
    for fwd, inv, s64 in ((1, 1, 0), (1, 0, 0), (0, 1, 0), (1, 1, 1), (0, 0, 1)):
        x, a, r = _run(rc, Wd, om, _geom(g), 0.01, forward_single_pass=fwd, inverse_single_pass=inv,
                       fp64_sums=s64)
        err = rel_l2(x, x0)
        print(f"{name} forward {fwd} inverse {inv} fp64 sums {s64}: xi vs two-pass {err:.2e}")
        assert np.array_equal(a, a0)
        assert r["n_active"] == r0["n_active"] and r["n_columns"] == r0["n_columns"]
        assert r["n_nonfinite"] == 0 and r["n_u_guard"] == r0["n_u_guard"]
        assert err <= 1e-6


def test_single_pass_with_given_incident_field(rc):
    """The incident field of the paper's point sources (Sec. 5) added after the inverse
    transform (the INC form of the recovery), N = 64 (clusters of 4).  The interference
    of the eleven sources leaves near-zeros of u on X, where xi = Re(sum conj(u) V) /
    sum |u|^2 is fixed only to the rounding of the transforms amplified by 1 / |u|: the
    two forms (radix 8 and 16 column passes) agree to the mixed path's bound (1e-5), and
    to 1e-6 in the weight of the least-squares denominator."""
    import torch
    from synth import paper_workload
    from paper_1911_10487_gb300 import Geometry
    pw = paper_workload("thick", n=64, m=24, m1=16)
    geom = Geometry(pw.n, pw.m, pw.z1, pw.z2, tuple(pw.zy), pw.period)
    om = [float(x) for x in pw.omegas]
    u0 = rc.incident_point_sources(pw.sources, om, geom, precision="mixed")
    xi_t = torch.from_numpy(np.ascontiguousarray(pw.xi)).to(rc.device, torch.float32)
    W = rc.forward_born(xi_t, om, geom, precision="mixed", incident=u0)
    torch.cuda.synchronize()
    nz = torch.randn(W.shape, dtype=torch.complex64, device=rc.device, generator=torch.Generator(rc.device).manual_seed(3))
    W = W + 1e-2 * torch.linalg.vector_norm(W) / torch.linalg.vector_norm(nz) * nz
    kw = dict(solve_form=1, incident=u0)
    x0, a0, r0 = _run(rc, W, om, geom, 1e-2, forward_single_pass=0, inverse_single_pass=0, **kw)
    assert a0.sum() > 0
    den = (u0.abs() ** 2).sum(0).double().cpu().numpy()  # sum over the frequencies of |u0|^2
    for fwd, inv, s64 in ((1, 1, 0), (1, 1, 1), (0, 1, 0)):
        x, a, r = _run(rc, W, om, geom, 1e-2, forward_single_pass=fwd, inverse_single_pass=inv, fp64_sums=s64, **kw)
        err = rel_l2(x, x0)
        werr = np.sqrt(np.sum(den * (x - x0) ** 2) / np.sum(den * x0 ** 2))
        print(f"incident field: forward {fwd} inverse {inv} fp64 sums {s64}: xi vs two-pass {err:.2e}, "
              f"weighted {werr:.2e}")
        assert np.array_equal(a, a0)
        assert err <= 1e-5 and werr <= 1e-6


def test_mixed_path_refuses_noise_below_its_resolution(rc):
    import torch
    from paper_1911_10487_gb300 import FlatLayerError
    from paper_1911_10487_gb300._abi import FS_EUNSUPPORTED, FS_MIXED_MIN_NOISE
    g, om, W, _ = case("r24", 0.01)
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(device=rc.device, dtype=torch.complex64)
    with pytest.raises(FlatLayerError) as ei:
        rc.reconstruct(Wd, list(om), _geom(g), 0.0, precision="mixed", delta_floor=1e-10)
    assert ei.value.status == FS_EUNSUPPORTED
    with pytest.raises(FlatLayerError):
        rc.reconstruct(Wd, list(om), _geom(g), 0.5 * FS_MIXED_MIN_NOISE, precision="mixed", delta_floor=0.0)
    # at the limit, with a given alpha, and in FP64 the same data are accepted
    rc.reconstruct(Wd, list(om), _geom(g), FS_MIXED_MIN_NOISE, precision="mixed", delta_floor=0.0)
    rc.reconstruct(Wd, list(om), _geom(g), 0.0, precision="mixed", delta_floor=1e-10, alpha_mode=1,
                   alpha_given=[1e-3] * len(om))
    rc.reconstruct(Wd.to(torch.complex128), list(om), _geom(g), 0.0, precision="fp64", delta_floor=1e-10)
    torch.cuda.synchronize()
