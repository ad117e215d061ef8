"""The rank-one closed form of the per-mode problem (fs_options.solve_form = 1) and
the truncated-SVD regulariser, through the C ABI, against the FP64 oracle (SVD per
mode, bisection for the discrepancy root).  Same tolerances as the dense form:
xi rel. L2 <= 1e-10 (FS_FP64), <= 1e-5 (FS_MIXED); identical active sets; alpha per
mode <= 1e-7 (FP64).  The closed form and the dense form on the GPU agree to
rounding (<= 1e-12).

TSVD in FS_MIXED: truncation at rank one is the pseudo-inverse, which damps no
mode, so any rounding of the data reaches V~ amplified by the inverse of the mode's
singular value.  The route therefore transforms its complex64 data in FP64, and it is
compared with the oracle applied to the same complex64 data (promoted exactly to
complex128): the quantisation of W to complex64 is the caller's input, not an error
of the method, and it is what the complex128 oracle would additionally see
(printed, not asserted).  Tolerance 1e-5 as for every mixed result."""
import numpy as np
import pytest

from _cases import case, oracle_result
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu

NAMES = ["c1", "r8", "r12", "r24", "r48", "r96", "r192", "r256"]
TOL_TSVD_MIXED = 1e-5


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


def run(rc, name, delta, precision, **opts):
    import torch
    g, om, W, _ = case(name, delta)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(device=rc.device, dtype=dt)
    xi, c, alpha = rc.reconstruct(Wd, list(om), _geom(g), delta, precision=precision, want_alpha=True, **opts)
    torch.cuda.synchronize()
    return xi.double().cpu().numpy(), alpha.cpu().numpy(), rc.report()


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tikhonov_rank1_matches_oracle(rc, name, precision):
    ref = oracle_result(name, 0.01)
    xi, alpha, rep = run(rc, name, 0.01, precision, solve_form=1)
    err = rel_l2(xi, ref.xi)
    act = np.isfinite(alpha)
    assert np.array_equal(act, ref.active)
    ra = np.max(np.abs(alpha[act] / ref.alpha[act] - 1)) if act.any() else 0.0
    print(f"{name} {precision}: xi {err:.2e}, alpha {ra:.2e}, floors {rep['n_alpha_floor']}")
    assert err <= (1e-10 if precision == "fp64" else 1e-5)
    if precision == "fp64":
        assert ra <= 1e-7


@pytest.mark.parametrize("name", ["c1", "r48", "r256"])
def test_rank1_equals_dense_form(rc, name):
    x1, a1, _ = run(rc, name, 0.05, "fp64", solve_form=1)
    x0, a0, _ = run(rc, name, 0.05, "fp64")
    assert rel_l2(x1, x0) <= 1e-12
    act = np.isfinite(a0)
    assert np.array_equal(np.isfinite(a1), act)


@pytest.mark.parametrize("name", ["c1", "r48", "r96", "r256"])
def test_mixed_rank1_equals_mixed_dense_form(rc, name):
    """Both mixed forms solve the problem of the same FP32 data with FP32-rounded kernel
    factors to about FP64 accuracy (two-float closed form; refinement of the dense solve
    against a two-float residual): their xi agree far inside the 1e-5 bound.  Their alpha
    agree to the dense form's FP32 root on its Lanczos model (both sit ~1e-4 from the
    oracle's, the sensitivity of the root to the FP32 rounding of the data)."""
    x1, a1, _ = run(rc, name, 0.01, "mixed", solve_form=1)
    x0, a0, _ = run(rc, name, 0.01, "mixed")
    act = np.isfinite(a0)
    assert np.array_equal(np.isfinite(a1), act)
    err = rel_l2(x1, x0)
    ra = np.max(np.abs(a1[act] / a0[act] - 1)) if act.any() else 0.0
    print(f"{name}: mixed rank-one vs mixed dense: xi {err:.2e}, alpha {ra:.2e}")
    assert err <= 1e-6
    assert ra <= 1e-3


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tsvd_matches_oracle(rc, name, precision):
    ref = oracle_result(name, 0.01, regularizer="tsvd")
    xi, alpha, _ = run(rc, name, 0.01, precision, solve_form=1, regularizer=1)
    act = np.isfinite(alpha)
    assert np.all(alpha[act] == 0.0)
    err = rel_l2(xi, ref.xi)
    if precision == "fp64":
        assert np.array_equal(act, ref.active)
        print(f"tsvd {name} fp64: xi {err:.2e}")
        assert err <= 1e-10
        return
    from oracle import inverse
    g, om, W, _ = case(name, 0.01)
    W32 = W.astype(np.complex64).astype(np.complex128)
    ref32 = inverse.reconstruct(W32, om, g, 0.01, opts=inverse.Options(regularizer="tsvd"))
    err32 = rel_l2(xi, ref32.xi)
    print(f"tsvd {name} mixed: xi {err32:.2e} vs the oracle on the same complex64 data, "
          f"{err:.2e} vs the oracle on the complex128 data")
    assert np.sum(act != ref32.active) <= 2
    assert err32 <= TOL_TSVD_MIXED


def test_given_alpha_rank1(rc):
    g, om, W, _ = case("r24", 0.01)
    given = [3e-2, 1e-1]
    ref = oracle_result("r24", 0.01, alpha_given=tuple(given))
    xi, alpha, _ = run(rc, "r24", 0.01, "fp64", solve_form=1, alpha_mode=1, alpha_given=given)
    assert rel_l2(xi, ref.xi) <= 1e-10


def test_batch_rank1_equals_single_calls(rc):
    import torch
    items, singles = [], []
    for name in ("c1", "r24", "r96"):
        g, om, W, _ = case(name, 0.01)
        Wd = torch.from_numpy(np.ascontiguousarray(W)).to(device=rc.device, dtype=torch.complex64)
        items.append((Wd, list(om), _geom(g), 0.01))
        xi, _, _ = rc.reconstruct(Wd, list(om), _geom(g), 0.01, precision="mixed", solve_form=1)
        singles.append(xi.cpu().numpy())
    res = rc.reconstruct_batch(items, "mixed", n_streams=3, solve_form=1)
    torch.cuda.synchronize()
    for (xi, _), ref in zip(res, singles):
        assert np.array_equal(xi.cpu().numpy(), ref)


def test_invalid_combinations(rc):
    from paper_1911_10487_gb300 import FlatLayerError
    with pytest.raises(FlatLayerError, match="FS_EUNSUPPORTED"):
        run(rc, "r12", 0.01, "fp64", regularizer=1)
    with pytest.raises(FlatLayerError, match="FS_EINVAL"):
        run(rc, "r12", 0.01, "fp64", solve_form=1, regularizer=1, alpha_mode=1, alpha_given=[1.0])
    with pytest.raises(FlatLayerError, match="FS_EINVAL"):
        run(rc, "r12", 0.01, "fp64", solve_form=2)
