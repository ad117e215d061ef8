"""Parity on the 128 x 128 x 64 workload itself (32 data planes, k0 = 8 pi, three
Gaussian inclusions) at the three noise levels of that workload, 0, 1 % and 5 %, in
both precisions; the mixed path's FP64 route, forced and as taken at delta = 0; and
the thin data layer of Sec. 5.4 (two planes), where xi is compared in the weight of
its least-squares denominator (see that test).

Tolerances as in test_gpu_parity: xi rel. L2 <= 1e-10 (FS_FP64) and <= 1e-5
(FS_MIXED) against the FP64 oracle on the complex128 data; identical active sets.
At delta = 0 the noise level is delta_floor = 1e-5 (the reading of "0 % noise"):
alpha sits near its floor on the strong modes, where phi is flat in alpha, so alpha
is compared per mode only loosely there (1e-3), as in test_gpu_parity.
"""
import numpy as np
import pytest

from _cases import case, oracle_result
from oracle.metrics import rel_l2
from test_gpu_parity import TOL_FP64, TOL_MIXED, check_against_oracle, run_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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


@pytest.mark.parametrize("delta", [0.0, 0.01, 0.05])
def test_c2_fp64(rc, delta):
    g, om, W, _ = case("c2", delta)
    ref = oracle_result("c2", delta)
    err = check_against_oracle(run_gpu(rc, g, om, W, delta), ref, TOL_FP64,
                               alpha_tol=1e-3 if delta == 0 else 1e-7)
    print(f"c2 fp64 delta={delta}: xi rel L2 {err:.3e}")


@pytest.mark.parametrize("delta", [0.0, 0.01, 0.05])
def test_c2_mixed(rc, delta):
    g, om, W, _ = case("c2", delta)
    ref = oracle_result("c2", delta)
    xi, c, alpha, rep = run_gpu(rc, g, om, W, delta, precision="mixed")
    err = rel_l2(xi, ref.xi)
    act = np.isfinite(alpha)
    print(f"c2 mixed delta={delta}: xi rel L2 {err:.3e}, active {act.sum()}/{ref.active.sum()}, "
          f"fp64 route {rep['n_fp64_fallback']}, refine sweeps {rep['n_refine_iters']}")
    assert err <= TOL_MIXED, err
    assert xi.dtype == np.float32
    # the classification is decided on FP32 norms: equal sets except at a tie
    assert np.sum(act != ref.active) <= 2


def test_mixed_fp64_route_forced(rc):
    """fp64_switch above every alpha/tr sends every active mode to the FP64 route."""
    g, om, W, _ = case("c2", 0.01)
    ref = oracle_result("c2", 0.01)
    xi, c, alpha, rep = run_gpu(rc, g, om, W, 0.01, precision="mixed", fp64_switch=1e300)
    err = rel_l2(xi, ref.xi)
    print(f"forced FP64 route: xi rel L2 {err:.3e}, {rep['n_fp64_fallback']} of {rep['n_active']} modes")
    assert rep["n_fp64_fallback"] == rep["n_active"] > 0
    assert err <= TOL_MIXED


def test_mixed_fp64_route_at_floor_cases(rc):
    """At delta = 0 some modes have alpha at its floor; the mixed path decides and
    solves those in FP64 (the floor case is taken when phi(alpha_floor) >= delta_nu)."""
    g, om, W, _ = case("c2", 0.0)
    ref = oracle_result("c2", 0.0)
    xi, c, alpha, rep = run_gpu(rc, g, om, W, 0.0, precision="mixed")
    print(f"delta 0: floor cases oracle {ref.counts['alpha_floor']}, gpu {rep['n_alpha_floor']}; "
          f"fp64 route {rep['n_fp64_fallback']}")
    assert ref.counts["alpha_floor"] > 0
    assert rep["n_fp64_fallback"] >= ref.counts["alpha_floor"]
    assert rep["n_alpha_floor"] == ref.counts["alpha_floor"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_thin_layer_two_planes(rc, precision):
    """Sec. 5.4: data on two planes 0.01 apart.  With two values per mode the
    discrepancy test (tau = 2) passes about 0.3 % of the pure-noise modes, among them
    strongly evanescent ones (sigma_1 ~ 1e-63 at N = 256): their solutions, amplified
    by 1/sigma, dominate V and u, and xi = Re(conj(u) V)/|u|^2 is then fixed only to the
    relative rounding of those giant terms wherever |u|^2 falls far below its maximum.
    What is determined, and asserted: the active sets (exactly), alpha per mode, and xi
    weighted by the least-squares denominator D = sum_omega |u|^2 -- from xi D = num,
    an error eps in num and D gives ||(xi' - xi) D|| <= 2 eps ||xi D|| -- within the
    FP64 tolerance.  The unweighted error is printed.  Those profiles exceed the FP32
    range, which the mixed path must report (FS_ENONFINITE)."""
    g, om, W, _ = case("thin256", 0.01)
    ref = oracle_result("thin256", 0.01)
    xi, c, alpha, rep = run_gpu(rc, g, om, W, 0.01, precision=precision)
    den = np.sum(np.abs(ref.u) ** 2, axis=0)
    werr = np.linalg.norm((xi - ref.xi) * den) / np.linalg.norm(ref.xi * den)
    act = np.isfinite(alpha)
    print(f"thin layer {precision}: xi weighted by sum |u|^2 {werr:.3e}, unweighted {rel_l2(xi, ref.xi):.3e}; "
          f"active {act.sum()}/{ref.active.sum()}; sum |u|^2 spans {den.min():.1e}..{den.max():.1e}")
    if precision == "fp64":
        assert np.array_equal(act, ref.active)
        ra = np.abs(alpha[ref.active] / ref.alpha[ref.active] - 1)
        print(f"alpha max rel err {ra.max():.2e}")
        assert ra.max() <= 1e-6
        assert rep["n_active"] == int(ref.active.sum())
        assert werr <= TOL_FP64
    else:
        # the noise-mode profiles (|V~| up to ~1e61 here) leave the FP32 range of the mixed
        # path's profiles: the path must say so (FS_ENONFINITE), not return silently
        from paper_1911_10487_gb300._abi import FS_ENONFINITE
        assert np.sum(act != ref.active) <= 2
        assert rc.sync_status() == FS_ENONFINITE
        assert rc.report()["n_nonfinite"] > 0
