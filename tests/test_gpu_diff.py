"""Derivatives of the fixed-alpha reconstruction on the GPU (through the C ABI)
against the oracle's SVD-based derivatives, central differences of the GPU
forward map, and the dot-product test.

Tolerances (relative L2): FS_FP64 1e-10 for xi, Phi, the VJP and the JVP against
the oracle (the per-mode systems are factored in FP64 at a conditioning set by
alpha / ||A||_F^2 >= 1e-4 here); 1e-12 for the dot-product test; 1e-6 for central
differences with h = 1e-6 (truncation ~h^2, round-off ~1e-16/h).  FS_MIXED keeps
the per-mode work in FP64 but carries W, the FFTs and step 3 in FP32: 1e-5.
"""
import numpy as np
import pytest

from _cases import case
from oracle import adjoint
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu

CASES = ["c1", "r24", "r48"]


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


def _log_alpha(g, om):
    """alpha_omega a decade or two below the largest ||A_nu||^2 of the frequency."""
    return np.array([np.log(3e-2 * np.max(np.linalg.svd(o ** 2 * adjoint.data_matrices(o, g),
                                                         compute_uv=False)[..., 0] ** 2)) for o in om])


_ORACLE = {}


def oracle_tape(name):
    if name not in _ORACLE:
        g, om, W, _ = case(name, 0.01)
        la = _log_alpha(g, om)
        _ORACLE[name] = (g, om, W, la, adjoint.forward(W, om, g, la))
    return _ORACLE[name]


def _plan(rc, name, precision):
    from paper_1911_10487_gb300.diff import DiffPlan
    g, om, W, la, t = oracle_tape(name)
    return DiffPlan(rc, _geom(g), om, precision)


def _dev(rc, a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=rc.device, dtype=dtype)


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forward_matches_oracle(rc, name, precision):
    import torch
    g, om, W, la, t = oracle_tape(name)
    plan = _plan(rc, name, precision)
    xi, c, phi, _ = plan.forward(_dev(rc, W, plan.cdt), _dev(rc, la, torch.float64), want_c=True)
    torch.cuda.synchronize()
    tol = 1e-10 if precision == "fp64" else 1e-5
    e_xi, e_phi = rel_l2(xi.double().cpu().numpy(), t.xi), _rel(phi.cpu().numpy(), t.phi)
    print(f"{name} {precision}: xi {e_xi:.2e} phi {e_phi:.2e}")
    assert e_xi <= tol and e_phi <= tol
    cc = c.double().cpu().numpy()
    assert np.allclose(cc, 1.0 / np.sqrt(1.0 - t.xi), rtol=10 * tol, atol=0)
    plan.close()


def test_forward_equals_given_alpha_reconstruction(rc):
    """Same map as fs_reconstruct with alpha_mode = 1 (a different kernel path)."""
    import torch
    g, om, W, la, t = oracle_tape("r24")
    plan = _plan(rc, "r24", "fp64")
    Wd = _dev(rc, W, torch.complex128)
    xi, _, _, _ = plan.forward(Wd, _dev(rc, la, torch.float64))
    xi2, _, _ = rc.reconstruct(Wd, list(om), _geom(g), 0.01, precision="fp64", alpha_mode=1,
                               alpha_given=list(np.exp(la)))
    torch.cuda.synchronize()
    assert rel_l2(xi.cpu().numpy(), xi2.cpu().numpy()) <= 1e-10
    plan.close()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vjp_matches_oracle(rc, name, precision):
    import torch
    g, om, W, la, t = oracle_tape(name)
    rng = np.random.default_rng(5)
    gxi = rng.standard_normal(t.xi.shape)
    gphi = rng.standard_normal(len(om)) / t.phi
    gW_ref, gla_ref = adjoint.vjp(t, gxi, gphi)
    plan = _plan(rc, name, precision)
    _, _, _, tape = plan.forward(_dev(rc, W, plan.cdt), _dev(rc, la, torch.float64))
    gW, gla = plan.vjp(tape, _dev(rc, gxi, plan.rdt), _dev(rc, gphi, torch.float64))
    torch.cuda.synchronize()
    tol = 1e-10 if precision == "fp64" else 1e-5
    e_W, e_a = _rel(gW.cpu().numpy().astype(np.complex128), gW_ref), _rel(gla.cpu().numpy(), gla_ref)
    print(f"{name} {precision}: grad W {e_W:.2e} grad log alpha {e_a:.2e}")
    assert e_W <= tol and e_a <= tol
    plan.close()


@pytest.mark.parametrize("name", CASES)
def test_jvp_matches_oracle(rc, name):
    import torch
    g, om, W, la, t = oracle_tape(name)
    rng = np.random.default_rng(6)
    nd = 3
    dW = rng.standard_normal((nd,) + W.shape) + 1j * rng.standard_normal((nd,) + W.shape)
    dla = rng.standard_normal((nd, len(om)))
    dla[0] = 0.0
    plan = _plan(rc, name, "fp64")
    _, _, _, tape = plan.forward(_dev(rc, W, torch.complex128), _dev(rc, la, torch.float64))
    dxi, dphi = plan.jvp(tape, _dev(rc, dW, torch.complex128), _dev(rc, dla, torch.float64))
    torch.cuda.synchronize()
    for d in range(nd):
        rx, rp = adjoint.jvp(t, dW[d], dla[d])
        e_x, e_p = _rel(dxi[d].cpu().numpy(), rx), _rel(dphi[d].cpu().numpy(), rp)
        print(f"{name} dir {d}: dxi {e_x:.2e} dphi {e_p:.2e}")
        assert e_x <= 1e-10 and e_p <= 1e-10
    plan.close()


def test_dot_product_and_chunking(rc):
    """<J x, y> = <x, J^T y> on the GPU alone, and 20 directions (two launches of
    at most 16) equal the directions run one at a time."""
    import torch
    g, om, W, la, t = oracle_tape("c1")
    plan = _plan(rc, "c1", "fp64")
    rng = np.random.default_rng(9)
    _, _, _, tape = plan.forward(_dev(rc, W, torch.complex128), _dev(rc, la, torch.float64))
    nd = 20
    dW = _dev(rc, rng.standard_normal((nd,) + W.shape) + 1j * rng.standard_normal((nd,) + W.shape),
              torch.complex128)
    dla = _dev(rc, rng.standard_normal((nd, len(om))), torch.float64)
    dxi, dphi = plan.jvp(tape, dW, dla)
    gxi = _dev(rc, rng.standard_normal(t.xi.shape), torch.float64)
    gphi = _dev(rc, rng.standard_normal(len(om)) / t.phi, torch.float64)
    gW, gla = plan.vjp(tape, gxi, gphi)
    for d in (0, 7, 19):
        lhs = float((dxi[d] * gxi).sum() + (dphi[d] * gphi).sum())
        rhs = float((torch.conj(gW) * dW[d]).real.sum() + (gla * dla[d]).sum())
        assert abs(lhs - rhs) <= 1e-12 * float((dxi[d] * gxi).abs().sum() + (dphi[d] * gphi).abs().sum())
        one_x, one_p = plan.jvp(tape, dW[d], dla[d])
        assert torch.equal(one_x, dxi[d]) and torch.equal(one_p, dphi[d])
    plan.close()


def test_jvp_matches_central_differences(rc):
    """FP64 GPU forward map differenced with h = 1e-6 along W and log alpha."""
    import torch
    g, om, W, la, t = oracle_tape("r24")
    plan = _plan(rc, "r24", "fp64")
    rng = np.random.default_rng(10)
    Wd, lad = _dev(rc, W, torch.complex128), _dev(rc, la, torch.float64)
    _, _, _, tape = plan.forward(Wd, lad)
    h = 1e-6
    for kind in ("re", "im", "alpha"):
        if kind == "alpha":
            dW = torch.zeros_like(Wd)
            dla = _dev(rc, rng.standard_normal(len(om)), torch.float64)
        else:
            d = rng.standard_normal(W.shape) + 1j * rng.standard_normal(W.shape)
            d = d.real + 0j if kind == "re" else 1j * d.imag
            dW = _dev(rc, d * np.linalg.norm(W) / np.linalg.norm(d), torch.complex128)
            dla = torch.zeros_like(lad)
        dxi, dphi = plan.jvp(tape, dW, dla)
        xp, _, pp, _ = plan.forward(Wd + h * dW, lad + h * dla)
        xm, _, pm, _ = plan.forward(Wd - h * dW, lad - h * dla)
        fd_x = ((xp - xm) / (2 * h)).cpu().numpy()
        fd_p = ((pp - pm) / (2 * h)).cpu().numpy()
        e_x, e_p = _rel(dxi.cpu().numpy(), fd_x), _rel(dphi.cpu().numpy(), fd_p)
        print(f"{kind}: dxi vs FD {e_x:.2e}, dphi vs FD {e_p:.2e}")
        assert e_x <= 1e-6 and e_p <= 1e-6
    plan.close()


def test_autograd_function(rc):
    import torch
    from paper_1911_10487_gb300.diff import reconstruct_diff
    g, om, W, la, t = oracle_tape("r24")
    plan = _plan(rc, "r24", "fp64")
    Wd = _dev(rc, W, torch.complex128).requires_grad_(True)
    lad = _dev(rc, la, torch.float64).requires_grad_(True)
    xi, phi = reconstruct_diff(Wd, lad, plan)
    w = _dev(rc, np.random.default_rng(11).standard_normal(t.xi.shape), torch.float64)
    loss = (xi * w).sum() + (phi / phi.detach()).sum()
    gW, gla = torch.autograd.grad(loss, (Wd, lad))
    rW, ra = adjoint.vjp(t, w.cpu().numpy(), 1.0 / t.phi)
    assert _rel(gW.cpu().numpy(), rW) <= 1e-10 and _rel(gla.cpu().numpy(), ra) <= 1e-10
    # only log alpha requires grad: W-bar is not formed
    xi, phi = reconstruct_diff(Wd.detach(), lad, plan)
    (gla2,) = torch.autograd.grad(phi.sum(), lad)
    _, ra2 = adjoint.vjp(t, np.zeros_like(t.xi), np.ones(len(om)))
    assert _rel(gla2.cpu().numpy(), ra2) <= 1e-10
    plan.close()


def test_tune_log_alpha_reaches_global_discrepancy(rc):
    import torch
    from paper_1911_10487_gb300.diff import tune_log_alpha
    g, om, W, la, t = oracle_tape("c1")
    target = adjoint.discrepancy_target(W, 0.01)
    root = adjoint.global_discrepancy_log_alpha(W, om, g, target)
    plan = _plan(rc, "c1", "fp64")
    la_t, hist = tune_log_alpha(plan, _dev(rc, W, torch.complex128), _dev(rc, la + 6.0, torch.float64),
                                _dev(rc, target, torch.float64), steps=50)
    la_gpu = la_t.cpu().numpy()
    print("tuned", la_gpu, "root", root, "misfit", hist[-1].item())
    assert np.all(np.abs(np.exp(la_gpu - root) - 1.0) < 1e-6)
    plan.close()


def test_invalid_arguments(rc):
    import torch
    from paper_1911_10487_gb300 import FlatLayerError
    from paper_1911_10487_gb300._abi import fs_reconstruct_jvp
    plan = _plan(rc, "r24", "fp64")
    with pytest.raises(FlatLayerError, match="n_dir"):
        fs_reconstruct_jvp(rc.ctx, plan.plan, None, None, 0, None, None, None)
    with pytest.raises(ValueError):
        plan.forward(torch.zeros((1, 2, 3, 3), dtype=torch.complex128, device=rc.device),
                     torch.zeros(2, dtype=torch.float64, device=rc.device))
    plan.close()
