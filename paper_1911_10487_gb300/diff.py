"""Differentiable fixed-alpha reconstruction (include/flatlayer_diff.h).

The map (W, log alpha_omega) -> (xi, Phi_omega) of Algorithm 2 at a given
Tikhonov parameter per frequency, with Phi_omega = sum_nu ||A_nu V~_nu - W~_nu||^2
the discrepancy of Sec. 4 summed over the modes.  Its forward pass, VJP and JVP
run in the library's kernels; this module only allocates the caller-owned tape
and scratch buffers as PyTorch tensors and wires the calls into autograd.

  plan = DiffPlan(rc, geom, omega, "fp64")
  xi, phi = reconstruct_diff(W, log_alpha, plan)      # differentiable in W, log_alpha
  dxi, dphi = plan.jvp(tape, dW)                      # forward-mode, many directions

Uses built on it: ``tune_log_alpha`` (alpha per frequency by Gauss-Newton-scaled
gradient steps on the misfit sum_omega (Phi_omega / target_omega - 1)^2, whose
root is the global discrepancy principle) and ``jvp_study`` (sensitivity of xi
to data perturbations, Sec. 5.3, as Jacobian-vector products).
"""
from __future__ import annotations

from ._abi import (FS_FP64, fs_diff_plan_create, fs_diff_plan_destroy, fs_diff_scratch_bytes,
                   fs_diff_tape_bytes, fs_reconstruct_diff, fs_reconstruct_jvp, fs_reconstruct_vjp)

_ALIGN = 256


def _aligned(nbytes, device):
    """(tensor, 256-byte aligned device address) holding nbytes."""
    import torch
    buf = torch.empty(nbytes + _ALIGN, dtype=torch.uint8, device=device)
    p = buf.data_ptr()
    return buf, p + (-p) % _ALIGN


class Tape:
    """Caller-owned record of one forward pass (kept alive by autograd)."""

    def __init__(self, plan):
        self.buf, self.ptr = _aligned(plan.tape_bytes, plan.device)


class DiffPlan:
    """Normal matrices of one geometry / frequency list / precision, plus buffers."""

    def __init__(self, rc, geom, omega, precision: str = "fp64", c0: float = 1.0, eps_u: float = 1e-8):
        import torch
        from . import PRECISIONS
        self.rc, self.geom, self.omega = rc, geom, [float(x) for x in omega]
        self.prec = PRECISIONS[precision]
        self.device = rc.device
        self.cdt = torch.complex128 if self.prec == FS_FP64 else torch.complex64
        self.rdt = torch.float64 if self.prec == FS_FP64 else torch.float32
        self.plan = fs_diff_plan_create(rc.ctx, geom.c_struct(), self.prec, self.omega, c0, eps_u)
        self.tape_bytes = fs_diff_tape_bytes(self.plan)
        self._scratch = {}

    def close(self):
        if getattr(self, "plan", None) is not None:
            fs_diff_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def scratch(self, n_dir: int = 1) -> int:
        """Address of a scratch buffer for n_dir JVP directions (reused: calls are
        ordered on the context's stream)."""
        k = min(max(n_dir, 1), 16)
        if k not in self._scratch:
            self._scratch[k] = _aligned(fs_diff_scratch_bytes(self.plan, k), self.device)
        return self._scratch[k][1]

    def _check_W(self, W, lead=()):
        g = self.geom
        shape = tuple(lead) + (len(self.omega), g.m1, g.n, g.n)
        if W.dtype != self.cdt or W.device != self.device or not W.is_contiguous() or tuple(W.shape) != shape:
            raise ValueError(f"expected a contiguous {self.cdt} tensor of shape {shape} on {self.device}")

    def _check_la(self, la, lead=()):
        import torch
        shape = tuple(lead) + (len(self.omega),)
        if la.dtype != torch.float64 or la.device != self.device or not la.is_contiguous() or tuple(la.shape) != shape:
            raise ValueError(f"log alpha must be a contiguous float64 tensor of shape {shape} on {self.device}")

    def forward(self, W, log_alpha, tape: Tape | None = None, want_c: bool = False):
        """(xi, c or None, phi, tape) at alpha = exp(log_alpha)."""
        import torch
        self._check_W(W)
        self._check_la(log_alpha)
        g = self.geom
        tape = tape or Tape(self)
        xi = torch.empty((g.m, g.n, g.n), dtype=self.rdt, device=self.device)
        c = torch.empty_like(xi) if want_c else None
        phi = torch.empty(len(self.omega), dtype=torch.float64, device=self.device)
        fs_reconstruct_diff(self.rc.ctx, self.plan, tape.ptr, self.scratch(1), W.data_ptr(), log_alpha.data_ptr(),
                            xi.data_ptr(), c.data_ptr() if c is not None else None, phi.data_ptr())
        return xi, c, phi, tape

    def vjp(self, tape: Tape, grad_xi=None, grad_phi=None, want_W: bool = True, want_alpha: bool = True):
        """(grad W or None, grad log alpha or None) of <grad_xi, xi> + <grad_phi, phi>."""
        import torch
        g = self.geom
        if grad_xi is not None:
            grad_xi = grad_xi.to(self.rdt).contiguous()
        if grad_phi is not None:
            grad_phi = grad_phi.to(torch.float64).contiguous()
        gW = torch.empty((len(self.omega), g.m1, g.n, g.n), dtype=self.cdt, device=self.device) if want_W else None
        gla = torch.empty(len(self.omega), dtype=torch.float64, device=self.device) if want_alpha else None
        fs_reconstruct_vjp(self.rc.ctx, self.plan, tape.ptr, self.scratch(1),
                           grad_xi.data_ptr() if grad_xi is not None else None,
                           grad_phi.data_ptr() if grad_phi is not None else None,
                           gW.data_ptr() if gW is not None else None, gla.data_ptr() if gla is not None else None)
        return gW, gla

    def jvp(self, tape: Tape, dW, dlog_alpha=None):
        """(dxi [n_dir, M, N, N], dphi [n_dir, n_omega]) for dW [n_dir, n_omega, M1, N, N]
        (a single direction may omit the leading axis)."""
        import torch
        single = dW.dim() == 4
        if single:
            dW = dW.unsqueeze(0)
            if dlog_alpha is not None:
                dlog_alpha = dlog_alpha.unsqueeze(0)
        nd = dW.shape[0]
        self._check_W(dW, (nd,))
        if dlog_alpha is not None:
            self._check_la(dlog_alpha, (nd,))
        g = self.geom
        dxi = torch.empty((nd, g.m, g.n, g.n), dtype=self.rdt, device=self.device)
        dphi = torch.empty((nd, len(self.omega)), dtype=torch.float64, device=self.device)
        fs_reconstruct_jvp(self.rc.ctx, self.plan, tape.ptr, self.scratch(nd), nd, dW.data_ptr(),
                           dlog_alpha.data_ptr() if dlog_alpha is not None else None, dxi.data_ptr(),
                           dphi.data_ptr())
        return (dxi[0], dphi[0]) if single else (dxi, dphi)


def _function():
    import torch

    class ReconstructFixedAlpha(torch.autograd.Function):
        """(W, log_alpha) -> (xi, phi); backward through the library's VJP."""

        @staticmethod
        def forward(ctx, W, log_alpha, plan):
            ctx.set_materialize_grads(False)
            xi, _, phi, tape = plan.forward(W.detach(), log_alpha.detach())
            ctx.plan, ctx.tape = plan, tape
            return xi, phi

        @staticmethod
        def backward(ctx, gxi, gphi):
            if gxi is None and gphi is None:
                return None, None, None
            gW, gla = ctx.plan.vjp(ctx.tape, gxi, gphi, want_W=ctx.needs_input_grad[0],
                                   want_alpha=ctx.needs_input_grad[1])
            return gW, gla, None

    return ReconstructFixedAlpha


_FN = None


def reconstruct_diff(W, log_alpha, plan: DiffPlan):
    """Differentiable (xi, phi) of the fixed-alpha reconstruction."""
    global _FN
    if _FN is None:
        _FN = _function()
    return _FN.apply(W, log_alpha, plan)


def gauss_newton_step(r, J, max_step=2.0):
    """Step on log alpha for the misfit sum (r_omega)^2, r = Phi/target - 1, with
    J = dr/dlog alpha (diagonal: Phi_omega depends on alpha_omega only): the
    gradient 2 r J scaled by the Gauss-Newton curvature 2 J^2, clipped to
    +-max_step.  Works on numpy arrays and torch tensors alike."""
    step = -(2 * r * J) / (2 * J * J)
    return step.clip(-max_step, max_step)


def tune_log_alpha(plan: DiffPlan, W, log_alpha0, target, steps: int = 50, max_step: float = 2.0):
    """alpha per frequency with Phi_omega(alpha) = target_omega (the global
    discrepancy principle), by `steps` Gauss-Newton-scaled gradient steps on the
    misfit; gradients from the library's VJP.  Returns (log_alpha, history of the
    misfit) as device tensors; no host synchronisation inside the loop."""
    import torch
    la = log_alpha0.detach().clone().to(torch.float64)
    target = target.to(torch.float64)
    hist = []
    for _ in range(steps):
        xi, _, phi, tape = plan.forward(W, la)
        r = phi / target - 1.0
        _, J = plan.vjp(tape, None, 1.0 / target, want_W=False, want_alpha=True)  # dr/dlog alpha
        hist.append((r * r).sum())
        la = la + gauss_newton_step(r, J, max_step)
    return la, torch.stack(hist)


def jvp_study(plan: DiffPlan, tape: Tape, W, directions, xi):
    """Sensitivity of xi to data perturbations (Sec. 5.3) as JVPs.
    directions: [n_dir, n_omega, M1, N, N] perturbations of W.  Returns
    (dxi [n_dir, M, N, N], amplification ||dxi||/||xi|| / (||dW||/||W||) [n_dir])."""
    import torch
    dxi, _ = plan.jvp(tape, directions)
    nd = directions.shape[0]
    rel_in = torch.linalg.vector_norm(directions.reshape(nd, -1), dim=1) / torch.linalg.vector_norm(W)
    rel_out = torch.linalg.vector_norm(dxi.reshape(nd, -1).double(), dim=1) / torch.linalg.vector_norm(xi.double())
    return dxi, rel_out / rel_in
