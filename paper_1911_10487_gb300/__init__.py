"""GB300 (sm_103a) implementation of the flat-layer inverse-acoustics algorithm
(Bakushinsky & Leonov, arXiv 1911.10487, Algorithm 2).

The computation runs in the CUDA library libflatlayer.so behind the C ABI of
include/flatlayer.h; ``_abi`` binds it with ctypes under the same names.
``Reconstructor`` is a convenience layer that uses PyTorch only to hold device
memory and to pick the CUDA stream.  There is no CPU fallback: if the library is
missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import _abi
from ._abi import (FORWARD_METHODS, FS_FP64, FS_MIXED, FlatLayerError, fs_create, fs_default_options, fs_destroy,
                   fs_forward, fs_forward_born, fs_get_report, fs_last_error, fs_reconstruct, fs_reconstruct_batch,
                   fs_reconstruct_host, fs_reconstruct_static, fs_reserve, fs_sync_status, fs_version,
                   fs_workspace_generation, fs_workspace_size,
                   make_geometry, make_options, make_problem)

__all__ = ["Geometry", "KernelPlan", "Reconstructor", "FS_FP64", "FS_MIXED", "FlatLayerError", "fs_create",
           "fs_default_options", "fs_destroy", "fs_forward", "fs_forward_born", "fs_get_report", "fs_last_error", "fs_reconstruct",
           "fs_reconstruct_batch", "fs_reconstruct_host", "fs_reconstruct_static", "fs_reserve", "fs_sync_status",
           "fs_version", "fs_workspace_generation",
           "fs_workspace_size", "make_geometry", "make_options", "make_problem"]

PRECISIONS = {"fp64": FS_FP64, "mixed": FS_MIXED}


@dataclass(frozen=True)
class Geometry:
    """N x N x M grid of X = [-L/2, L/2)^2 x [z1, z2] and the data planes zy (all > z2)."""
    n: int
    m: int
    z1: float
    z2: float
    zy: tuple
    period: float = 2.0

    @property
    def m1(self) -> int:
        return len(self.zy)

    def c_struct(self):
        return make_geometry(self.n, self.m, self.z1, self.z2, self.zy, self.period)


class KernelPlan:
    """Sampled-G kernel tables (Sec. 5: G~ from the FFT of sampled G) for one geometry,
    precision and frequency list; pass it as ``kernel_plan=`` to
    Reconstructor.reconstruct.  Holds (M1 M + M) N^2 n_omega x 16 bytes of device memory."""

    def __init__(self, rc: "Reconstructor", geom: Geometry, omega, precision: str = "fp64", c0: float = 1.0):
        self.geom, self.omega, self.precision, self.c0 = geom, list(omega), precision, c0
        self.handle = _abi.fs_kernel_plan_create(rc.ctx, geom.c_struct(), PRECISIONS[precision], self.omega, c0)

    @property
    def nbytes(self) -> int:
        return _abi.fs_kernel_plan_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            _abi.fs_kernel_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Reconstructor:
    """One library context bound to a CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Reconstructor needs a CUDA GPU")
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = fs_create(device, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            fs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reconstruct(self, W, omega, geom: Geometry, delta: float, c0: float = 1.0,
                    precision: str = "fp64", want_c: bool = True, want_alpha: bool = False,
                    out=None, **options):
        """xi (and c, alpha) from data W[n_omega, M1, N, N] on the device.

        W must be complex128 for precision='fp64' and complex64 for 'mixed'.
        Returns (xi, c, alpha) tensors (c/alpha None unless requested)."""
        import torch
        prec = PRECISIONS[precision]
        want = torch.complex128 if prec == FS_FP64 else torch.complex64
        rdt = torch.float64 if prec == FS_FP64 else torch.float32
        if W.dtype != want or W.device != self.device or not W.is_contiguous():
            raise ValueError(f"W must be a contiguous {want} tensor on {self.device}")
        n_om = len(omega)
        if tuple(W.shape) != (n_om, geom.m1, geom.n, geom.n):
            raise ValueError(f"W shape {tuple(W.shape)} != {(n_om, geom.m1, geom.n, geom.n)}")
        if out is None:
            xi = torch.empty((geom.m, geom.n, geom.n), dtype=rdt, device=self.device)
            c = torch.empty_like(xi) if want_c else None
            alpha = (torch.full((n_om, geom.n, geom.n), float("inf"), dtype=torch.float64,
                                device=self.device) if want_alpha else None)
        else:
            xi, c, alpha = out
        if isinstance(options.get("kernel_plan"), KernelPlan):
            options["kernel_plan"] = options["kernel_plan"].handle
        if "incident" in options and hasattr(options["incident"], "data_ptr"):
            u0 = options["incident"]
            if u0.dtype != W.dtype or tuple(u0.shape) != (n_om, geom.m, geom.n, geom.n) or not u0.is_contiguous():
                raise ValueError("incident must be a contiguous [n_omega, M, N, N] tensor of W's dtype")
            options["incident"] = u0.data_ptr()
        opts = make_options(**options) if options else None
        fs_reconstruct(self.ctx, geom.c_struct(), prec, W.data_ptr(), omega, delta, c0, opts,
                       xi.data_ptr(), c.data_ptr() if c is not None else None,
                       alpha.data_ptr() if alpha is not None else None)
        return xi, c, alpha

    def reconstruct_batch(self, items, precision: str = "fp64", c0: float = 1.0, n_streams: int = 8,
                          outs=None, **options):
        """Independent problems in one call.  items: sequence of (W, omega, geom, delta);
        returns [(xi, c)] (allocated unless `outs` gives them)."""
        import torch
        prec = PRECISIONS[precision]
        want = torch.complex128 if prec == FS_FP64 else torch.complex64
        rdt = torch.float64 if prec == FS_FP64 else torch.float32
        probs, res = [], []
        for j, (W, omega, geom, delta) in enumerate(items):
            if W.dtype != want or W.device != self.device or not W.is_contiguous():
                raise ValueError(f"problem {j}: W must be a contiguous {want} tensor on {self.device}")
            if tuple(W.shape) != (len(omega), geom.m1, geom.n, geom.n):
                raise ValueError(f"problem {j}: W shape does not match its geometry")
            if outs is None:
                xi = torch.empty((geom.m, geom.n, geom.n), dtype=rdt, device=self.device)
                c = torch.empty_like(xi)
            else:
                xi, c = outs[j]
            res.append((xi, c))
            probs.append(make_problem(geom.c_struct(), W.data_ptr(), omega, delta, c0, xi.data_ptr(),
                                      c.data_ptr() if c is not None else None))
        opts = make_options(**options) if options else None
        fs_reconstruct_batch(self.ctx, probs, prec, opts, n_streams)
        return res

    def incident_point_sources(self, sources, omega, geom: Geometry, c0: float = 1.0, precision: str = "fp64"):
        """Incident field u0[n_omega, M, N, N] on the X planes of point sources (x, y, z, a),
        Sec. 5, in the periodic model (grid nodes -L/2 + i L/N)."""
        import torch
        prec = PRECISIONS[precision]
        cdt = torch.complex128 if prec == FS_FP64 else torch.complex64
        u0 = torch.empty((len(omega), geom.m, geom.n, geom.n), dtype=cdt, device=self.device)
        _abi.fs_incident_point_sources(self.ctx, geom.c_struct(), prec, sources, omega, c0, u0.data_ptr())
        return u0

    def forward_born(self, xi, omega, geom: Geometry, c0: float = 1.0, precision: str = "fp64", incident=None):
        """Single-scattering data W[n_omega, M1, N, N] of xi[M, N, N] (device tensors); the
        plane incident wave unless `incident` (u0[n_omega, M, N, N] on X) is given."""
        import torch
        prec = PRECISIONS[precision]
        rdt = torch.float64 if prec == FS_FP64 else torch.float32
        cdt = torch.complex128 if prec == FS_FP64 else torch.complex64
        if xi.dtype != rdt or xi.device != self.device or not xi.is_contiguous():
            raise ValueError(f"xi must be a contiguous {rdt} tensor on {self.device}")
        if tuple(xi.shape) != (geom.m, geom.n, geom.n):
            raise ValueError("xi shape does not match the geometry")
        W = torch.empty((len(omega), geom.m1, geom.n, geom.n), dtype=cdt, device=self.device)
        if incident is not None and (incident.dtype != cdt or tuple(incident.shape) != (len(omega), geom.m, geom.n, geom.n)
                                     or not incident.is_contiguous()):
            raise ValueError("incident must be a contiguous [n_omega, M, N, N] tensor of the working precision")
        fs_forward_born(self.ctx, geom.c_struct(), prec, xi.data_ptr(), omega, c0, W.data_ptr(),
                        incident.data_ptr() if incident is not None else None)
        return W

    def forward(self, xi, omega, geom: Geometry, c0: float = 1.0, precision: str = "fp64", max_iter: int = 500,
                rtol: float = None, want_u: bool = False, method: str = "fixed_point", incident=None):
        """Data W[n_omega, M1, N, N] of xi[M, N, N] with full scattering: method
        "fixed_point" (Algorithm 1, the fixed point of eq. 6, to ||U~_{n+1} - U~_n|| <=
        rtol ||U~0||), "gmres" (restarted GMRES to a relative residual rtol) or
        "fixed_point_gmres" (GMRES where Algorithm 1 fails); rtol defaults to 1e-13 in
        FP64 and 1e-6 in the mixed precision.  Returns (W, u or None, iterations per
        frequency); raises FlatLayerError (FS_ENOCONV) when a frequency does not converge.  The
        plane incident wave unless `incident` (u0[n_omega, M, N, N] on X) is given."""
        import torch
        prec = PRECISIONS[precision]
        rdt = torch.float64 if prec == FS_FP64 else torch.float32
        cdt = torch.complex128 if prec == FS_FP64 else torch.complex64
        if xi.dtype != rdt or xi.device != self.device or not xi.is_contiguous():
            raise ValueError(f"xi must be a contiguous {rdt} tensor on {self.device}")
        if tuple(xi.shape) != (geom.m, geom.n, geom.n):
            raise ValueError("xi shape does not match the geometry")
        if rtol is None:
            rtol = 1e-13 if prec == FS_FP64 else 1e-6
        W = torch.empty((len(omega), geom.m1, geom.n, geom.n), dtype=cdt, device=self.device)
        u = torch.empty((len(omega), geom.m, geom.n, geom.n), dtype=cdt, device=self.device) if want_u else None
        if incident is not None and (incident.dtype != cdt or tuple(incident.shape) != (len(omega), geom.m, geom.n, geom.n)
                                     or not incident.is_contiguous()):
            raise ValueError("incident must be a contiguous [n_omega, M, N, N] tensor of the working precision")
        its = fs_forward(self.ctx, geom.c_struct(), prec, xi.data_ptr(), omega, c0, FORWARD_METHODS[method], max_iter,
                         rtol, W.data_ptr(), u.data_ptr() if u is not None else None,
                         incident.data_ptr() if incident is not None else None)
        return W, u, its

    def report(self) -> dict:
        return fs_get_report(self.ctx)

    def sync_status(self) -> int:
        """fs_status of what the kernels of the last reconstruction found (synchronises)."""
        return fs_sync_status(self.ctx)

    def reserve(self, geom: Geometry, n_omega: int, precision: str = "fp64"):
        """Size the workspace for reconstructions up to this problem (before graph capture)."""
        fs_reserve(self.ctx, geom.c_struct(), n_omega, PRECISIONS[precision])

    def workspace_generation(self) -> int:
        """Reallocations of the workspace so far (a captured graph is stale once it changes)."""
        return fs_workspace_generation(self.ctx)
