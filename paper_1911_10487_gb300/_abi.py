"""ctypes binding of the C ABI in include/flatlayer.h (argument marshalling only).

Every entry point of the header appears here under the same name.  The shared
library must have been built (``paper_1911_10487_gb300.build.build()``); loading
fails loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libflatlayer.so")
_lib = None

FS_OK, FS_EINVAL, FS_ENOMEM, FS_ECUDA, FS_EUNSUPPORTED, FS_ENOCONV, FS_ENONFINITE, FS_ETIMEOUT = range(8)
FS_FP64, FS_MIXED = 0, 1
FS_MIXED_MIN_NOISE = 1e-6  # include/flatlayer.h: smallest max(delta, delta_floor) of a mixed reconstruction
STATUS_NAMES = {0: "FS_OK", 1: "FS_EINVAL", 2: "FS_ENOMEM", 3: "FS_ECUDA", 4: "FS_EUNSUPPORTED", 5: "FS_ENOCONV",
                6: "FS_ENONFINITE", 7: "FS_ETIMEOUT"}

# every function declared in include/*.h
EXPORTS = ("fs_version", "fs_default_options", "fs_create", "fs_destroy", "fs_last_error",
           "fs_workspace_size", "fs_reconstruct", "fs_reconstruct_host", "fs_forward_born", "fs_forward",
           "fs_get_report", "fs_sync_status", "fs_measure_alu_peaks", "fs_eval_reciprocals", "fs_check_bounded_wait", "fs_reconstruct_static", "fs_reconstruct_batch",
           "fs_diff_plan_create", "fs_diff_plan_destroy", "fs_diff_tape_bytes", "fs_diff_scratch_bytes",
           "fs_reconstruct_diff", "fs_reconstruct_vjp", "fs_reconstruct_jvp",
           "fs_kernel_plan_create", "fs_kernel_plan_destroy", "fs_kernel_plan_bytes", "fs_incident_point_sources",
           "fs_reserve", "fs_workspace_generation")


class fs_geometry(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("m1", C.c_int), ("period", C.c_double),
                ("z1", C.c_double), ("z2", C.c_double), ("zy", C.POINTER(C.c_double))]


class fs_options(C.Structure):
    _fields_ = [("tau", C.c_double), ("delta_floor", C.c_double), ("alpha_rel", C.c_double),
                ("eps_u", C.c_double), ("alpha_mode", C.c_int),
                ("alpha_given", C.POINTER(C.c_double)), ("max_iter", C.c_int),
                ("refine_iters", C.c_int), ("fp64_switch", C.c_double), ("stage_timing", C.c_int),
                ("solve_blocks_per_sm", C.c_int), ("solve_form", C.c_int), ("regularizer", C.c_int),
                ("kernel_plan", C.c_void_p), ("classify_single_pass", C.c_int), ("fft_tile", C.c_int),
                ("forward_single_pass", C.c_int), ("inverse_single_pass", C.c_int),
                ("fp64_sums", C.c_int), ("incident", C.c_void_p)]


STAGES = ("fft_x_forward", "fft_y_forward_norms", "classify", "solve", "ifft_y_gather", "ifft_x_recover")


class fs_problem(C.Structure):
    _fields_ = [("geom", fs_geometry), ("W", C.c_void_p), ("omega", C.POINTER(C.c_double)),
                ("n_omega", C.c_int), ("delta", C.c_double), ("c0", C.c_double), ("xi", C.c_void_p),
                ("c", C.c_void_p)]


class fs_report(C.Structure):
    _fields_ = [(k, C.c_longlong) for k in (
        "n_modes", "n_active", "n_zeroed", "n_grazing", "n_alpha_floor", "n_root_capped",
        "n_u_guard", "n_nan_c", "n_fp64_fallback", "n_refine_iters", "n_columns", "n_nonfinite", "n_timeouts")] + \
        [("ms_stage", C.c_float * 6)]

    def as_dict(self):
        d = {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "ms_stage"}
        d["ms_stage"] = dict(zip(STAGES, [float(x) for x in self.ms_stage]))
        return d


class fs_alu_peaks(C.Structure):
    _fields_ = [("fp64_tflops", C.c_double), ("fp32_tflops", C.c_double),
                ("fp64_fma_cycles_1lane", C.c_double), ("fp64_fma_cycles_warp", C.c_double),
                ("fp64_div_cycles_1lane", C.c_double), ("sms", C.c_int), ("clock_mhz", C.c_double)]


class FlatLayerError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libflatlayer.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: build it with paper_1911_10487_gb300.build.build()")
        L = C.CDLL(_LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
        L.fs_version.restype = C.c_char_p
        L.fs_version.argtypes = []
        L.fs_default_options.restype = ip
        L.fs_default_options.argtypes = [C.POINTER(fs_options)]
        L.fs_create.restype = ip
        L.fs_create.argtypes = [C.POINTER(vp), ip, vp]
        L.fs_destroy.restype = None
        L.fs_destroy.argtypes = [vp]
        L.fs_last_error.restype = C.c_char_p
        L.fs_last_error.argtypes = [vp]
        L.fs_workspace_size.restype = ip
        L.fs_workspace_size.argtypes = [C.POINTER(fs_geometry), ip, ip, C.POINTER(C.c_size_t)]
        L.fs_reconstruct.restype = ip
        L.fs_reconstruct.argtypes = [vp, C.POINTER(fs_geometry), ip, vp, dp, ip, C.c_double, C.c_double,
                                     C.POINTER(fs_options), vp, vp, dp]
        L.fs_reconstruct_host.restype = ip
        L.fs_reconstruct_host.argtypes = [vp, C.POINTER(fs_geometry), ip, vp, dp, ip, C.c_double, C.c_double,
                                          C.POINTER(fs_options), vp, vp]
        L.fs_forward_born.restype = ip
        L.fs_forward_born.argtypes = [vp, C.POINTER(fs_geometry), ip, vp, vp, dp, ip, C.c_double, vp]
        L.fs_incident_point_sources.restype = ip
        L.fs_incident_point_sources.argtypes = [vp, C.POINTER(fs_geometry), ip, dp, ip, dp, ip, C.c_double, vp]
        L.fs_forward.restype = ip
        L.fs_forward.argtypes = [vp, C.POINTER(fs_geometry), ip, vp, vp, dp, ip, C.c_double, ip, ip, C.c_double, vp,
                                 vp, C.POINTER(C.c_int)]
        L.fs_reconstruct_batch.restype = ip
        L.fs_reconstruct_batch.argtypes = [vp, C.POINTER(fs_problem), ip, ip, C.POINTER(fs_options), ip]
        L.fs_reconstruct_static.restype = ip
        L.fs_reconstruct_static.argtypes = [C.POINTER(fs_geometry), ip, vp, dp, ip, C.c_double, C.c_double,
                                            C.POINTER(fs_options), vp, vp, vp]
        L.fs_measure_alu_peaks.restype = ip
        L.fs_measure_alu_peaks.argtypes = [ip, C.POINTER(fs_alu_peaks)]
        L.fs_get_report.restype = ip
        L.fs_get_report.argtypes = [vp, C.POINTER(fs_report)]
        L.fs_sync_status.restype = ip
        L.fs_sync_status.argtypes = [vp]
        L.fs_reserve.restype = ip
        L.fs_reserve.argtypes = [vp, C.POINTER(fs_geometry), ip, ip]
        L.fs_workspace_generation.restype = C.c_ulonglong
        L.fs_workspace_generation.argtypes = [vp]
        L.fs_kernel_plan_create.restype = ip
        L.fs_kernel_plan_create.argtypes = [vp, C.POINTER(fs_geometry), ip, dp, ip, C.c_double, C.POINTER(vp)]
        L.fs_kernel_plan_destroy.restype = None
        L.fs_kernel_plan_destroy.argtypes = [vp]
        L.fs_kernel_plan_bytes.restype = C.c_size_t
        L.fs_kernel_plan_bytes.argtypes = [vp]
        L.fs_eval_reciprocals.restype = ip
        L.fs_eval_reciprocals.argtypes = [vp, ip, vp, vp]
        L.fs_check_bounded_wait.restype = ip
        L.fs_check_bounded_wait.argtypes = [ip, C.c_uint, C.POINTER(C.c_longlong)]
        L.fs_diff_plan_create.restype = ip
        L.fs_diff_plan_create.argtypes = [vp, C.POINTER(fs_geometry), ip, dp, ip, C.c_double, C.c_double,
                                          C.POINTER(vp)]
        L.fs_diff_plan_destroy.restype = None
        L.fs_diff_plan_destroy.argtypes = [vp]
        L.fs_diff_tape_bytes.restype = C.c_size_t
        L.fs_diff_tape_bytes.argtypes = [vp]
        L.fs_diff_scratch_bytes.restype = C.c_size_t
        L.fs_diff_scratch_bytes.argtypes = [vp, ip]
        L.fs_reconstruct_diff.restype = ip
        L.fs_reconstruct_diff.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.fs_reconstruct_vjp.restype = ip
        L.fs_reconstruct_vjp.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.fs_reconstruct_jvp.restype = ip
        L.fs_reconstruct_jvp.argtypes = [vp, vp, vp, ip, vp, vp, vp, vp]
        _lib = L
    return _lib


# ---- same-named thin wrappers ---------------------------------------------------

def fs_version() -> str:
    return lib().fs_version().decode()


def fs_default_options() -> fs_options:
    o = fs_options()
    lib().fs_default_options(C.byref(o))
    return o


def fs_create(device: int = 0, stream: int = 0):
    h = C.c_void_p()
    st = lib().fs_create(C.byref(h), int(device), C.c_void_p(stream or None))
    if st != FS_OK:
        raise FlatLayerError(st, f"fs_create(device={device}) failed")
    return h


def fs_destroy(ctx) -> None:
    lib().fs_destroy(ctx)


def fs_last_error(ctx) -> str:
    return lib().fs_last_error(ctx).decode()


def fs_workspace_size(geom: fs_geometry, n_omega: int, prec: int) -> int:
    b = C.c_size_t()
    st = lib().fs_workspace_size(C.byref(geom), int(n_omega), int(prec), C.byref(b))
    if st != FS_OK:
        raise FlatLayerError(st, "fs_workspace_size")
    return int(b.value)


def _check(ctx, st, what):
    if st != FS_OK:
        raise FlatLayerError(st, f"{what}: {fs_last_error(ctx)}")


def fs_reconstruct(ctx, geom, prec, W_ptr, omega, delta, c0, opts, xi_ptr, c_ptr=None, alpha_ptr=None):
    om = (C.c_double * len(omega))(*[float(x) for x in omega])
    st = lib().fs_reconstruct(ctx, C.byref(geom), int(prec), C.c_void_p(W_ptr), om, len(omega),
                              float(delta), float(c0), C.byref(opts) if opts is not None else None,
                              C.c_void_p(xi_ptr), C.c_void_p(c_ptr or None),
                              C.cast(C.c_void_p(alpha_ptr or None), C.POINTER(C.c_double)))
    _check(ctx, st, "fs_reconstruct")


def fs_reconstruct_host(ctx, geom, prec, W_ptr, omega, delta, c0, opts, xi_ptr, c_ptr=None):
    om = (C.c_double * len(omega))(*[float(x) for x in omega])
    st = lib().fs_reconstruct_host(ctx, C.byref(geom), int(prec), C.c_void_p(W_ptr), om, len(omega),
                                   float(delta), float(c0), C.byref(opts) if opts is not None else None,
                                   C.c_void_p(xi_ptr), C.c_void_p(c_ptr or None))
    _check(ctx, st, "fs_reconstruct_host")


def fs_forward_born(ctx, geom, prec, xi_ptr, omega, c0, W_ptr, incident_ptr=None):
    om = (C.c_double * len(omega))(*[float(x) for x in omega])
    st = lib().fs_forward_born(ctx, C.byref(geom), int(prec), C.c_void_p(xi_ptr), C.c_void_p(incident_ptr or None), om,
                               len(omega), float(c0), C.c_void_p(W_ptr))
    _check(ctx, st, "fs_forward_born")


def fs_incident_point_sources(ctx, geom, prec, sources, omega, c0, u0_ptr):
    """sources: sequence of (x, y, z, amplitude)."""
    flat = [float(v) for src in sources for v in src]
    sp = (C.c_double * len(flat))(*flat)
    om = (C.c_double * len(omega))(*[float(x) for x in omega])
    st = lib().fs_incident_point_sources(ctx, C.byref(geom), int(prec), sp, len(sources), om, len(omega), float(c0),
                                         C.c_void_p(u0_ptr))
    _check(ctx, st, "fs_incident_point_sources")


FS_FIXED_POINT, FS_GMRES, FS_FIXED_POINT_GMRES = 0, 1, 2
FORWARD_METHODS = {"fixed_point": FS_FIXED_POINT, "gmres": FS_GMRES, "fixed_point_gmres": FS_FIXED_POINT_GMRES}


def fs_forward(ctx, geom, prec, xi_ptr, omega, c0, method, max_iter, rtol, W_ptr, u_ptr=None, incident_ptr=None):
    """Returns the iterations each frequency took."""
    om = (C.c_double * len(omega))(*[float(x) for x in omega])
    its = (C.c_int * len(omega))()
    st = lib().fs_forward(ctx, C.byref(geom), int(prec), C.c_void_p(xi_ptr), C.c_void_p(incident_ptr or None), om,
                          len(omega), float(c0), int(method), int(max_iter), float(rtol), C.c_void_p(W_ptr),
                          C.c_void_p(u_ptr or None), its)
    _check(ctx, st, "fs_forward")
    return [int(x) for x in its]


def fs_reconstruct_batch(ctx, problems, prec, opts=None, n_streams=8):
    """problems: sequence of fs_problem (keep their buffers alive while the call runs)."""
    arr = (fs_problem * len(problems))(*problems)
    st = lib().fs_reconstruct_batch(ctx, arr, len(problems), int(prec),
                                    C.byref(opts) if opts is not None else None, int(n_streams))
    _check(ctx, st, "fs_reconstruct_batch")


def make_problem(geom, W_ptr, omega, delta, c0, xi_ptr, c_ptr=None) -> fs_problem:
    om = (C.c_double * len(omega))(*[float(x) for x in omega])
    p = fs_problem(geom, C.c_void_p(W_ptr), C.cast(om, C.POINTER(C.c_double)), len(omega), float(delta),
                   float(c0), C.c_void_p(xi_ptr), C.c_void_p(c_ptr or None))
    p._keep = (om, geom)
    return p


def fs_get_report(ctx) -> dict:
    r = fs_report()
    st = lib().fs_get_report(ctx, C.byref(r))
    _check(ctx, st, "fs_get_report")
    return r.as_dict()


def fs_kernel_plan_create(ctx, geom, prec, omega, c0=1.0):
    """Sampled-G kernel tables for this geometry, precision and frequency list (device)."""
    om = (C.c_double * len(omega))(*[float(x) for x in omega])
    plan = C.c_void_p()
    st = lib().fs_kernel_plan_create(ctx, C.byref(geom), int(prec), om, len(omega), float(c0), C.byref(plan))
    _check(ctx, st, "fs_kernel_plan_create")
    return plan


def fs_kernel_plan_destroy(plan) -> None:
    lib().fs_kernel_plan_destroy(plan)


def fs_kernel_plan_bytes(plan) -> int:
    return int(lib().fs_kernel_plan_bytes(plan))


def fs_sync_status(ctx) -> int:
    """Device-side status of the last reconstruction (synchronises); returns the fs_status."""
    return int(lib().fs_sync_status(ctx))


def fs_reserve(ctx, geom, n_omega, prec):
    """Size the context's workspace for fs_reconstruct on this problem (raises on error)."""
    st = lib().fs_reserve(ctx, C.byref(geom), int(n_omega), int(prec))
    if st != FS_OK:
        raise FlatLayerError(st, fs_last_error(ctx))


def fs_workspace_generation(ctx) -> int:
    """Reallocations of the context's workspace so far."""
    return int(lib().fs_workspace_generation(ctx))


def fs_eval_reciprocals(x_ptr, n, out_ptr, stream=0) -> int:
    """The library's reciprocal helpers beside CUDA's 1/x and rsqrt (device pointers)."""
    return int(lib().fs_eval_reciprocals(C.c_void_p(x_ptr), int(n), C.c_void_p(out_ptr), C.c_void_p(stream or None)))


def fs_check_bounded_wait(blocks, polls) -> int:
    """Timeouts counted by a device-side barrier that nothing completes (see the header)."""
    t = C.c_longlong()
    st = lib().fs_check_bounded_wait(int(blocks), int(polls), C.byref(t))
    if st != 0:
        raise FlatLayerError(FS_ECUDA, f"fs_check_bounded_wait returned {st}")
    return int(t.value)


def make_geometry(n, m, z1, z2, zy, period=2.0):
    """fs_geometry for an N x N x M grid; keeps the zy array alive on the struct."""
    zy_arr = (C.c_double * len(zy))(*[float(z) for z in zy])
    g = fs_geometry(int(n), int(m), len(zy), float(period), float(z1), float(z2),
                    C.cast(zy_arr, C.POINTER(C.c_double)))
    g._keep = zy_arr
    return g


def make_options(**kw) -> fs_options:
    """Defaults of fs_default_options, overridden by keyword (alpha_given: sequence)."""
    o = fs_default_options()
    known = {name for name, _ in fs_options._fields_}
    for k, v in kw.items():
        if k not in known:
            raise TypeError(f"unknown fs_options field {k!r}")
        if k == "alpha_given":
            arr = (C.c_double * len(v))(*[float(x) for x in v])
            o.alpha_given = C.cast(arr, C.POINTER(C.c_double))
            o._keep = arr
        elif k in ("kernel_plan", "incident"):
            setattr(o, k, v.value if isinstance(v, C.c_void_p) else v)
        else:
            setattr(o, k, v)
    return o


def fs_measure_alu_peaks(device: int = 0) -> dict:
    r = fs_alu_peaks()
    st = lib().fs_measure_alu_peaks(int(device), C.byref(r))
    if st != 0:
        raise FlatLayerError(st, "fs_measure_alu_peaks")
    return {k: getattr(r, k) for k, _ in r._fields_}


def fs_reconstruct_static(geom, prec, W_ptr, omega, delta, c0, opts, xi_ptr, c_ptr=None, stream=0) -> int:
    """Allocation-free reconstruction (see include/flatlayer.h); returns the fs_status."""
    om = (C.c_double * len(omega))(*[float(x) for x in omega])
    return lib().fs_reconstruct_static(C.byref(geom), int(prec), C.c_void_p(W_ptr), om, len(omega), float(delta),
                                       float(c0), C.byref(opts) if opts is not None else None,
                                       C.c_void_p(xi_ptr), C.c_void_p(c_ptr or None), C.c_void_p(stream or None))


# ---- derivatives at fixed alpha (include/flatlayer_diff.h) -------------------------

def fs_diff_plan_create(ctx, geom, prec, omega, c0=1.0, eps_u=1e-8):
    om = (C.c_double * len(omega))(*[float(x) for x in omega])
    plan = C.c_void_p()
    st = lib().fs_diff_plan_create(ctx, C.byref(geom), int(prec), om, len(omega), float(c0), float(eps_u),
                                   C.byref(plan))
    _check(ctx, st, "fs_diff_plan_create")
    return plan


def fs_diff_plan_destroy(plan) -> None:
    lib().fs_diff_plan_destroy(plan)


def fs_diff_tape_bytes(plan) -> int:
    return int(lib().fs_diff_tape_bytes(plan))


def fs_diff_scratch_bytes(plan, n_dir: int = 1) -> int:
    return int(lib().fs_diff_scratch_bytes(plan, int(n_dir)))


def fs_reconstruct_diff(ctx, plan, tape, scratch, W, log_alpha, xi, c=None, phi=None):
    """Pointer arguments are device addresses (ints) or None; ctx only for errors."""
    st = lib().fs_reconstruct_diff(plan, tape, scratch, W, log_alpha, xi, c, phi)
    _check(ctx, st, "fs_reconstruct_diff")


def fs_reconstruct_vjp(ctx, plan, tape, scratch, grad_xi, grad_phi, grad_W, grad_log_alpha):
    st = lib().fs_reconstruct_vjp(plan, tape, scratch, grad_xi, grad_phi, grad_W, grad_log_alpha)
    _check(ctx, st, "fs_reconstruct_vjp")


def fs_reconstruct_jvp(ctx, plan, tape, scratch, n_dir, dW, dlog_alpha, dxi, dphi=None):
    st = lib().fs_reconstruct_jvp(plan, tape, scratch, int(n_dir), dW, dlog_alpha, dxi, dphi)
    _check(ctx, st, "fs_reconstruct_jvp")
