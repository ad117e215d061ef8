"""The C-ABI library builds, loads and exports every entry point its header
declares; host-only entry points behave as documented (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def abi():
    from paper_1911_10487_gb300 import build
    build.build()
    from paper_1911_10487_gb300 import _abi
    return _abi


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(fs_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_header_declares_expected_entry_points(abi):
    assert declared_functions() == sorted(abi.EXPORTS)


def test_library_exports_every_declared_symbol(abi):
    L = C.CDLL(abi.library_path())
    for name in declared_functions():
        assert hasattr(L, name), name


def test_version_and_defaults(abi):
    assert "sm_103a" in abi.fs_version()
    o = abi.fs_default_options()
    assert (o.tau, o.delta_floor, o.alpha_rel, o.eps_u) == (2.0, 1e-5, 1e-6, 1e-8)
    assert (o.alpha_mode, o.max_iter, o.refine_iters, o.fp64_switch, o.stage_timing) == (0, 100, 8, 1e-4, 0)
    assert o.solve_blocks_per_sm == 2
    assert (o.solve_form, o.regularizer) == (0, 0)
    assert abi.lib().fs_default_options(None) == abi.FS_EINVAL


def test_workspace_size_scales(abi):
    g = abi.make_geometry(32, 16, 0.2, 1.0, [1.2 + 0.05 * k for k in range(8)])
    b64 = abi.fs_workspace_size(g, 1, abi.FS_FP64)
    b32 = abi.fs_workspace_size(g, 1, abi.FS_MIXED)
    assert b64 > b32 > 0
    assert abi.fs_workspace_size(g, 2, abi.FS_FP64) > b64


def test_null_context_is_rejected_without_gpu(abi):
    g = abi.make_geometry(32, 16, 0.2, 1.0, [1.3])
    om = (C.c_double * 1)(1.0)
    st = abi.lib().fs_reconstruct(None, C.byref(g), 0, None, om, 1, 0.0, 1.0, None, None, None, None)
    assert st == abi.FS_EINVAL
    assert abi.lib().fs_get_report(None, None) == abi.FS_EINVAL
    assert abi.fs_last_error(None) == "null context"
    abi.fs_destroy(None)


def test_forward_entry_points_reject_a_null_context_without_gpu(abi):
    g = abi.make_geometry(32, 16, 0.2, 1.0, [1.3])
    om = (C.c_double * 1)(1.0)
    its = (C.c_int * 1)()
    st = abi.lib().fs_forward(None, C.byref(g), 0, None, None, om, 1, 1.0, abi.FS_FIXED_POINT, 10, 1e-13, None, None,
                              its)
    assert st == abi.FS_EINVAL
    st = abi.lib().fs_forward_born(None, C.byref(g), 0, None, None, om, 1, 1.0, None)
    assert st == abi.FS_EINVAL
    assert abi.STATUS_NAMES[abi.FS_ENOCONV] == "FS_ENOCONV"
    assert sorted(abi.FORWARD_METHODS.values()) == [abi.FS_FIXED_POINT, abi.FS_GMRES, abi.FS_FIXED_POINT_GMRES]


def test_transform_options_and_strict_option_names(abi):
    o = abi.fs_default_options()
    assert (o.forward_single_pass, o.inverse_single_pass, o.fp64_sums) == (1, 0, 0)
    with pytest.raises(TypeError):
        abi.make_options(forward_single=1)  # a misspelt field is an error, not a no-op


def test_mixed_noise_limit_is_checked_before_any_device_work(abi):
    """FS_MIXED with the discrepancy principle below FS_MIXED_MIN_NOISE is refused by the
    argument checks (the allocation-free entry runs them before touching the device)."""
    text = open(os.path.join(ROOT, "include", "flatlayer.h")).read()
    assert float(re.search(r"#define FS_MIXED_MIN_NOISE ([0-9.e+-]+)", text).group(1)) == abi.FS_MIXED_MIN_NOISE
    g = abi.make_geometry(32, 16, 0.2, 1.0, [1.2 + 0.05 * k for k in range(8)])
    om = (C.c_double * 1)(1.0)
    L = abi.lib()
    for delta, floor in ((0.0, 1e-10), (0.5 * abi.FS_MIXED_MIN_NOISE, 0.0)):
        o = abi.make_options(delta_floor=floor)
        st = L.fs_reconstruct_static(C.byref(g), abi.FS_MIXED, None, om, 1, delta, 1.0, C.byref(o), None, None, None)
        assert st == abi.FS_EUNSUPPORTED
    # the same arguments pass that check in FP64, and with a given alpha (then fail on the NULL W)
    o = abi.make_options(delta_floor=1e-10)
    assert L.fs_reconstruct_static(C.byref(g), abi.FS_FP64, None, om, 1, 0.0, 1.0, C.byref(o), None, None,
                                   None) == abi.FS_EINVAL
    o = abi.make_options(delta_floor=1e-10, alpha_mode=1, alpha_given=[1e-3])
    assert L.fs_reconstruct_static(C.byref(g), abi.FS_MIXED, None, om, 1, 0.0, 1.0, C.byref(o), None, None,
                                   None) == abi.FS_EINVAL


def test_misaligned_buffers_refused_before_any_device_work(abi):
    """A buffer off its element boundary (W: the complex element, xi and c: the real one)
    is refused with FS_EINVAL by the argument checks; the allocation-free entry runs them
    before touching the device, and the pointers are never dereferenced on the host."""
    g = abi.make_geometry(32, 16, 0.2, 1.0, [1.2 + 0.05 * k for k in range(8)])
    om = (C.c_double * 1)(1.0)
    L = abi.lib()
    base = 1 << 20  # fake addresses: only their alignment is looked at
    for prec, cx, re_ in ((abi.FS_FP64, 16, 8), (abi.FS_MIXED, 8, 4)):
        for W, xi, c in ((base + cx // 2, base, None), (base, base + re_ // 2, None), (base, base, base + 2)):
            st = L.fs_reconstruct_static(C.byref(g), prec, C.c_void_p(W), om, 1, 0.01, 1.0, None,
                                         C.c_void_p(xi), C.c_void_p(c), None)
            assert st == abi.FS_EINVAL, (prec, W - base, xi - base, c)


def test_reserve_and_generation_without_a_context(abi):
    g = abi.make_geometry(32, 16, 0.2, 1.0, [1.3])
    assert abi.lib().fs_reserve(None, C.byref(g), 1, abi.FS_MIXED) == abi.FS_EINVAL
    assert abi.fs_workspace_generation(None) == 0
