"""The allocation-free entry point fs_reconstruct_static.

It exists for callers that cannot call cudaMalloc (a framework that owns all
device memory, or a caller that must not allocate or synchronise once running).
Through the C ABI it must give the same xi as fs_reconstruct, within the parity
tolerances of the other GPU tests, on two calls in a row (the shared scratch
keeps the previous call's contents), and reject a problem too large for its
fixed scratch.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from _cases import case
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}


def _context_result(name, precision, **opts):
    import torch
    from paper_1911_10487_gb300 import Geometry, Reconstructor
    g, om, W, _ = case(name, 0.01)
    geom = Geometry(g.n, g.m, g.z1, g.z2, tuple(g.zy), g.period)
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to("cuda", cdt)
    rc = Reconstructor(0)
    ref, ref_c, _ = rc.reconstruct(Wd, list(om), geom, 0.01, precision=precision, **opts)
    torch.cuda.synchronize()
    out = ref.cpu().numpy(), ref_c.cpu().numpy()
    rc.close()
    return g, om, Wd, out


def _static_call(g, om, Wd, precision, **opts):
    import torch
    from paper_1911_10487_gb300 import FS_FP64, FS_MIXED
    from paper_1911_10487_gb300._abi import FS_OK, fs_reconstruct_static, make_geometry, make_options
    rdt = torch.float64 if precision == "fp64" else torch.float32
    prec = FS_FP64 if precision == "fp64" else FS_MIXED
    gs = make_geometry(g.n, g.m, g.z1, g.z2, g.zy, g.period)
    xi = torch.full((g.m, g.n, g.n), float("nan"), dtype=rdt, device="cuda")
    c = torch.full_like(xi, float("nan"))
    st = fs_reconstruct_static(gs, prec, Wd.data_ptr(), list(om), 0.01, 1.0, make_options(**opts) if opts else None,
                               xi.data_ptr(), c.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == FS_OK
    torch.cuda.synchronize()
    return xi.cpu().numpy(), c.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_entry_matches_context_entry(precision):
    from paper_1911_10487_gb300 import build
    build.build()
    g, om, Wd, (ref, ref_c) = _context_result("c1", precision)
    for call in range(2):
        xi, c = _static_call(g, om, Wd, precision)
        err = rel_l2(xi, ref)
        assert err <= TOL[precision], (call, err)
        assert rel_l2(c, ref_c) <= TOL[precision]


def test_static_entry_sequence_of_problems():
    """Calls of different size, precision and solve form one after the other on the
    shared scratch: the twiddles and counters are rewritten per call and no stale
    contents of a larger earlier call are read."""
    from paper_1911_10487_gb300 import build
    build.build()
    seq = [("r24", "mixed", {}), ("c1", "fp64", {}), ("c1", "fp64", {"solve_form": 1}),
           ("r48", "mixed", {"solve_form": 1, "regularizer": 1}), ("r24", "fp64", {}), ("c1", "mixed", {})]
    for name, precision, opts in seq:
        g, om, Wd, (ref, ref_c) = _context_result(name, precision, **opts)
        xi, c = _static_call(g, om, Wd, precision, **opts)
        err = rel_l2(xi, ref)
        print(f"{name} {precision} {opts}: {err:.2e}")
        assert err <= TOL[precision], (name, precision, opts, err)


def test_static_entry_rejects_oversize_problem():
    import torch
    from paper_1911_10487_gb300 import build
    build.build()
    from paper_1911_10487_gb300._abi import FS_EUNSUPPORTED, FS_FP64, fs_reconstruct_static, make_geometry
    n, m, m1 = 256, 64, 32  # far beyond the 32 MiB scratch in FP64
    gs = make_geometry(n, m, 0.2, 1.0, [1.2 + 0.01 * k for k in range(m1)])
    W = torch.zeros((1, m1, n, n), dtype=torch.complex128, device="cuda")
    xi = torch.zeros((m, n, n), dtype=torch.float64, device="cuda")
    st = fs_reconstruct_static(gs, FS_FP64, W.data_ptr(), [8 * np.pi], 0.01, 1.0, None, xi.data_ptr())
    assert st == FS_EUNSUPPORTED
