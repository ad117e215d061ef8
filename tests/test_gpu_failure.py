"""Failure reporting of the device path, with failures made on the host (no GPU
fault): a NaN or Inf planted in the data W is found by the kernels and reported by
fs_sync_status (FS_ENONFINITE) and fs_report.n_nonfinite, and the next clean call on
the same context reports FS_OK again.  Also the scalar reciprocals that replace FP64
division and square root in the kernels, against CUDA's own 1/x and rsqrt(x) over
the whole exponent range, including the paths that fall back to the division."""
import numpy as np
import pytest

from _cases import case

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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_data_reported(rc, precision, bad):
    import torch
    from paper_1911_10487_gb300._abi import FS_ENONFINITE, FS_OK
    g, om, W, _ = case("r24", 0.01)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(device=rc.device, dtype=dt)
    rc.reconstruct(Wd, list(om), _geom(g), 0.01, precision=precision)
    assert rc.sync_status() == FS_OK
    assert rc.report()["n_nonfinite"] == 0
    Wb = Wd.clone()
    Wb[1, 2, 5, 7] = complex(bad, 0.0)  # one value of the second frequency
    xi, _, _ = rc.reconstruct(Wb, list(om), _geom(g), 0.01, precision=precision)
    assert rc.sync_status() == FS_ENONFINITE
    rep = rc.report()
    print(rep)
    assert rep["n_nonfinite"] >= 1
    # a NaN spreads over every mode of its frequency through the transform; an Inf
    # at least over its row and column
    assert rep["n_nonfinite"] <= g.n * g.n
    rc.reconstruct(Wd, list(om), _geom(g), 0.01, precision=precision)
    assert rc.sync_status() == FS_OK


def test_nonfinite_batch_reported(rc):
    import torch
    from paper_1911_10487_gb300._abi import FS_ENONFINITE, FS_OK
    items = []
    for name in ("r12", "r24"):
        g, om, W, _ = case(name, 0.01)
        items.append((torch.from_numpy(np.ascontiguousarray(W)).to(rc.device), list(om), _geom(g), 0.01))
    rc.reconstruct_batch(items, "fp64", n_streams=2)
    assert rc.sync_status() == FS_OK
    items[1][0][0, 0, 0, 0] = complex(float("nan"), 0.0)
    rc.reconstruct_batch(items, "fp64", n_streams=2)
    assert rc.sync_status() == FS_ENONFINITE


def ulp_err(a, b):
    """|a - b| in units of the last place of b (float64)."""
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_reciprocals_match_cuda():
    import torch
    from paper_1911_10487_gb300 import build
    build.build()
    from paper_1911_10487_gb300._abi import fs_eval_reciprocals
    rng = np.random.default_rng(5)
    tiny = np.finfo(np.float64).tiny
    # every binade from the smallest normal to the largest, random mantissas, both signs
    # for the reciprocal; plus the edges: subnormal inputs, results that leave the
    # normal range (1/x below tiny), h = +-511 of rsqrt64's exponent split, and 1, 2, 4
    ex = np.arange(-1022, 1024)
    x = np.ldexp(1.0 + rng.random(ex.size), ex)
    edges = np.array([tiny, 2 * tiny, np.nextafter(tiny, 0), 5e-324, 1e-310, np.finfo(np.float64).max,
                      np.ldexp(1.0, 1022), np.ldexp(1.5, 1023), np.ldexp(1.0, -1022), np.ldexp(1.0, -1021),
                      1.0, 2.0, 4.0, 0.5, 3.0])
    pos = np.concatenate([x, edges])
    allx = np.concatenate([pos, -pos])
    xd = torch.from_numpy(allx).cuda()
    out = torch.empty((6, allx.size), dtype=torch.float64, device="cuda")
    assert fs_eval_reciprocals(xd.data_ptr(), allx.size, out.data_ptr()) == 0
    torch.cuda.synchronize()
    rcp64, div, rsq64, rsq, rcp32, rsq32 = out.cpu().numpy()
    normal_res = (np.abs(div) >= tiny) & np.isfinite(div)
    e_rcp = ulp_err(rcp64[normal_res], div[normal_res])
    print(f"rcp64: max {e_rcp.max():.2f} ulp over {normal_res.sum()} inputs")
    assert e_rcp.max() <= 1.0
    # where 1/x is subnormal or infinite (x subnormal), rcp64 falls back to the division
    assert np.array_equal(rcp64[~normal_res], div[~normal_res])
    p = slice(0, pos.size)
    e_rsq = ulp_err(rsq64[p], rsq[p])
    print(f"rsqrt64: max {e_rsq.max():.2f} ulp vs CUDA rsqrt")
    assert e_rsq.max() <= 2.0
    # against the exactly rounded value (rsqrt itself is within 1 ulp of it)
    ref = 1.0 / np.sqrt(pos)
    assert ulp_err(rsq64[p], ref).max() <= 2.0
    # FP32-accurate versions: relative error within a few FP32 ulps at every exponent
    rel32 = np.abs(rcp32[normal_res] / div[normal_res] - 1)
    assert np.array_equal(rcp32[~normal_res], div[~normal_res])
    assert rel32.max() <= 2.5e-7, rel32.max()
    rel32s = np.abs(rsq32[p] / ref - 1)
    assert rel32s.max() <= 2.5e-7, rel32s.max()
    # negative inputs: rsqrt64 and rsqrt32 return what 1/sqrt(x) gives (NaN)
    assert np.all(np.isnan(rsq64[pos.size:])) and np.all(np.isnan(rsq32[pos.size:]))


def test_bounded_wait_runs_out_and_the_context_stays_usable(rc):
    """A device-side barrier that nothing completes (its target exceeds the grid): each
    block's wait gives up after its poll limit and counts a timeout; the GPU context is
    usable afterwards (a reconstruction runs and reports FS_OK)."""
    import torch
    from paper_1911_10487_gb300._abi import FS_OK, fs_check_bounded_wait
    assert fs_check_bounded_wait(4, 2000) == 4
    g, om, W, _ = case("r24", 0.01)
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(rc.device)
    rc.reconstruct(Wd, list(om), _geom(g), 0.01)
    assert rc.sync_status() == FS_OK
    assert rc.report()["n_timeouts"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["c1", "r12", "r48", "r256"])
def test_single_pass_classification_equals_three_kernel_form(rc, name, precision):
    """The cooperative single-pass classification and the three-kernel form decide the
    same modes; xi agrees to the rounding of ||W||^2 (grouped differently)."""
    import torch
    g, om, W, _ = case(name, 0.01)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(device=rc.device, dtype=dt)
    out = []
    for single in (1, 0):
        xi, _, alpha = rc.reconstruct(Wd, list(om), _geom(g), 0.01, precision=precision, want_alpha=True,
                                      classify_single_pass=single)
        torch.cuda.synchronize()
        out.append((xi.double().cpu().numpy(), np.isfinite(alpha.cpu().numpy()), rc.report()))
    (x1, a1, r1), (x0, a0, r0) = out
    assert np.array_equal(a1, a0)
    assert r1["n_active"] == r0["n_active"] and r1["n_columns"] == r0["n_columns"]
    assert r1["n_timeouts"] == 0
    from oracle.metrics import rel_l2
    assert rel_l2(x1, x0) <= (1e-12 if precision == "fp64" else 1e-6)


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_workspace_reserve_generation_and_growth_during_capture():
    """fs_reserve sizes the workspace once (the generation counts the reallocation), calls
    up to that size allocate nothing, and a call that would grow the workspace while the
    stream is captured is refused with FS_EUNSUPPORTED instead of freeing memory a graph
    refers to."""
    import torch
    from paper_1911_10487_gb300 import FlatLayerError, Reconstructor
    from paper_1911_10487_gb300._abi import FS_EUNSUPPORTED
    rc = Reconstructor(0, stream=torch.cuda.Stream())
    try:
        g_small, om_s, W_s, _ = case("r24", 0.01)
        g_big, om_b, W_b, _ = case("r48", 0.01)
        gen0 = rc.workspace_generation()
        rc.reserve(_geom(g_small), len(om_s), "mixed")
        assert rc.workspace_generation() == gen0 + 1
        rc.reserve(_geom(g_small), len(om_s), "mixed")  # already large enough
        assert rc.workspace_generation() == gen0 + 1
        Ws = torch.from_numpy(np.ascontiguousarray(W_s)).to(rc.device, torch.complex64)
        Wb = torch.from_numpy(np.ascontiguousarray(W_b)).to(rc.device, torch.complex64)
        xi = torch.empty((g_big.m, g_big.n, g_big.n), dtype=torch.float32, device=rc.device)
        with torch.cuda.stream(rc.stream):
            rc.reconstruct(Ws, list(om_s), _geom(g_small), 0.01, precision="mixed")
        torch.cuda.synchronize()
        assert rc.workspace_generation() == gen0 + 1
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=rc.stream):
            with pytest.raises(FlatLayerError) as ei:
                rc.reconstruct(Wb, list(om_b), _geom(g_big), 0.01, precision="mixed", out=(xi, None, None))
        assert ei.value.status == FS_EUNSUPPORTED
        assert rc.workspace_generation() == gen0 + 1
        torch.cuda.synchronize()
    finally:
        rc.close()
