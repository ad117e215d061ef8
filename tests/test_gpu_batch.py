"""Batched reconstruction (many uneven problems in one call, fork/join streams):
each problem's xi must equal the single-problem result bit for bit (same kernels,
deterministic arithmetic) and the oracle within the parity tolerances."""
import numpy as np
import pytest

from _cases import case, oracle_result
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu

NAMES = ["c1", "r8", "r12", "r24", "r48", "r96"]


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


def _items(rc, precision):
    import torch
    from paper_1911_10487_gb300 import Geometry
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    out = []
    for nm in NAMES:
        g, om, W, _ = case(nm, 0.01)
        geom = Geometry(g.n, g.m, g.z1, g.z2, tuple(g.zy), g.period)
        out.append((torch.from_numpy(np.ascontiguousarray(W)).to(rc.device, dt), list(om), geom, 0.01))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_single_problem_calls(rc, precision):
    import torch
    items = _items(rc, precision)
    singles = []
    for W, om, geom, d in items:
        xi, _, _ = rc.reconstruct(W, om, geom, d, precision=precision)
        singles.append(xi.cpu().numpy())
    for ns in (1, 5, 16):
        res = rc.reconstruct_batch(items, precision, n_streams=ns)
        torch.cuda.synchronize()
        for nm, (xi, c), ref in zip(NAMES, res, singles):
            assert np.array_equal(xi.cpu().numpy(), ref), (nm, ns)
    rep = rc.report()
    assert rep["n_modes"] == sum(len(om) * g.n * g.n for _, om, g, _ in items)


def test_batch_matches_oracle_fp64(rc):
    import torch
    items = _items(rc, "fp64")
    res = rc.reconstruct_batch(items, "fp64", n_streams=4)
    torch.cuda.synchronize()
    for nm, (xi, _) in zip(NAMES, res):
        err = rel_l2(xi.cpu().numpy(), oracle_result(nm, 0.01).xi)
        assert err <= 1e-10, (nm, err)


def test_batch_reports_the_bad_problem(rc):
    import torch
    from paper_1911_10487_gb300 import FlatLayerError, Geometry
    items = _items(rc, "fp64")[:3]
    W = torch.zeros((1, 2, 16, 16), dtype=torch.complex128, device=rc.device)
    items.append((W, [1.0], Geometry(16, 4, 0.2, 1.0, (0.9, 1.3)), 0.01))  # a data plane inside X
    with pytest.raises(FlatLayerError, match="problem 3"):
        rc.reconstruct_batch(items, "fp64")


def test_tuner_picks_and_caches(rc, tmp_path):
    from paper_1911_10487_gb300.tuner import CANDIDATES, BatchTuner
    items = _items(rc, "mixed")[:3]
    path = str(tmp_path / "tune.json")
    t = BatchTuner(path)
    cfg = t.best(rc, items, "mixed", repeats=1)
    assert cfg in CANDIDATES
    assert BatchTuner(path).best(rc, items, "mixed") == cfg  # read back from the JSON cache
