"""Host logic of the batch autotuner (no GPU): the batch signature and the cache."""
import json

from paper_1911_10487_gb300.tuner import CANDIDATES, BatchTuner, signature
from paper_1911_10487_gb300 import Geometry


def _item(n, m, m1, n_omega):
    g = Geometry(n, m, 0.2, 1.0, tuple(1.2 + 0.01 * k for k in range(m1)))
    return (None, [1.0] * n_omega, g, 0.01)


class _NoGPU:
    """A context that must not be touched when the configuration is cached."""
    def __getattr__(self, name):
        raise AssertionError(f"the tuner used the context ({name}) for a cached batch")


def test_signature_is_a_multiset_per_precision():
    a = [_item(64, 16, 4, 1), _item(128, 32, 8, 2), _item(64, 16, 4, 1)]
    b = [a[1], a[2], a[0]]
    assert signature(a, "mixed") == signature(b, "mixed")
    assert signature(a, "mixed") != signature(a, "fp64")
    assert signature(a, "mixed") != signature(a[:2], "mixed")


def test_cached_configuration_needs_no_timing(tmp_path):
    items = [_item(128, 32, 8, 2), _item(64, 16, 4, 1)]
    path = tmp_path / "tuner.json"
    key = signature(items, "mixed")
    path.write_text(json.dumps({key: {"config": [8, 3, 1, 0], "ms": {"8,3,1,0": 1.0}}}))
    t = BatchTuner(str(path))
    assert t.best(_NoGPU(), items, "mixed") == (8, 3, 1, 0)
    # a fresh tuner without the file has nothing cached
    assert key not in BatchTuner(None).cache


def test_candidates_cover_streams_blocks_per_sm_tiles_and_classification():
    assert sorted({s for s, _, _, _ in CANDIDATES}) == [1, 2, 4, 8, 16, 32, 64]
    assert sorted({b for _, b, _, _ in CANDIDATES}) == [1, 2, 3]
    assert sorted({t for _, _, t, _ in CANDIDATES}) == [0, 1]
    assert sorted({c for _, _, _, c in CANDIDATES}) == [0, 1]
    assert len(CANDIDATES) == len(set(CANDIDATES)) == 84


def test_rank_one_candidates_do_not_vary_the_dense_solve_blocks():
    from paper_1911_10487_gb300.tuner import candidates
    r1 = candidates({"solve_form": 1})
    assert {b for _, b, _, _ in r1} == {1} and len(r1) == len(set(r1)) == 28
    assert candidates() == CANDIDATES
