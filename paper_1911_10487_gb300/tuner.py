"""Autotuner for batched reconstructions.

For a batch signature (the sorted multiset of (N, M, M1, n_omega) and the
precision) it times the candidate launch configurations -- the number of
concurrent streams the batch is dealt over and the resident blocks per SM of the
per-mode solve -- with CUDA events on the library's stream, and keeps the fastest.
Results are cached in memory and, if a path is given, in a JSON file.
"""
from __future__ import annotations

import json
import os

CANDIDATES = [(s, b) for s in (1, 2, 4, 8, 16) for b in (1, 2, 3)]


def signature(items, precision):
    key = sorted((g.n, g.m, g.m1, len(om)) for (_, om, g, _) in items)
    return f"{precision}:" + ";".join("x".join(map(str, k)) for k in key)


class BatchTuner:
    def __init__(self, path: str | None = None):
        self.path = path
        self.cache = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = json.load(f)

    def best(self, rc, items, precision="mixed", repeats=3, outs=None):
        """(n_streams, solve_blocks_per_sm) for this batch, timing it if unseen."""
        import torch
        key = signature(items, precision)
        if key in self.cache:
            return tuple(self.cache[key]["config"])
        timings = {}
        with torch.cuda.stream(rc.stream):
            for s, b in CANDIDATES:
                rc.reconstruct_batch(items, precision, n_streams=s, outs=outs, solve_blocks_per_sm=b)  # warm
                t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0.record(rc.stream)
                for _ in range(repeats):
                    rc.reconstruct_batch(items, precision, n_streams=s, outs=outs, solve_blocks_per_sm=b)
                t1.record(rc.stream)
                t1.synchronize()
                timings[f"{s},{b}"] = t0.elapsed_time(t1) / repeats
        best = min(timings, key=timings.get)
        cfg = tuple(int(x) for x in best.split(","))
        self.cache[key] = {"config": list(cfg), "ms": timings}
        if self.path:
            with open(self.path, "w") as f:
                json.dump(self.cache, f, indent=1)
        return cfg
