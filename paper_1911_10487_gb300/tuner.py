"""Autotuner for batched reconstructions.

For a batch signature (the sorted multiset of (N, M, M1, n_omega) and the
precision) it times the candidate launch configurations -- the number of
concurrent streams the batch is dealt over (1 to 64), the resident blocks per SM of
the dense per-mode solve, the tile shape of the transform passes (fs_options.fft_tile:
2048-element tiles with radix cap 16, or 1024-element tiles with radix cap 8) and
the form of the classification (fs_options.classify_single_pass: three kernels, or
one cooperative launch) --
with CUDA events on the library's stream, and keeps the fastest.  The signature
ignores the plane heights and the noise level: they change neither the launch
shapes nor the work per mode of the transforms.  Results are cached in memory and,
if a path is given, in a JSON file.
"""
from __future__ import annotations

import json
import os

STREAMS = (1, 2, 4, 8, 16, 32, 64)
CANDIDATES = [(s, b, t, c) for s in STREAMS for b in (1, 2, 3) for t in (0, 1) for c in (0, 1)]


def candidates(options=None):
    """The candidate configurations for a batch; resident blocks per SM only matter to
    the dense per-mode solve, so with the rank-one form (solve_form 1) they are not
    varied."""
    if (options or {}).get("solve_form") == 1:
        return [(s, 1, t, c) for s in STREAMS for t in (0, 1) for c in (0, 1)]
    return list(CANDIDATES)


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

    def best(self, rc, items, precision="mixed", repeats=3, outs=None, options=None):
        """(n_streams, solve_blocks_per_sm, fft_tile, classify_single_pass) for this batch,
        timing it if unseen.  options: further fs_options fields, fixed for every
        candidate (part of the cache key)."""
        import torch
        options = dict(options or {})
        key = signature(items, precision)
        if options:
            key += "|" + ",".join(f"{k}={v}" for k, v in sorted(options.items()))
        if key in self.cache:
            return tuple(self.cache[key]["config"])
        timings = {}
        with torch.cuda.stream(rc.stream):
            for s, b, t, c in candidates(options):
                kw = dict(n_streams=s, outs=outs, solve_blocks_per_sm=b, fft_tile=t, classify_single_pass=c,
                          **options)
                rc.reconstruct_batch(items, precision, **kw)  # warm
                t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0.record(rc.stream)
                for _ in range(repeats):
                    rc.reconstruct_batch(items, precision, **kw)
                t1.record(rc.stream)
                t1.synchronize()
                timings[f"{s},{b},{t},{c}"] = t0.elapsed_time(t1) / repeats
        best = min(timings, key=timings.get)
        cfg = tuple(int(x) for x in best.split(","))
        self.cache[key] = {"config": list(cfg), "ms": timings}
        if self.path:
            with open(self.path, "w") as f:
                json.dump(self.cache, f, indent=1)
        return cfg
