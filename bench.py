#!/usr/bin/env python
"""Throughput of the flat-layer reconstruction (Algorithm 2) on one GB300.

Workload: single frequency k0 = 8 pi, X grid 128 x 128 x 64 in [-1,1]^2 x [0.2,1.0],
32 data planes in [1.2, 1.6], xi = 3 seeded Gaussian inclusions (widths 0.05-0.2,
peaks +-0.1), 1% noise.  Data W are made on the device by the library's own
single-scattering forward kernel (synthetic; no dataset).

A step = one full reconstruction W -> (xi, c): 2D FFT of the data planes, mode
norms, discrepancy classification, per-mode Tikhonov solve + eq. (9), inverse FFTs
and the pointwise xi/c recovery, replayed as one CUDA graph.  The headline is the
mixed-precision path with the rank-one closed form of the per-mode problem (exact
for the Weyl kernel); the plain FP64 path is measured in the same run, and both
again with the dense per-mode solve (`dense_form`).  L2 is flushed (256 MiB write)
before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU FP64 oracle on the same workload (one full
reconstruction per step, data made by the oracle itself).  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ξ voxel·frequencies/s: mixed/batched vs plain FP64 path at stated error vs oracle"
UNIT = "voxel*freq/s"
WORKLOAD = "c2"
DELTA = 0.01
FLUSH_BYTES = 256 << 20
STAGES = ("fft_x_forward", "fft_y_forward_norms", "classify", "solve", "ifft_y_gather", "ifft_x_recover")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch on this workload,
# from one ncu capture of the current kernels (None: not captured since the kernel
# changed); to be measured again whenever a kernel changes
SOLVE_DRAM_BYTES = 237056  # k_solve<float> (dense form, mixed): 237 KB read, nothing written
STAGE_DRAM_BYTES = {"ifft_x_recover": 4249600}  # k_ifft_rows_recover<float>: 4.25 MB read, writes stay in L2
STAGE_KERNELS = {"fft_x_forward": "k_fft2_plane<float>", "fft_y_forward_norms": "k_mode_norms<float>",
                 "classify": "k_classify_flags + k_classify_scatter", "ifft_y_gather": "k_ifft_cols_gather<float>",
                 "ifft_x_recover": "k_ifft_rows_recover<float>"}
HEAD_FORM = 1  # the headline's per-mode solver: the rank-one closed form
# kernels of one mixed step: 2D FFT (one pass at N <= 128, two beyond), mode norms,
# classify (flags, scatter), solve, gather + y-IFFT, x-IFFT + recover; the plain FP64
# path transforms in two passes
KERNELS_PER_STEP_MIXED = 7
KERNELS_PER_STEP = 8


def mixed_kernels(n):
    return KERNELS_PER_STEP_MIXED + (1 if n > 128 else 0)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, ms_local, world):
    """Whole-job throughput of `world` replicas that each process units_per_rank in
    ms_local: all units over the slowest rank's time (weak scaling, max over ranks)."""
    ms = max_over_ranks(ms_local, world)
    return world * units_per_rank / (ms * 1e-3), ms


def make_inputs(rc, wl, geom):
    """Noisy data W (complex128, device): library forward kernel + seeded noise."""
    import torch
    xi = torch.from_numpy(np.ascontiguousarray(wl.xi)).to(rc.device)
    W = rc.forward_born(xi, list(wl.omegas), geom, precision="fp64")
    n = torch.from_numpy(wl.noise()).to(rc.device)
    for j in range(W.shape[0]):
        W[j] += DELTA * torch.linalg.vector_norm(W[j]) * n[j] / torch.linalg.vector_norm(n[j])
    torch.cuda.synchronize()
    return W


def algorithmic_bytes(stage, wl, rep, sc, single=False):
    """Bytes a stage must move at minimum (one launch), sc = bytes per complex; single:
    the forward 2D transform in one pass (the mixed path), so that its first stage is the
    whole transform and the second the mode norms alone."""
    F, N2, M, M1 = len(wl.omegas), wl.n * wl.n, wl.m, wl.m1
    sr = sc // 2
    act, cols = rep["n_active"], rep["n_columns"]
    data = F * M1 * N2 * sc
    if stage == "fft_x_forward":
        return 2 * data
    if stage == "fft_y_forward_norms":
        return (0 if single else 2 * data) + data + 8 * F * N2
    if stage == "classify":
        return 8 * F * N2 + 4 * F * N2 + 4 * act
    if stage == "solve":
        return act * (M1 + 2 * M) * sc
    if stage == "ifft_y_gather":
        return 4 * F * N2 + act * 2 * M * sc + 2 * M * wl.n * cols * sc
    if stage == "ifft_x_recover":
        return 2 * M * wl.n * cols * sc + 2 * M * N2 * sr
    raise KeyError(stage)


def stage_flops(stage, wl, rep, single=False):
    """Real flops of a stage's transforms for one launch (5 L log2 L per complex line of
    length L); the solve's count is solve_flops; classification does no flops.  single:
    as in algorithmic_bytes."""
    F, N, M, M1 = len(wl.omegas), wl.n, wl.m, wl.m1
    line = 5.0 * N * np.log2(N)
    if stage == "fft_x_forward":
        return (2 if single else 1) * F * M1 * N * line
    if stage == "fft_y_forward_norms":
        return 0.0 if single else F * M1 * N * line
    if stage == "ifft_y_gather":
        return F * 2 * M * rep["n_columns"] * line
    if stage == "ifft_x_recover":
        return F * 2 * M * N * line
    if stage == "solve":
        return solve_flops(wl, rep)
    return 0.0


def solve_flops(wl, rep, iters=8):
    """Algorithmic real flops of the per-mode solve for one launch: per active mode,
    kernel assembly 6 M1 M, normal matrix 4 M1^2 M, I_alpha evaluations of the
    discrepancy (4/3 M1^3 + 16 M1^2 each, the cost of one Hermitian factorisation and
    two triangular solves) and V~ = A^H y 8 M1 M."""
    M, M1 = wl.m, wl.m1
    per = 6 * M1 * M + 4 * M1 * M1 * M + iters * (4 * M1 ** 3 / 3 + 16 * M1 * M1) + 8 * M1 * M
    return rep["n_active"] * per


def run_ours(args, rank, world, local):
    import torch
    from paper_1911_10487_gb300 import Geometry, Reconstructor, fs_reconstruct_host, FS_MIXED, build
    from paper_1911_10487_gb300._abi import make_options
    from synth import workload
    build.build()
    wl = workload(WORKLOAD)
    geom = Geometry(wl.n, wl.m, wl.z1, wl.z2, tuple(wl.zy))
    om = [float(x) for x in wl.omegas]
    stream = torch.cuda.Stream()
    rc = Reconstructor(local, stream=stream)
    with torch.cuda.stream(stream):
        W64 = make_inputs(rc, wl, geom)
        W32 = W64.to(torch.complex64)
    torch.cuda.synchronize()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=rc.device)
    outs = {}
    graphs = {}
    cases = (("mixed", W32, torch.float32), ("fp64", W64, torch.float64))
    # the headline takes the rank-one closed form of the per-mode problem (solve_form 1,
    # exact for the Weyl kernel); the dense form (solve_form 0) is measured beside it
    forms = {"": HEAD_FORM, "_dense": 0}
    for prec, W, rdt in cases[::-1]:  # size the workspace (largest first) before any capture
        for tag, form in forms.items():
            xi = torch.empty((wl.m, wl.n, wl.n), dtype=rdt, device=rc.device)
            outs[prec + tag] = (xi, torch.empty_like(xi))
            with torch.cuda.stream(stream):
                rc.reconstruct(W, om, geom, DELTA, precision=prec, out=(xi, outs[prec + tag][1], None),
                               solve_form=form)
            torch.cuda.synchronize()
    for prec, W, rdt in cases:
        for tag, form in forms.items():
            xi, c = outs[prec + tag]
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                rc.reconstruct(W, om, geom, DELTA, precision=prec, out=(xi, c, None), solve_form=form)
            torch.cuda.synchronize()
            graphs[prec + tag] = g

    def timed(prec, K, Wm, clocks=None):
        g = graphs[prec]
        with torch.cuda.stream(stream):
            for _ in range(Wm):
                flush.zero_()
                g.replay()
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if clocks:
            clocks.start()
        with torch.cuda.stream(stream):
            for s, e in ev:
                flush.zero_()
                s.record(stream)
                g.replay()
                e.record(stream)
        torch.cuda.synchronize()
        if clocks:
            ck = clocks.stop()
        barrier(world)
        torch.cuda.synchronize()
        ms = sum(s.elapsed_time(e) for s, e in ev) / K
        return ms, (ck if clocks else None)

    clocks = Clocks(local)
    ms_mixed, ck = timed("mixed", args.steps, args.warmup, clocks)
    ms_fp64, _ = timed("fp64", args.steps, args.warmup)
    vox = wl.voxel_freqs
    value, ms_mixed = job_value(vox, ms_mixed, world)
    value_fp64, ms_fp64 = job_value(vox, ms_fp64, world)
    ms_dense = {p: max_over_ranks(timed(p + "_dense", args.steps, args.warmup)[0], world) for p in ("mixed", "fp64")}

    # per-kernel durations (CUDA events recorded by the library between its kernels)
    stage_ms = {}
    reps = {}
    for prec, W in (("mixed", W32), ("fp64", W64)):
        for tag, form in forms.items():
            xi, c = outs[prec + tag]
            acc = np.zeros(6)
            n = max(3, min(args.steps, 20))
            for _ in range(n):
                with torch.cuda.stream(stream):
                    flush.zero_()
                    rc.reconstruct(W, om, geom, DELTA, precision=prec, out=(xi, c, None), stage_timing=1,
                                   solve_form=form)
                rep = rc.report()
                acc += np.array([rep["ms_stage"][s] for s in STAGES])
            stage_ms[prec + tag] = dict(zip(STAGES, (acc / n).tolist()))
            reps[prec + tag] = rep

    # end to end through the C ABI with host buffers (copies inside the timed region)
    W_h = W32.cpu().pin_memory()
    # the step's result is xi; c (an optional output of the same call) stays on the device
    xi_h = torch.empty((wl.m, wl.n, wl.n), dtype=torch.float32).pin_memory()
    gstruct = geom.c_struct()

    e2e_opts = make_options(solve_form=HEAD_FORM)

    def e2e_once():
        fs_reconstruct_host(rc.ctx, gstruct, FS_MIXED, W_h.data_ptr(), om, DELTA, 1.0, e2e_opts, xi_h.data_ptr(),
                            None)

    for _ in range(args.warmup):
        flush.zero_()
        e2e_once()
    tot = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_once()
        tot += time.perf_counter() - t0
    e2e_ms = max_over_ranks(1e3 * tot / args.steps, world)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "128x128x64 X grid, 32 data planes, k0=8pi, 3 Gaussian inclusions, 1% noise",
                   "n": wl.n, "m": wl.m, "m1": wl.m1, "n_omega": len(om), "delta": DELTA,
                   "precision": "mixed (FP32 transforms and kernel factors, FP64 scalars, sums and eq. (9))",
                   "solve_form": "rank-one closed form of the per-mode Tikhonov problem (exact for the Weyl "
                                 "kernel; the dense form is reported under dense_form)",
                   "cuda_graph": True, "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": KERNELS_PER_STEP_MIXED * args.steps,
        "fp64_path": {"value": value_fp64, "ms_per_step": ms_fp64, "dtype": "f64",
                      "stage_ms": stage_ms["fp64"]},
        "dense_form": {p: {"value": world * wl.voxel_freqs / (ms_dense[p] * 1e-3), "ms_per_step": ms_dense[p],
                           "stage_ms": stage_ms[p + "_dense"],
                           "n_refine_iters": reps[p + "_dense"]["n_refine_iters"],
                           "n_fp64_fallback": reps[p + "_dense"]["n_fp64_fallback"]}
                       for p in ("mixed", "fp64")},
        "stage_ms": stage_ms["mixed"],
        "e2e": {"value": world * vox / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(W_h.numel() * 8), "d2h_bytes_per_step": int(xi_h.numel() * 4),
                "transfer": "page-locked host buffers read (W) and written (xi) by the kernels themselves "
                            "over the host link, inside the timed call; wall clock around fs_reconstruct_host"},
        "clocks": ck,
    }
    # per-stage rooflines, both precisions: algorithmic bytes against the measured copy
    # bandwidth and algorithmic flops against the measured FMA peak of the stage's
    # arithmetic (FP32 in the mixed path, FP64 in the plain one).  Stage times are the
    # library's event timers of an uncaptured run (launch gaps included)
    hbm, src = peaks()
    from paper_1911_10487_gb300._abi import fs_measure_alu_peaks
    alu = fs_measure_alu_peaks(local)
    stage_roof = {}
    for prec, sc, pk in (("mixed", 8, alu["fp32_tflops"]), ("fp64", 16, alu["fp64_tflops"])):
        stage_roof[prec] = {}
        for stg, ms in stage_ms[prec].items():
            if stg == "solve":
                continue  # a latency-bound chain per mode: no stream of bytes or flops to rate
            byt = algorithmic_bytes(stg, wl, reps[prec], sc, prec == "mixed")
            fl = stage_flops(stg, wl, reps[prec], prec == "mixed")
            gbs = byt / (ms * 1e-3) / 1e9
            tfl = fl / (ms * 1e-3) / 1e12
            stage_roof[prec][stg] = {"ms": ms, "bytes": byt, "gbs": gbs, "hbm_frac": gbs / hbm, "flops": fl,
                                     "tflops": tfl, "alu_frac": tfl / pk}
    result["stage_roofline"] = {"peaks": {"hbm_gbs": hbm, "hbm_source": src, "fp32_tflops": alu["fp32_tflops"],
                                          "fp64_tflops": alu["fp64_tflops"],
                                          "alu_source": "measured (fs_measure_alu_peaks)"},
                                "note": "stage times from the library's event timers, launch gaps included",
                                **stage_roof}
    # roofline of the dominant kernel of the headline (mixed) path: the transform pass
    # with the largest time, against the measured copy bandwidth (its algorithmic bytes:
    # what it must read and write once)
    sm = {k: v for k, v in stage_ms["mixed"].items() if k != "solve"}
    dom = max(sm, key=sm.get)
    byt = algorithmic_bytes(dom, wl, reps["mixed"], 8, True)
    ach = byt / (sm[dom] * 1e-3) / 1e9
    result["roofline"] = {"kernel": STAGE_KERNELS[dom], "stage": dom, "bound": "hbm", "achieved": ach, "peak": hbm,
                          "unit": "GB/s", "frac": ach / hbm, "traffic": STAGE_DRAM_BYTES.get(dom), "peak_source": src,
                          "algorithmic_bytes": byt,
                          "note": "the rank-one solve (" + f"{stage_ms['mixed']['solve'] * 1e3:.1f}" +
                                  " us) is a per-mode latency chain of O(M + M1) work"}
    # the dense per-mode solve: bound by the plain ALUs (the FP32 pipe in the mixed
    # path); peak = the library's own FP32 FMA microbenchmark on this GPU
    flops = solve_flops(wl, reps["mixed_dense"])
    t_solve = stage_ms["mixed_dense"]["solve"]
    ach = flops / (t_solve * 1e-3) / 1e12
    result["dense_form"]["mixed"]["roofline"] = {
        "kernel": "k_solve<float>", "bound": "alu", "achieved": ach, "peak": alu["fp32_tflops"], "unit": "TFLOP/s",
        "frac": ach / alu["fp32_tflops"], "traffic": SOLVE_DRAM_BYTES,
        "peak_source": "measured (fs_measure_alu_peaks, FP32 FMA)", "algorithmic_flops": flops,
        "fp64_peak_tflops": alu["fp64_tflops"]}
    result["counts"] = {k: v for k, v in reps["mixed"].items() if k != "ms_stage"}
    return result, rc, wl, geom, om, W64, outs


def run_forward(rc, wl, geom, om, reps=3):
    """Algorithm 1 (fs_forward) on the headline geometry and inclusions: the full-
    scattering data of the same xi, both precisions, and GMRES in FP64.  Each call synchronises once per
    iteration (the stopping test is on the host), so the time is host wall clock around
    whole calls; the FP64 and mixed data are compared with each other."""
    import torch
    xi64 = torch.from_numpy(np.ascontiguousarray(wl.xi)).to(rc.device)
    out = {"workload": "128x128x64 X grid, 32 data planes, k0=8pi, 3 Gaussian inclusions (the headline xi)",
           "stopping": "||U~_{n+1} - U~_n|| <= rtol ||U~0|| (rtol 1e-13 FP64, 1e-6 mixed)"}
    Ws = {}
    for prec, x in (("fp64", xi64), ("mixed", xi64.float())):
        from paper_1911_10487_gb300 import FlatLayerError
        try:
            rc.forward(x, om, geom, precision=prec)  # warm-up (workspace, twiddles)
        except FlatLayerError as e:
            out[prec] = {"not_converged": str(e)}
            continue
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            W, _, its = rc.forward(x, om, geom, precision=prec)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        ms = 1e3 * float(np.median(ts))
        it = int(sum(its))
        Ws[prec] = W
        out[prec] = {"ms": ms, "iterations": its, "ms_per_iteration": ms / max(it, 1),
                     "voxel_freq_iterations_per_s": wl.voxel_freqs * max(it, 1) / (ms * 1e-3)}
    if len(Ws) == 2:
        a, b = Ws["mixed"].to(torch.complex128), Ws["fp64"]
        out["mixed_vs_fp64_rel_l2"] = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    # the Krylov solver on the same problem (FP64, relative residual 1e-13)
    from paper_1911_10487_gb300 import FlatLayerError
    try:
        rc.forward(xi64, om, geom, method="gmres")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Wg, _, its = rc.forward(xi64, om, geom, method="gmres")
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0)
        out["gmres_fp64"] = {"ms": ms, "operator_applications": its}
        if "fp64" in Ws:
            out["gmres_vs_fixed_point_rel_l2"] = float(torch.linalg.vector_norm(Wg - Ws["fp64"]) /
                                                       torch.linalg.vector_norm(Ws["fp64"]))
    except FlatLayerError as e:
        out["gmres_fp64"] = {"not_converged": str(e)}
    return out


def run_batch(args, local, flush, world):
    """64 independent problems of uneven size (grids 64^2x16 .. 256^2x64, 1-8
    frequencies, 4-32 data planes, 1% noise) in one fs_reconstruct_batch call,
    launch configuration from the batch autotuner, replayed as one CUDA graph.
    Its own Reconstructor, so that growing the workspace cannot invalidate the
    single-problem graphs."""
    import torch
    from paper_1911_10487_gb300 import Geometry, Reconstructor
    from paper_1911_10487_gb300.tuner import BatchTuner
    from synth.workloads import batch_c4
    stream = torch.cuda.Stream()
    rc = Reconstructor(local, stream=stream)
    wls = batch_c4()
    items = {"fp64": [], "mixed": []}
    outs = {"fp64": [], "mixed": []}
    with torch.cuda.stream(stream):
        for wl in wls:
            geom = Geometry(wl.n, wl.m, wl.z1, wl.z2, tuple(wl.zy))
            om = [float(x) for x in wl.omegas]
            W = make_inputs(rc, wl, geom)
            items["fp64"].append((W, om, geom, DELTA))
            items["mixed"].append((W.to(torch.complex64), om, geom, DELTA))
            for prec, rdt in (("fp64", torch.float64), ("mixed", torch.float32)):
                xi = torch.empty((wl.m, wl.n, wl.n), dtype=rdt, device=rc.device)
                outs[prec].append((xi, torch.empty_like(xi)))
    torch.cuda.synchronize()
    tuner = BatchTuner()
    res = {}
    cfgs = {}
    for prec in ("fp64", "mixed"):  # FP64 first: it sizes the workspace for both
        if args.batch_config:  # a fixed launch configuration (profiling runs): no tuning
            cfgs[prec] = tuple(int(x) for x in args.batch_config.split(","))
        else:
            cfgs[prec] = tuner.best(rc, items[prec], prec, repeats=2, outs=outs[prec],
                                    options={"solve_form": HEAD_FORM})
    graphs = {}
    for prec in ("fp64", "mixed"):
        s_, b_, t_, c_ = cfgs[prec]
        kw = dict(n_streams=s_, outs=outs[prec], solve_blocks_per_sm=b_, fft_tile=t_, classify_single_pass=c_,
                  solve_form=HEAD_FORM)
        with torch.cuda.stream(stream):
            rc.reconstruct_batch(items[prec], prec, **kw)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            rc.reconstruct_batch(items[prec], prec, **kw)
        torch.cuda.synchronize()
        graphs[prec] = g
    vox = sum(wl.voxel_freqs for wl in wls)
    K = max(3, min(args.steps, 10))
    for prec in ("mixed", "fp64"):
        g = graphs[prec]
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                flush.zero_()
                g.replay()
        torch.cuda.synchronize()
        barrier(world)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        with torch.cuda.stream(stream):
            for s, e in ev:
                flush.zero_()
                s.record(stream)
                g.replay()
                e.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in ev) / K, world)
        # the batch's compulsory HBM traffic: every problem's data W read once and xi, c
        # written once (a lower bound of the algorithmic bytes: the intermediates of
        # this workload's 4-16 MB problems stay in the 129 MB L2 between kernels)
        sc = 16 if prec == "fp64" else 8
        byt = sum(len(wl.omegas) * wl.m1 * wl.n * wl.n * sc + 2 * wl.m * wl.n * wl.n * (sc // 2) for wl in wls)
        hbm, src = peaks()
        gbs = byt / (ms * 1e-3) / 1e9
        res[prec] = {"value": world * vox / (ms * 1e-3), "ms_per_step": ms,
                     "tuned": {"n_streams": cfgs[prec][0], "solve_blocks_per_sm": cfgs[prec][1],
                               "fft_tile": cfgs[prec][2], "classify_single_pass": cfgs[prec][3],
                               "solve_form": HEAD_FORM},
                     "roofline": {"bound": "hbm", "compulsory_bytes": byt, "achieved": gbs, "peak": hbm,
                                  "unit": "GB/s", "frac": gbs / hbm, "peak_source": src,
                                  "note": "W read once, xi and c written once per problem"}}
    grids = {}
    for wl in wls:
        k = f"{wl.n}^2x{wl.m}"
        grids[k] = grids.get(k, 0) + 1
    out = {"workload": "64 independent problems, grids " + ", ".join(f"{k}: {v}" for k, v in sorted(grids.items()))
                       + ", 1-8 frequencies in [2pi,12pi], 4-32 data planes, 1% noise",
           "voxel_freqs": vox, "steps": K, "cuda_graph": True, "unit": UNIT,
           "l2": "flushed (256 MiB write) before every timed step",
           "mixed": res["mixed"], "fp64": res["fp64"],
           "gpu_launches_per_step": sum(mixed_kernels(wl.n) for wl in wls)}
    # smallest problem of the batch against the oracle (a parity spot check at full batch)
    j = min(range(len(wls)), key=lambda i: wls[i].voxel_freqs * wls[i].m1)
    out["spot_problem"] = wls[j].name
    out["_spot"] = (wls[j], items["fp64"][j][0].cpu().numpy(), items["fp64"][j][1],
                    outs["mixed"][j][0].double().cpu().numpy(), outs["fp64"][j][0].cpu().numpy())
    rc.close()
    return out


def run_diff(args, local, flush, world):
    """Derivatives at fixed alpha per frequency on 128x128x64, 4 frequencies
    (4pi..10pi), 32 data planes, 3 Gaussians, 1% noise: alpha tuned by 50
    Gauss-Newton-scaled gradient steps on sum (Phi/target - 1)^2, 16 seeded data
    perturbations of 1% pushed through as JVPs, one full VJP; full-size checks by
    the dot-product test and a central difference (h = 1e-6, FP64)."""
    import torch
    from paper_1911_10487_gb300 import Geometry, Reconstructor
    from paper_1911_10487_gb300.diff import DiffPlan, jvp_study, tune_log_alpha
    from synth import noise_direction, workload
    wl = workload("c5")
    stream = torch.cuda.Stream()
    rc = Reconstructor(local, stream=stream)
    geom = Geometry(wl.n, wl.m, wl.z1, wl.z2, tuple(wl.zy))
    om = [float(x) for x in wl.omegas]
    F, N2 = len(om), wl.n * wl.n
    rng = np.random.default_rng(44)
    nd = 16
    dirs = noise_direction(rng, (nd, F, wl.m1, wl.n, wl.n))
    out = {"workload": "128x128x64 X grid, 32 data planes, 4 frequencies 4pi..10pi, 3 Gaussians, 1% noise",
           "voxel_freqs": wl.voxel_freqs}

    def ev():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    with torch.cuda.stream(stream):
        W64 = make_inputs(rc, wl, geom)
        tgt = torch.stack([N2 * (2.0 * DELTA * torch.linalg.vector_norm(W64[j])) ** 2 for j in range(F)]).double()
        la0 = torch.zeros(F, dtype=torch.float64, device=rc.device)
        dW_all = torch.from_numpy(dirs).to(rc.device)
        for j in range(F):  # each direction scaled to 1% of ||W_omega|| per frequency
            nrm = torch.linalg.vector_norm(dW_all[:, j].reshape(nd, -1), dim=1).reshape(nd, 1, 1, 1)
            dW_all[:, j] *= DELTA * torch.linalg.vector_norm(W64[j]) / nrm
        for prec in ("mixed", "fp64"):
            W = W64 if prec == "fp64" else W64.to(torch.complex64)
            dW = dW_all if prec == "fp64" else dW_all.to(torch.complex64)
            t0, t1 = ev()
            t0.record(stream)
            plan = DiffPlan(rc, geom, om, prec)
            t1.record(stream)
            tune_log_alpha(plan, W, la0, tgt, steps=3)  # warm-up
            a0, a1 = ev()
            a0.record(stream)
            la, hist = tune_log_alpha(plan, W, la0, tgt, steps=50)
            a1.record(stream)
            plan.jvp(plan.forward(W, la)[3], dW)  # warm-up of the JVP scratch
            reps = max(3, min(args.steps, 10))
            f0, f1 = ev()
            f0.record(stream)
            for _ in range(reps):
                flush.zero_()
                xi, _, phi, tape = plan.forward(W, la)
            f1.record(stream)
            gxi = torch.ones_like(xi)
            b0, b1 = ev()
            b0.record(stream)
            for _ in range(reps):
                flush.zero_()
                gW, gla = plan.vjp(tape, gxi, None)
            b1.record(stream)
            j0, j1 = ev()
            j0.record(stream)
            dxi, amp = jvp_study(plan, tape, W, dW, xi)
            j1.record(stream)
            torch.cuda.synchronize()
            # full-size checks: dot-product test on direction 0; FP64 central difference
            lhs = float((dxi[0].double() * gxi.double()).sum())
            rhs = float((torch.conj(gW[0:F]).to(torch.complex128) * dW[0].to(torch.complex128)).real.sum())
            res = {"ms_plan_normal_matrices": t0.elapsed_time(t1),
                   "ms_tune_alpha_50_steps": a0.elapsed_time(a1),
                   "ms_forward": f0.elapsed_time(f1) / reps, "ms_vjp": b0.elapsed_time(b1) / reps,
                   "ms_jvp_16_directions": j0.elapsed_time(j1),
                   "forward_voxel_freqs_per_s": wl.voxel_freqs / (f0.elapsed_time(f1) / reps * 1e-3),
                   "tuned_log_alpha": la.cpu().tolist(), "misfit_first_last": [float(hist[0]), float(hist[-1])],
                   "jvp_amplification_mean_max": [float(amp.mean()), float(amp.max())],
                   "dot_product_rel_err": abs(lhs - rhs) / abs(lhs)}
            if prec == "fp64":
                h = 1e-6
                xp = plan.forward(W + h * dW[0], la)[0]
                xm = plan.forward(W - h * dW[0], la)[0]
                fd = (xp - xm) / (2 * h)
                res["central_difference_rel_err"] = float(torch.linalg.vector_norm(fd - dxi[0]) /
                                                          torch.linalg.vector_norm(fd))
            out[prec] = res
            plan.close()
    torch.cuda.synchronize()
    rc.close()
    return out


def graph_time(stream, flush, fn, steps, warmup, world):
    """Capture fn() as a CUDA graph on `stream` and time `steps` replays (L2 flushed
    before each) with CUDA events; returns ms per replay, max over ranks."""
    import torch
    with torch.cuda.stream(stream):
        fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.zero_()
            g.replay()
    torch.cuda.synchronize()
    barrier(world)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            g.replay()
            b.record(stream)
    torch.cuda.synchronize()
    return max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / steps, world)


def run_sampled(args, local, flush, world):
    """The sampled-G kernel (Sec. 5: G~ from the FFT of sampled G) on the headline
    workload: kernel plan build once per precision, then the reconstruction with the
    dense per-mode solve on the tabulated A_nu (numerically full rank) and the Toeplitz
    eq. (9), replayed as a CUDA graph.  Same data as the headline (the library's
    single-scattering kernel plus seeded noise)."""
    import torch
    from paper_1911_10487_gb300 import Geometry, KernelPlan, Reconstructor
    from synth import workload
    wl = workload(WORKLOAD)
    geom = Geometry(wl.n, wl.m, wl.z1, wl.z2, tuple(wl.zy))
    om = [float(x) for x in wl.omegas]
    stream = torch.cuda.Stream()
    rc = Reconstructor(local, stream=stream)
    with torch.cuda.stream(stream):
        W64 = make_inputs(rc, wl, geom)
    torch.cuda.synchronize()
    out = {"workload": "128x128x64 X grid, 32 data planes, k0=8pi, 1% noise; sampled-G kernel, dense form",
           "voxel_freqs": wl.voxel_freqs, "steps": args.steps}
    xis = {}
    for prec, W, rdt in (("fp64", W64, torch.float64), ("mixed", W64.to(torch.complex64), torch.float32)):
        t0 = time.perf_counter()
        plan = KernelPlan(rc, geom, om, prec)
        torch.cuda.synchronize()
        plan_ms = 1e3 * (time.perf_counter() - t0)
        xi = torch.empty((wl.m, wl.n, wl.n), dtype=rdt, device=rc.device)
        c = torch.empty_like(xi)
        torch.cuda.synchronize()  # inputs made on the default stream

        def step():
            rc.reconstruct(W, om, geom, DELTA, precision=prec, out=(xi, c, None), kernel_plan=plan)

        ms = graph_time(stream, flush, step, args.steps, args.warmup, world)
        with torch.cuda.stream(stream):
            step()
        rep = rc.report()
        out[prec] = {"value": world * wl.voxel_freqs / (ms * 1e-3), "ms_per_step": ms, "plan_ms": plan_ms,
                     "plan_bytes": plan.nbytes, "n_active": rep["n_active"],
                     "n_fp64_fallback": rep["n_fp64_fallback"], "n_refine_iters": rep["n_refine_iters"]}
        xis[prec] = xi.double().cpu().numpy()
        plan.close()
    out["_check"] = (wl, W64.cpu().numpy(), om, xis)
    rc.close()
    return out


def delta_l2_planes(xi, xi_true):
    """Delta_L2(z) of Sec. 5.3 per X plane (NaN where xi_true vanishes on the plane)."""
    m = xi_true.shape[0]
    d = np.linalg.norm((xi - xi_true).reshape(m, -1), axis=1)
    n = np.linalg.norm(xi_true.reshape(m, -1), axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(n > 0, d / n, np.nan)


def run_paper(args, local, flush, world):
    """The paper's own experiment (Sec. 5, 5.3, 5.4) at full size: X = [-10,10]^2 x
    [-0.5,1.5] on 128 x 128 x 71, data on 71 planes of [6.01, 6.5] (thick) or 2 of
    [6.01, 6.02] (thin), 11 point sources (0, y, 6), the three-bump xi (A0 = 0.3),
    omega = 1, 2, 3 solved together (least squares over omega), noise 0, 1e-7, 1e-5
    (delta_floor 1e-10).  Data: the library's point-source incident field and its
    single-scattering kernel.  M1 = 71 is solved in the rank-one form.  Reports the
    time of one reconstruction (CUDA graph) and Delta_L2(z) against the true xi."""
    import torch
    from paper_1911_10487_gb300 import Geometry, Reconstructor
    from paper_1911_10487_gb300._abi import FS_MIXED_MIN_NOISE
    from synth import paper_workload
    stream = torch.cuda.Stream()
    rc = Reconstructor(local, stream=stream)
    res = {"workload": "paper geometry (Sec. 5): 128^2 x 71 X grid, 11 point sources, three bumps A0=0.3, "
                       "omega 1,2,3; thick layer 71 planes, thin layer 2 planes; rank-one form; delta_floor 1e-10"}
    for layer in ("thick", "thin"):
        pw = paper_workload(layer)
        geom = Geometry(pw.n, pw.m, pw.z1, pw.z2, tuple(pw.zy), pw.period)
        om = [float(x) for x in pw.omegas]
        with torch.cuda.stream(stream):
            u0 = rc.incident_point_sources(pw.sources, om, geom, precision="fp64")
            xi_t = torch.from_numpy(np.ascontiguousarray(pw.xi)).to(rc.device)
            W0 = rc.forward_born(xi_t, om, geom, precision="fp64", incident=u0)
            nz = torch.from_numpy(pw.noise()).to(rc.device)
        torch.cuda.synchronize()
        lr = {"voxel_freqs": pw.voxel_freqs, "m1": pw.m1}
        for delta in (pw.deltas if layer == "thick" else (0.0, 1e-7)):
            W = W0.clone()
            if delta > 0:
                for j in range(W.shape[0]):
                    W[j] += delta * torch.linalg.vector_norm(W0[j]) * nz[j] / torch.linalg.vector_norm(nz[j])
            entry = {}
            for prec in ("fp64", "mixed"):
                if prec == "mixed" and max(delta, 1e-10) < FS_MIXED_MIN_NOISE:
                    entry[prec] = {"unsupported": f"noise level below the mixed path's FP32 data resolution "
                                                  f"(FS_MIXED_MIN_NOISE = {FS_MIXED_MIN_NOISE:g}): FS_FP64 only"}
                    continue
                cdt = torch.complex128 if prec == "fp64" else torch.complex64
                rdt = torch.float64 if prec == "fp64" else torch.float32
                Wp, up = W.to(cdt), u0.to(cdt)
                xi = torch.empty((pw.m, pw.n, pw.n), dtype=rdt, device=rc.device)
                c = torch.empty_like(xi)
                torch.cuda.synchronize()  # inputs made on the default stream

                def step():
                    rc.reconstruct(Wp, om, geom, delta, precision=prec, out=(xi, c, None), solve_form=1,
                                   incident=up, delta_floor=1e-10)

                ms = graph_time(stream, flush, step, max(3, min(args.steps, 10)), args.warmup, world)
                dz = delta_l2_planes(xi.double().cpu().numpy(), pw.xi)
                rep = rc.report()
                entry[prec] = {"value": world * pw.voxel_freqs / (ms * 1e-3), "ms_per_step": ms,
                               "n_active": rep["n_active"], "n_nonfinite": rep["n_nonfinite"],
                               "delta_l2_z": {"min": float(np.nanmin(dz)), "median": float(np.nanmedian(dz)),
                                              "max": float(np.nanmax(dz)),
                                              "per_plane": [round(float(x), 5) for x in dz]}}
            lr[f"delta={delta:g}"] = entry
        res[layer] = lr
    rc.close()
    return res


def cpu_baseline(wl, W_np, om, rows=None):
    from oracle import inverse
    from oracle.grid import Geometry as OG
    g = OG(wl.n, wl.m, wl.z1, wl.z2, tuple(wl.zy))
    opts = inverse.Options(mode_rows=rows)
    t0 = time.perf_counter()
    res = inverse.reconstruct(W_np, om, g, DELTA, opts=opts)
    return time.perf_counter() - t0, res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-problem batch measurement")
    ap.add_argument("--no-diff", action="store_true", help="skip the derivative measurement")
    ap.add_argument("--no-forward", action="store_true", help="skip the full-scattering forward measurement")
    ap.add_argument("--no-sampled", action="store_true", help="skip the sampled-G kernel measurement")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper-geometry workload")
    ap.add_argument("--batch-config", default="",
                    help="n_streams,solve_blocks_per_sm,fft_tile,classify_single_pass for both batch precisions "
                         "instead of the autotuner's choice (for profiling runs)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":  # host cores only: no device is touched
        return run_reference(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
    rank, world, local = dist_setup(args.gpus)
    result, rc, wl, geom, om, W64, outs = run_ours(args, rank, world, local)
    batch = None
    if not args.no_batch:
        import torch
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=rc.device)
        batch = run_batch(args, local, flush, world)
        spot = batch.pop("_spot")
        result["batch"] = batch
    if not args.no_diff:
        import torch
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=rc.device)
        result["differentiation"] = run_diff(args, local, flush, world)
    if not args.no_forward:
        result["forward_fixed_point"] = run_forward(rc, wl, geom, om)
    sampled_check = None
    if not args.no_sampled:
        import torch
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=rc.device)
        sp = run_sampled(args, local, flush, world)
        sampled_check = sp.pop("_check")
        result["sampled_kernel"] = sp
    if not args.no_paper:
        import torch
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=rc.device)
        result["paper_geometry"] = run_paper(args, local, flush, world)
    if rank == 0:
        import torch
        W_np = W64.cpu().numpy()
        if not args.no_cpu_baseline:
            t, ref = cpu_baseline(wl, W_np, om)
            from oracle.metrics import rel_l2
            result["cpu_baseline"] = {"value": wl.voxel_freqs / t, "unit": UNIT, "cores": os.cpu_count(),
                                      "kind": "oracle",
                                      "sample": "one full reconstruction of the workload (NumPy/SciPy FP64)"}
            result["rel_err_vs_oracle"] = {
                "mixed": rel_l2(outs["mixed"][0].double().cpu().numpy(), ref.xi),
                "fp64": rel_l2(outs["fp64"][0].cpu().numpy(), ref.xi)}
            # Delta_L2(z) of Sec. 5.3: per X plane, the reconstruction against the true xi
            # (a property of the method and the data, not of the implementation: the
            # oracle's own value is given beside the GPU's)
            from oracle.metrics import delta_l2_z
            dz = {"oracle": delta_l2_z(ref.xi, wl.xi),
                  "mixed": delta_l2_z(outs["mixed"][0].double().cpu().numpy(), wl.xi),
                  "fp64": delta_l2_z(outs["fp64"][0].cpu().numpy(), wl.xi)}
            result["delta_l2_z_vs_true_xi"] = {
                "note": "per X plane z'_l, ||xi_rec - xi_true||_L2(xy) / ||xi_true||_L2(xy) (Sec. 5.3)",
                **{k: {"min": float(np.nanmin(v)), "median": float(np.nanmedian(v)), "max": float(np.nanmax(v)),
                       "per_plane": [round(float(x), 6) for x in v]} for k, v in dz.items()}}
            for p in ("mixed", "fp64"):
                result["dense_form"][p]["rel_err_vs_oracle"] = rel_l2(
                    outs[p + "_dense"][0].double().cpu().numpy(), ref.xi)
            if sampled_check is not None:
                from oracle import inverse
                from oracle.grid import Geometry as OG
                swl, sW, som, sxis = sampled_check
                sg = OG(swl.n, swl.m, swl.z1, swl.z2, tuple(swl.zy), kernel="sampled")
                t0 = time.perf_counter()
                sref = inverse.reconstruct(sW, som, sg, DELTA)
                result["sampled_kernel"]["oracle_s"] = time.perf_counter() - t0
                result["sampled_kernel"]["rel_err_vs_oracle"] = {p: rel_l2(x, sref.xi) for p, x in sxis.items()}
            if batch is not None:
                swl, sW, som, sxm, sx64 = spot
                _, sref = cpu_baseline(swl, sW, som)
                batch["spot_rel_err_vs_oracle"] = {"mixed": rel_l2(sxm, sref.xi), "fp64": rel_l2(sx64, sref.xi)}
        print(json.dumps(result))
    rc.close()


def run_reference(args, rank, world):
    """The oracle as the reference arm: rank 0 only, on host cores.  It builds the
    data itself (the oracle's own single-scattering operator plus the workload's
    seeded noise) and times one full reconstruction of the workload per step: no
    part of the library is loaded.  A step takes seconds, so at most 3 timed steps
    after one warm-up are run whatever --steps and --warmup ask."""
    if rank != 0:
        return
    from oracle import forward
    from oracle.grid import Geometry as OG
    from synth import workload
    wl = workload(WORKLOAD)
    g = OG(wl.n, wl.m, wl.z1, wl.z2, tuple(wl.zy))
    om = [float(x) for x in wl.omegas]
    W, _ = forward.make_data(wl.xi, om, g, method="born")
    W_np = forward.add_noise(W, DELTA, wl.noise())
    steps, warm = min(args.steps, 3), min(args.warmup, 1)
    for _ in range(warm):
        cpu_baseline(wl, W_np, om)
    tot = 0.0
    for _ in range(steps):
        t, _ = cpu_baseline(wl, W_np, om)
        tot += t
    ms = 1e3 * tot / steps
    value = wl.voxel_freqs / (ms * 1e-3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps,
           "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": "128x128x64 X grid, 32 data planes, k0=8pi, 3 Gaussian inclusions, 1% noise",
                      "n": wl.n, "m": wl.m, "m1": wl.m1, "n_omega": len(om), "delta": DELTA},
           "same_config": True,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"one full reconstruction of the workload per step (NumPy/SciPy FP64), "
                                      f"{steps} timed steps after {warm} warm-up (requested {args.steps}/"
                                      f"{args.warmup}: a step takes seconds); data from the oracle's own "
                                      f"single-scattering operator plus the seeded noise"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
