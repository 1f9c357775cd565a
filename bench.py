"""Benchmark: Y_lm evaluations per second on the 192^3 real-space DFT grid.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl shm|reference]
                    [--extras | --no-extras]

One step = one pass of the evaluator over the whole workload: all R_l^m,
l <= 9, at the 7,077,888 points of a 192^3 grid (spacing 0.3 bohr, centred on
a seeded off-grid atom), FP64 in and out (5.66 GB of output per step), every
value computed in binary64 arithmetic (SHM_STRICT_FP64: the paper's precision;
the float-float hybrid rows are reported beside it as an extra, labelled).
Inputs are resident in HBM when the timed region starts; input (170 MB) and
output (5.66 GB) both exceed the 126 MB L2, so no L2 flush is needed between
steps.

Prints one JSON line (rank 0).  N > 1 runs one process per GPU (torchrun);
each rank evaluates its own copy of the grid (weak scaling, no collective on
the data path; a barrier and a max-reduction of the elapsed time only).

--impl reference times the CPU FP64 oracle (test infrastructure, the paper
defines the reference values; there is no reference GPU code) on a bounded
sample of the same workload, on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Y_lm evals/s at lmax=9"
UNIT = "Y_lm/s"
WORKLOAD = "dft_grid_192cubed_fp64_lmax9"
LMAX = 9
N_SIDE = 192

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 pipe peak: measured in every run by shm_probe_fp64_rate (independent
# DFMA chains on every SM, CUDA events); the nominal 1.25 TFLOP/s dense FP64
# of a B300 (0.625e12 FP64 pipe instructions per second) only if that fails.
FP64_NOMINAL_TFLOPS = 1.25
HBM_FALLBACK_GBS = 6400.0
# FP64 pipe instructions per point of the all-binary64 rows at lmax 9
# (sh_row: DMUL + DFMA, counted by ncu sass__inst_executed_per_opcode).
STRICT_DP_PER_POINT_L9 = 242
# All-binary64 projectors on the 512-atom problem (lmax 2-4, 13,163,477
# points), FP64-pipe instructions per point counted by ncu
# (smsp__inst_executed_pipe_fp64.sum x 32 / points): 107.1 with every product
# on the FP64 pipe (strict form 1), 68.8 with the row products on the integer
# pipes (form 3, the default; the same bits).
STRICT_PROJ_DP_PER_POINT = {1: 107.1, 3: 68.8}
# FP64-pipe instructions per point of the all-binary64 complex, angle-input
# and spinor kernels at lmax 9 (ncu smsp__inst_executed_pipe_fp64.sum x 32 /
# points on the 96^3 grid; the output products of the complex and angle rows
# on the integer pipes).
STRICT_X_DP_PER_POINT = {"complex": 153.0, "angular": 192.0, "spinor": 960.5}
# binary64 products per point that the rows-tma-emu variants compute on the
# integer pipes instead (dmul_int, bitwise the DMUL results): the 90 output
# products s A, s B at lmax 9, and with the scales s = S q another 36.
EMU_PRODUCTS_L9 = {"rows-tma-emu-o-32": 90, "rows-tma-emu-os-32": 126}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- reference arm

def oracle_timing(points: np.ndarray, lmax: int, step_s: float, steps: int, warmup: int, nthreads: int = 0):
    """The one protocol by which this file times the oracle (the GPU line's
    cpu_baseline and the reference arm alike): size a prefix of `points` so
    that one call takes about step_s (a probe call on up to 20,000 points),
    make `warmup` untimed calls on it, then `steps` timed calls.  Returns the
    median Y/s over the timed calls, the prefix size and the thread count."""
    import oracle
    oracle.build()
    probe = min(points.shape[0], 20000)
    t0 = time.perf_counter()
    oracle.real_sh(points[:probe], lmax, nthreads=nthreads)
    dt = max(time.perf_counter() - t0, 1e-6)
    m = int(min(points.shape[0], max(probe, probe * step_s / dt)))
    nh = (lmax + 1) ** 2
    rates = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        oracle.real_sh(points[:m], lmax, nthreads=nthreads)
        if i >= warmup:
            rates.append(m * nh / (time.perf_counter() - t0))
    return statistics.median(rates), m, oracle.max_threads(nthreads)


def cpu_oracle_rate(points: np.ndarray, lmax: int, budget_s: float, nthreads: int = 0):
    """Y/s of the oracle on a bounded prefix of `points`: oracle_timing with
    one warm-up and three timed calls of about budget_s / 4 each."""
    return oracle_timing(points, lmax, budget_s / 4, 3, 1, nthreads)


def reference_step_budget(args) -> float:
    """Seconds of oracle work per step of the reference arm for this
    invocation's --steps / --warmup / --cpu-seconds: about two minutes for the
    whole run, at most --cpu-seconds (and 20 s) per step."""
    return min(args.cpu_seconds, 20.0, max(0.05, 120.0 / max(1, args.steps + args.warmup)))


def reference_arm_baseline(args):
    """The GPU line's cpu_baseline: the reference arm of this file (the oracle
    on the host cores) run as a fresh process with the per-step budget the
    reference arm gets for the same --steps / --warmup, so that both lines
    time the same prefix of the grid with the same program in the same kind
    of process (the oracle's rate depends on the prefix size: its threads'
    start-up is a larger share of a short call); three timed steps after
    three warm-up steps."""
    step_s = reference_step_budget(args)
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", "3", "--warmup", "3",
           "--step-budget", str(step_s)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=dict(os.environ, WORLD_SIZE="1",
                                                                                      RANK="0"))
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        ref = json.loads(lines[-1])
        cb = dict(ref["cpu_baseline"])
        cb["protocol"] = (cb.get("protocol", "") + "; measured by `bench.py --impl reference --steps 3 --warmup 3 "
                          f"--step-budget {step_s:.3g}` as a separate process (the reference arm's per-step budget "
                          "for this invocation's --steps / --warmup)")
        return cb
    except Exception as e:  # reported, never silently dropped
        return {"value": None, "unit": UNIT, "kind": "oracle", "error": repr(e)}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2510_05282_b300 import inputs
    pts = inputs.dft_grid_points(N_SIDE)
    nh = (LMAX + 1) ** 2
    # about two minutes for the whole run whatever --steps and --warmup are,
    # and at most --cpu-seconds per step; the same protocol as the GPU arm's
    # cpu_baseline (oracle_timing), with one call per step
    budget = args.step_budget if args.step_budget is not None else reference_step_budget(args)
    value, sample_pts, cores = oracle_timing(pts, LMAX, budget, args.steps, args.warmup)
    ms = pts.shape[0] * nh / value * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points": int(pts.shape[0]), "lmax": LMAX,
                   "note": "each step times the oracle on a prefix of the grid; ms_per_step is "
                           "extrapolated to the full grid"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {sample_pts} of {pts.shape[0]} grid points per step",
                         "protocol": "oracle_timing: median of the timed calls after warm-up calls"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm

def timed_launches(fn, steps, stream):
    """Per-launch CUDA-event durations (ms) on `stream` and the region length."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    region = starts[0].elapsed_time(ends[-1])
    return per, region


def graph_replay_timing(torch, fn, launches=20, replays=5, stream=None):
    """fn (one launch on `stream`) captured `launches` times into one CUDA
    graph and replayed: median ms per launch over the replays (outside the
    timed region; the launch overhead it removes is negligible next to a
    ms-scale kernel)."""
    try:
        gs = stream if stream is not None else torch.cuda.Stream()
        gs.wait_stream(torch.cuda.current_stream())
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=gs):
            for _ in range(launches):
                fn(gs)
        cur = torch.cuda.current_stream()
        g.replay()
        torch.cuda.synchronize()
        reps = []
        for _ in range(replays):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            g.replay()
            e1.record(cur)
            torch.cuda.synchronize()
            reps.append(e0.elapsed_time(e1) / launches)
        del g
        return {"launches_per_graph": launches, "replays": replays,
                "median_ms_per_launch": statistics.median(reps)}
    except Exception as e:  # reported, never silently dropped
        return {"error": repr(e)}


def gpu_id_for_smi(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def measure_eval(shm, torch, pts_np, dtype, lmax, steps, warmup, stream, strict=False):
    p = torch.from_numpy(pts_np).to(device="cuda", dtype=dtype)
    out = torch.empty((p.shape[0], (lmax + 1) ** 2), dtype=dtype, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            shm.eval_sh(p, lmax, out=out, stream=stream, strict=strict)
    torch.cuda.synchronize()
    per, region = timed_launches(lambda: shm.eval_sh(p, lmax, out=out, stream=stream, strict=strict), steps, stream)
    del out, p
    return per, region


def measure_fp64_peak(shm, reps=2):
    """The FP64 pipe rate of this GPU (shm_probe_fp64_rate: DFMA chains on
    every SM, six launch shapes, the fastest), best of `reps` probes, as
    TFLOP/s (2 flops per DFMA).  About 0.2 s per probe."""
    try:
        rates = [shm.probe_fp64_rate(1 << 12)[0] for _ in range(reps)]
        return {"tflops": 2.0 * max(rates) / 1e12, "dfma_per_s": max(rates), "runs": rates,
                "source": "measured: shm_probe_fp64_rate (independent DFMA chains, 4-16 per thread, 2-8 CTAs of "
                          "256 threads per SM, CUDA events; the fastest shape), best of 2"}
    except Exception as e:  # the nominal figure, said so
        return {"tflops": FP64_NOMINAL_TFLOPS, "dfma_per_s": FP64_NOMINAL_TFLOPS * 0.5e12,
                "source": f"nominal 1.25 TFLOP/s (probe failed: {e!r})"}


def run_gpu(args, rank, world):
    import torch

    import paper_2510_05282_b300 as shm
    from paper_2510_05282_b300 import build, inputs

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    shm.lib()
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    peaks, peaks_src = load_peaks()
    fp64 = measure_fp64_peak(shm)
    nh = (LMAX + 1) ** 2

    tdt = torch.float64 if args.dtype == "f64" else torch.float32
    es = 8 if args.dtype == "f64" else 4
    strict = args.dtype == "f64" and args.arith == "strict"
    tuned_ms = None
    if args.variant:
        for v in range(shm.eval_variant_count()):
            try:
                shm.set_eval_variant(LMAX, tdt, v, strict=strict)
            except shm.ShmError:
                continue
            if shm.eval_variant(LMAX, tdt, strict=strict) == args.variant:
                break
        else:
            raise SystemExit(f"unknown launch variant {args.variant}")
    pts = inputs.dft_grid_points(args.grid)
    n_total = pts.shape[0]
    shard = args.shard and world > 1
    if shard:  # strong scaling: this rank's contiguous part of the one grid
        from paper_2510_05282_b300.parallel import shard_range
        a, b = shard_range(n_total, rank, world)
        pts = np.ascontiguousarray(pts[a:b])
    if not args.variant and args.tune:  # tune on the workload's own size
        tuned_ms = shm.autotune(LMAX, tdt, min(pts.shape[0], 1 << 23), strict=strict)
    if args.dtype == "f32":
        pts = pts.astype(np.float32)
    n = pts.shape[0]
    p = torch.from_numpy(pts).cuda()
    out = torch.empty((n, nh), dtype=tdt, device="cuda")
    launch = lambda st: shm.eval_sh(p, LMAX, out=out, stream=st, strict=strict)  # noqa: E731
    for _ in range(args.warmup):
        launch(stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(gpu_id_for_smi(dev)) if rank == 0 else None
    if clocks:
        clocks.start()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    per, region = timed_launches(lambda: launch(stream), args.steps, stream)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist

        from paper_2510_05282_b300.parallel import max_over_ranks
        region = max_over_ranks(region, device="cuda")
        dist.barrier()
    clk = clocks.stop() if clocks else None
    graph = graph_replay_timing(torch, launch, stream=stream) if rank == 0 else None

    ms_per_step = region / args.steps
    value = (n_total if shard else world * n) * nh / (ms_per_step * 1e-3)
    launch_ms = statistics.mean(per)

    # roofline of the (single) kernel
    variant = shm.eval_variant(LMAX, tdt, strict=strict)
    hybrid = args.dtype == "f64" and "hybrid" in variant
    emu = EMU_PRODUCTS_L9.get(variant, 0)
    dp_pp = HYBRID_DP_PER_POINT_L9 if hybrid else STRICT_DP_PER_POINT_L9 - emu
    achieved_tflops = 2.0 * dp_pp * n / (launch_ms * 1e-3) / 1e12
    bytes_per_launch = n * (3 + nh) * es
    achieved_gbs = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    tpp = TRAFFIC_PER_POINT.get((args.dtype, variant))
    traffic = tpp * n if tpp else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": (WORKLOAD if args.grid == N_SIDE else f"dft_grid_{args.grid}cubed_fp64_lmax9")
                   .replace("fp64", "fp32" if args.dtype == "f32" else "fp64"),
                   "points": n_total, "points_per_rank": n, "lmax": LMAX, "grid": f"{args.grid}^3, h=0.3 bohr",
                   "out_bytes_per_step": n * nh * es,
                   "parallelism": (f"shard{world}" if shard else f"replicas{world}") if world > 1 else "single",
                   "l2": "no flush: 170 MB input and 5.66 GB output per step exceed the 126 MB L2",
                   "launch_variant": variant, "arithmetic": ARITHMETIC[(args.dtype, hybrid)],
                   "autotune_probe_ms": tuned_ms,
                   "timing": {"mean_ms_per_launch": launch_ms, "median_ms_per_launch": statistics.median(per),
                              "cuda_graph_replay": graph}},
        "roofline": roofline_object(args.dtype, hybrid, dp_pp, achieved_tflops, achieved_gbs, hbm_peak, peaks_src,
                                    traffic, fp64, emu, n, launch_ms),
        "gpu_launches": args.steps,
        "clocks": clk,
        "kernel_ms": launch_ms,
    }
    del out, p
    torch.cuda.synchronize()

    if rank == 0:
        # end to end through the host-buffer entry point (pinned host memory)
        e2e_steps = max(2, min(args.steps, args.e2e_steps))
        hin = torch.from_numpy(pts).pin_memory()
        hout = torch.empty((n, nh), dtype=tdt).pin_memory()
        ws = torch.empty(shm.eval_host_workspace_size(LMAX, tdt, 1 << 20), dtype=torch.uint8, device="cuda")
        shm.eval_host(hin, LMAX, hout, ws, stream=stream, strict=strict)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            shm.eval_host(hin, LMAX, hout, ws, stream=stream, strict=strict)
            stream.synchronize()
        dt = (time.perf_counter() - t0) / e2e_steps
        line["e2e"] = {"value": n * nh / dt, "unit": UNIT, "h2d_bytes_per_step": n * 3 * es,
                       "d2h_bytes_per_step": n * nh * es, "steps": e2e_steps,
                       "api": "shm_eval_host_ex (pinned host in/out, 1M-point chunks double-buffered)"
                              + (", SHM_STRICT_FP64" if strict else "")}
        del hin, hout, ws
        line["cpu_baseline"] = reference_arm_baseline(args)
        pts64 = pts.astype(np.float64)
        rate1, m1, _ = cpu_oracle_rate(pts64, LMAX, min(4.0, args.cpu_seconds / 2), nthreads=1)
        line["cpu_baseline"]["single_core"] = {"value": rate1, "unit": UNIT, "cores": 1,
                                               "sample": f"first {m1} grid points, 1 thread (in this process)"}
        if args.extras:
            line["extra"] = run_extras(args, shm, torch, inputs, stream, peaks, peaks_src, fp64)
        print(json.dumps(line), flush=True)
    return 0


ARITHMETIC = {
    ("f64", False): "binary64 throughout (SHM_STRICT_FP64): IEEE double multiply and fused multiply-add, CUDA's "
                    "binary64 rsqrt; with a rows-tma-emu variant part of the binary64 products are computed on the "
                    "integer pipes, bitwise equal to the DMUL results (shm_probe_dmul; GPU tests)",
    ("f64", True): "FP64 out, float-float arithmetic: binary64 for 1/r and the m = 0, 1 columns, float-float "
                   "(2 x FP32, ~48-bit significand) for the m >= 2 columns (72 of 100 values); within 1e-13 of "
                   "the l-shell norm of the FP64 oracle",
    ("f32", False): "FP32 (FP64 1/r for r < 1e-2; float-float m = 0, 1)",
    ("f32", True): "FP32 (FP64 1/r for r < 1e-2; float-float m = 0, 1)",
}

# DRAM bytes per point (dram__bytes_read.sum + dram__bytes_write.sum) of the
# evaluator at lmax 9 from ncu captures (profiles/), keyed by (dtype, launch
# variant); captures of the 96^3 grid are scaled to a full launch by the
# number of points.
TRAFFIC_PER_POINT = {
    # measured on the full 192^3 launch (1-pass captures)
    ("f64", "phased-hybrid-tma-128"): (174.86e6 + 5.75e9) / 7_077_888,
    ("f64", "phased-hybrid-128"): (169.99e6 + 5.61e9) / 7_077_888,
    ("f64", "staged-64"): (21.318144e6 + 648.666112e6) / 884_736,
    ("f64", "rows-tma-32"): (21.561344e6 + 652.576256e6) / 884_736,
    ("f64", "rows-tma-emu-o-32"): (21.400832e6 + 652.707840e6) / 884_736,
    ("f32", "staged-64"): (10.651648e6 + 294.209024e6) / 884_736,
}
# FP64 pipe instructions per point of the hybrid rows at lmax 9 (ncu
# sass__inst_executed_per_opcode of the 96^3 capture: DMUL 54 + DFMA 20).
HYBRID_DP_PER_POINT_L9 = 74


def roofline_object(dtype, hybrid, dp_pp, achieved_tflops, achieved_gbs, hbm_peak, peaks_src, traffic, fp64,
                    emu=0, n=0, launch_ms=0.0):
    """The bound of the evaluator kernel: the all-binary64 rows are FP64-pipe
    bound (242 FP64 instructions per point against 824 B per point: 3.4 ms
    at the measured FP64 rate against 0.9 ms of HBM); `achieved` counts the
    FP64 instructions the kernel executes (242 less the products it moves to
    the integer pipes).  The hybrid rows (74 FP64 instructions per point) and
    the FP32 rows are bound by the HBM traffic of their output.  The other
    figure is given beside it."""
    fp = {"achieved": achieved_tflops, "peak": fp64["tflops"], "unit": "TFLOP/s",
          "frac": achieved_tflops / fp64["tflops"],
          "def": f"{dp_pp} FP64 pipe instructions per point x 2 (FMA-equivalent flops) x points / mean launch time",
          "peak_source": fp64["source"]}
    hbm = {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": achieved_gbs / hbm_peak,
           "def": "algorithmic bytes (points in + rows out) / mean launch time", "peak_source": peaks_src}
    if dtype == "f64" and not hybrid:
        out = {"bound": "alu", "pipe": "fp64", **{k: fp[k] for k in ("achieved", "peak", "unit", "frac")},
               "traffic": traffic, "achieved_def": fp["def"], "peak_source": fp["peak_source"], "hbm": hbm}
        if emu:
            eq = 2.0 * STRICT_DP_PER_POINT_L9 * n / (launch_ms * 1e-3) / 1e12
            out["integer_pipe_products"] = {
                "per_point": emu, "note": "binary64 products computed on the integer pipes (dmul_int), bitwise the "
                                          "DMUL results; not counted in `achieved`",
                "binary64_equivalent_tflops": eq, "binary64_equivalent_frac_of_fp64_peak": eq / fp64["tflops"]}
        return out
    out = {"bound": "hbm", **{k: hbm[k] for k in ("achieved", "peak", "unit", "frac")}, "traffic": traffic,
           "achieved_def": hbm["def"], "peak_source": peaks_src}
    if dtype == "f64":
        out["fp64_pipe"] = fp
    return out


def run_extras(args, shm, torch, inputs, stream, peaks, peaks_src, fp64):
    """Other workloads, reported beside the headline (not part of `value`)."""
    res = {}
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    nh = (LMAX + 1) ** 2
    steps = max(5, min(args.steps, 50))
    g64 = inputs.dft_grid_points(N_SIDE)
    # the same grid with the default FP64 rows: float-float for m >= 2 (not binary64 arithmetic)
    if args.tune:
        shm.autotune(LMAX, torch.float64, g64.shape[0])
    per, region = measure_eval(shm, torch, g64, torch.float64, LMAX, steps, 3, stream)
    ms = statistics.mean(per)
    variant = shm.eval_variant(LMAX, torch.float64)
    hyb = "hybrid" in variant
    gbs = g64.shape[0] * (3 + nh) * 8 / (ms * 1e-3) / 1e9
    dp_pp = HYBRID_DP_PER_POINT_L9 if hyb else STRICT_DP_PER_POINT_L9
    tf = 2.0 * dp_pp * g64.shape[0] / (ms * 1e-3) / 1e12
    tpp = TRAFFIC_PER_POINT.get(("f64", variant))
    res["dft_grid_192cubed_f64out_ffarith_lmax9"] = {
        "value": g64.shape[0] * nh / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms, "launch_variant": variant,
        "dtype": "f64-out/ff-arith" if hyb else "f64", "arithmetic": ARITHMETIC[("f64", hyb)],
        "accuracy": "max normwise error 4.9e-14 on a 20,000-row sample of this grid (GPU tests; all-binary64 "
                    "rows: 1.4e-14; tolerance 1e-13)",
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                     "peak_source": peaks_src, "traffic": tpp * g64.shape[0] if tpp else None,
                     "fp64_pipe": {"achieved": tf, "peak": fp64["tflops"], "unit": "TFLOP/s",
                                   "frac": tf / fp64["tflops"], "peak_source": fp64["source"],
                                   "def": f"{dp_pp} FP64 pipe instructions per point"}}}
    # FP32 on the same grid: HBM-write bound
    g32 = g64.astype(np.float32)
    if args.tune:
        shm.autotune(LMAX, torch.float32, g32.shape[0])
    per, region = measure_eval(shm, torch, g32, torch.float32, LMAX, steps, 3, stream)
    ms = statistics.mean(per)
    gbs = g32.shape[0] * (3 + nh) * 4 / (ms * 1e-3) / 1e9
    res["dft_grid_192cubed_fp32_lmax9"] = {
        "value": g32.shape[0] * nh / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms,
        "launch_variant": shm.eval_variant(LMAX, torch.float32),
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": gbs / hbm_peak, "peak_source": peaks_src}}
    # the plain random-sphere set (65,600 points): latency-sized; binary64 and default rows
    sph = inputs.random_sphere_points(65_536)
    c_all, _, c_cores = cpu_oracle_rate(sph, LMAX, 2.0)
    c_one, c_m1, _ = cpu_oracle_rate(sph, LMAX, 2.0, nthreads=1)
    for strict, key in ((True, "random_sphere_65600_fp64_lmax9"), (False, "random_sphere_65600_f64out_ffarith_lmax9")):
        per, region = measure_eval(shm, torch, sph, torch.float64, LMAX, steps, 3, stream, strict=strict)
        ms = statistics.mean(per)
        res[key] = {"value": sph.shape[0] * nh / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms,
                    "launch_variant": shm.eval_variant(LMAX, torch.float64, strict=strict),
                    "arithmetic": ARITHMETIC[("f64", not strict)],
                    "cpu_oracle": {"value": c_all, "cores": c_cores, "unit": UNIT},
                    "cpu_oracle_single_core": {"value": c_one, "cores": 1, "unit": UNIT,
                                               "sample": f"first {c_m1} points"}}
    # the 1M-point random-sphere set in FP32 (HBM-write bound, fits in HBM many times over)
    sph32 = inputs.random_sphere_points(1 << 20).astype(np.float32)
    per, region = measure_eval(shm, torch, sph32, torch.float32, LMAX, steps, 3, stream)
    ms = statistics.mean(per)
    gbs = sph32.shape[0] * (3 + nh) * 4 / (ms * 1e-3) / 1e9
    c32, c32_m, c32_cores = cpu_oracle_rate(sph32.astype(np.float64), LMAX, 2.0)
    res["random_sphere_1M_fp32_lmax9"] = {
        "value": sph32.shape[0] * nh / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms,
        "cpu_oracle": {"value": c32, "cores": c32_cores, "unit": UNIT,
                       "sample": f"first {c32_m} points (FP64 oracle at the upcast FP32 inputs)"},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                     "peak_source": peaks_src, "note": "420 MB out: partly absorbed by the 126 MB L2"}}
    for fn in EXTRA_WORKLOADS:
        try:
            res.update(fn(args, shm, torch, inputs, stream, dict(peaks, fp64_probe=fp64), peaks_src))
        except Exception as e:  # reported, never silently dropped
            res[getattr(fn, "__name__", "extra")] = {"error": repr(e)}
    res["fp64_peak_probe"] = fp64
    return res


def extra_complex(args, shm, torch, inputs, stream, peaks, peaks_src):
    """Complex Y_l^m on the 192^3 grid (FP64 and FP32 out, interleaved re/im),
    and the angular interface on the grid's directions."""
    res = {}
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    nh = (LMAX + 1) ** 2
    g = inputs.dft_grid_points(N_SIDE)
    for dt, name, es, strict in _xdtypes(torch):
        p = torch.from_numpy(g).to(device="cuda", dtype=dt)
        out = torch.empty((p.shape[0], nh, 2), dtype=dt, device="cuda")
        fn = lambda: shm.eval_complex(p, LMAX, out=out, stream=stream, strict=strict)  # noqa: E731
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        per, _ = timed_launches(fn, max(5, min(args.steps, 30)), stream)
        ms = statistics.mean(per)
        gbs = p.shape[0] * (3 + 2 * nh) * es / (ms * 1e-3) / 1e9
        res[f"complex_dft_grid_192cubed_{name}_lmax9"] = {
            "value": p.shape[0] * nh / (ms * 1e-3), "unit": "complex Y_lm/s", "kernel_ms": ms,
            **xdtype_label(name),
            "roofline": (({"bound": "alu", **fp64_roofline("complex", p.shape[0], ms, peaks)}) if strict else
                         {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                          "peak_source": peaks_src}) | {"hbm_frac": gbs / hbm_peak}}
        del out, p
    # the angular interface on the same directions
    r = np.linalg.norm(g, axis=1)
    ang = np.stack([np.arccos(np.clip(g[:, 2] / r, -1, 1)), np.arctan2(g[:, 1], g[:, 0])], axis=1)
    for dt, name, es, strict in _xdtypes(torch):
        a = torch.from_numpy(ang).to(device="cuda", dtype=dt)
        out = torch.empty((a.shape[0], nh), dtype=dt, device="cuda")
        fn = lambda: shm.eval_angles(a, LMAX, out=out, stream=stream, strict=strict)  # noqa: E731
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        per, _ = timed_launches(fn, max(5, min(args.steps, 30)), stream)
        ms = statistics.mean(per)
        gbs = a.shape[0] * (2 + nh) * es / (ms * 1e-3) / 1e9  # (theta, phi) in, the row out
        res[f"angular_input_192cubed_directions_{name}_lmax9"] = {
            "value": a.shape[0] * nh / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms, **xdtype_label(name),
            "roofline": (({"bound": "alu", **fp64_roofline("angular", a.shape[0], ms, peaks)}) if strict else
                         {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                          "peak_source": peaks_src}) | {"hbm_frac": gbs / hbm_peak}}
        del out, a
    return res


# The extras' FP64 forms: "fp64" is binary64 throughout (SHM_STRICT_FP64);
# "f64out_ffarith" is the default FP64-out form with float-float m >= 2
# columns, labelled as such, never as FP64 arithmetic.
XDTYPES = ((None, "fp64", 8, True), (None, "f64out_ffarith", 8, False), (None, "fp32", 4, False))


def _xdtypes(torch):
    return tuple((torch.float32 if name == "fp32" else torch.float64, name, es, strict)
                 for _, name, es, strict in XDTYPES)


def fp64_roofline(kind, n_points, ms, peaks):
    """FP64-pipe fraction of an all-binary64 extra (measured DFMA rate of
    this run), from its FP64 instructions per point."""
    fp64 = peaks.get("fp64_probe")
    if not fp64:
        return {}
    dp = STRICT_X_DP_PER_POINT[kind]
    ach = 2.0 * dp * n_points / (ms * 1e-3) / 1e12
    return {"pipe": "fp64", "achieved": ach, "peak": fp64["tflops"], "unit": "TFLOP/s", "frac": ach / fp64["tflops"],
            "achieved_def": f"{dp} FP64 pipe instructions per point (ncu, lmax 9) x 2 x points / mean launch time",
            "fp64_peak_source": fp64["source"]}


def xdtype_label(name):
    if name == "fp64":
        return {"dtype": "f64", "arithmetic": "binary64 throughout (SHM_STRICT_FP64)"}
    if name == "f64out_ffarith":
        return {"dtype": "f64-out/ff-arith",
                "arithmetic": "FP64 out; binary64 1/r and m = 0, 1 columns, float-float (2 x FP32) m >= 2 columns; "
                              "within 1e-13 of the l-shell norm of the FP64 oracle"}
    return {"dtype": "f32", "arithmetic": "FP32 (FP64 1/r for r < 1e-2)"}


def extra_projectors(args, shm, torch, inputs, stream, peaks, peaks_src):
    """Fused projectors: 512 atoms, 40 bohr box, h = 0.2, spheres 2-5 bohr,
    lmax in {2, 3, 4}; FP64 and FP32.  The launch variant is picked by
    shm_projectors_autotune on this problem; the set-up (shm_projectors_prepare)
    runs once, and each timed call is shm_projectors_run: one persistent
    launch.  values/s = values per call / mean launch time."""
    res = {}
    prob = inputs.projector_problem()
    d = shm.DeviceProjectors(prob)
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    for dt, name, es in ((torch.float64, "fp64", 8), (torch.float32, "fp32", 4)):
        ws = d.workspace(dt)
        out = torch.empty(d.n_values, dtype=dt, device="cuda")
        tuned_ms = shm.projectors_autotune(d, dt, out, ws) if args.tune else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        shm.projectors_prepare(d, dt, ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        prepare_ms = e0.elapsed_time(e1)
        fn = lambda: shm.projectors_run(d, dt, out, ws, stream=stream)  # noqa: E731
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        per, _ = timed_launches(fn, max(5, min(args.steps, 30)), stream)
        ms = statistics.mean(per)
        graph = graph_replay_timing(torch, lambda st: shm.projectors_run(d, dt, out, ws, stream=st), stream=stream)
        err_bits = shm.projectors_check(ws, stream=stream)
        algo_bytes = d.n_values * es + d.n_points * 4
        gbs = algo_bytes / (ms * 1e-3) / 1e9
        key = "projectors_512atoms_f64out_ffarith" if es == 8 else f"projectors_512atoms_{name}"
        res[key] = {
            "value": d.n_values / (ms * 1e-3), "unit": "projector values/s", "ms_per_call": ms,
            "dtype": "f64-out/ff-arith" if es == 8 else "f32",
            "atoms": prob.n_atoms, "points": d.n_points, "values": d.n_values, "error_bits": err_bits,
            "launches_per_call": 1, "prepare_ms_once": prepare_ms, "launch_variant": shm.projectors_variant(dt),
            "autotune_best_ms": tuned_ms, "cuda_graph_replay": graph,
            "arithmetic": ("FP64 out: binary64 displacement (per-atom tables), r^2, 1/r and unit vector; "
                           "float-float (2 x FP32) log-grid index, radial cubic and harmonic rows; within 1e-13 "
                           "of the oracle" if es == 8 else "FP32 (FP64 1/r for |d| < 1e-2)"),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak, "peak_source": peaks_src, "algorithmic_bytes": algo_bytes,
                         "def": "values x element size + 4 B grid index per point, / mean launch time"}}
        del out, ws
    # FP64 with SHM_STRICT_FP64: binary64 tables, log-grid index and rows
    ws = d.workspace(torch.float64)
    out = torch.empty(d.n_values, dtype=torch.float64, device="cuda")
    shm.projectors_prepare(d, torch.float64, ws, stream=stream, strict=True)
    fn = lambda: shm.projectors_run(d, torch.float64, out, ws, stream=stream)  # noqa: E731
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    per, _ = timed_launches(fn, max(5, min(args.steps, 30)), stream)
    ms = statistics.mean(per)
    algo_bytes = d.n_values * 8 + d.n_points * 4
    gbs = algo_bytes / (ms * 1e-3) / 1e9
    form = shm.projectors_strict_form()
    roof = {"bound": "alu", "pipe": "fp64", "hbm_achieved": gbs, "hbm_peak": hbm_peak,
            "hbm_frac": gbs / hbm_peak, "hbm_unit": "GB/s", "hbm_peak_source": peaks_src,
            "algorithmic_bytes": algo_bytes}
    fp64 = peaks.get("fp64_probe")
    if fp64 and form in STRICT_PROJ_DP_PER_POINT:
        dp = STRICT_PROJ_DP_PER_POINT[form]
        ach = 2.0 * dp * d.n_points / (ms * 1e-3) / 1e12
        eq = 2.0 * STRICT_PROJ_DP_PER_POINT[1] * d.n_points / (ms * 1e-3) / 1e12
        roof.update({"achieved": ach, "peak": fp64["tflops"], "unit": "TFLOP/s", "frac": ach / fp64["tflops"],
                     "achieved_def": f"{dp} FP64 pipe instructions per point (ncu, this problem) x 2 x points / "
                                     "mean launch time", "peak_source": fp64["source"],
                     "binary64_equivalent_tflops": eq, "binary64_equivalent_frac_of_fp64_peak": eq / fp64["tflops"],
                     "binary64_equivalent_def": f"{STRICT_PROJ_DP_PER_POINT[1]} FP64 instructions per point of the "
                                                "form with every product on the FP64 pipe, at this time"})
    res["projectors_512atoms_fp64"] = {
        "value": d.n_values / (ms * 1e-3), "unit": "projector values/s", "ms_per_call": ms, "dtype": "f64",
        "launches_per_call": 1, "error_bits": shm.projectors_check(ws, stream=stream),
        "arithmetic": "binary64 throughout (SHM_STRICT_FP64)", "strict_form": form,
        "strict_form_def": "1: every product on the FP64 pipe; 2: the row's output products, 3: all its products "
                           "on the integer pipes (dmul_int, the same bits)",
        "roofline": roof}
    del out, ws
    # the oracle on the same problem (all host cores): the CPU baseline of this workload
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.projectors(prob)
    dt_cpu = time.perf_counter() - t0
    res["projectors_512atoms_fp64"]["cpu_oracle"] = {"value": d.n_values / dt_cpu, "unit": "projector values/s",
                                                     "cores": oracle.max_threads(0), "seconds": dt_cpu,
                                                     "sample": "the whole problem"}
    return res


def extra_serving(args, shm, torch, inputs, stream, peaks, peaks_src):
    """Serving: Poisson request streams (sizes log-uniform in [1e3, 4e6] points,
    lmax uniform in 0..9, dtype 50/50 FP32/FP64 -- FP64 requests with
    all-binary64 rows unless --serve-fp64 hybrid --, points generated on the
    device from each request's seed), continuous batching, per-rate throughput
    and latency percentiles.  A client thread collects every request as it
    completes (shm_serve_wait_any) and releases its rows; the client latency
    is submit -> that wait returning, the scheduler latency submit -> the
    scheduler seeing the request's last batch finish."""
    res = {}
    strict = args.serve_fp64 == "strict"
    for rate in args.serve_rates:
        reqs = inputs.serving_requests(rate, args.serve_seconds)
        with shm.Server(pool_bytes=48 << 30, max_slots=256, queue_capacity=2048, batch_points=8 << 20,
                        chunk_points=1 << 20, inflight_batches=3) as srv:
            stop = threading.Event()
            errors = []

            def collect():
                while True:
                    st, t, r = srv.wait_any(timeout_ms=20)
                    if st == 0:
                        srv.release(t)
                    elif st == 5:
                        if stop.is_set():
                            return
                    else:
                        errors.append(st)
                        srv.release(t)

            th = threading.Thread(target=collect, daemon=True)
            switch = sys.getswitchinterval()
            sys.setswitchinterval(1e-4)   # the collector gets the interpreter within 0.1 ms of a completion
            th.start()
            t0 = time.perf_counter()
            i = 0
            while i < len(reqs):
                # every request that has arrived, then sleep (without holding the
                # interpreter) until the next arrival
                now = time.perf_counter() - t0
                while i < len(reqs) and reqs[i].arrival_s <= now:
                    r = reqs[i]
                    srv.submit(r.n, r.lmax, r.dtype, seed=r.seed, strict=strict)
                    i += 1
                if i < len(reqs):
                    dt = reqs[i].arrival_s - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
            t_sub = time.perf_counter() - t0
            deadline = time.perf_counter() + 300
            while time.perf_counter() < deadline:
                st = srv.stats()
                if st["completed"] + st["rejected"] >= st["submitted"] and st["collected"] >= st["completed"]:
                    break
                time.sleep(0.001)
            wall = time.perf_counter() - t0
            stop.set()
            th.join(timeout=10)
            sys.setswitchinterval(switch)
            st = srv.stats()
        res[f"serve_poisson_{rate:g}_per_s"] = {
            "offered_req_per_s": rate, "submitted": st["submitted"], "submit_rate_achieved": len(reqs) / t_sub,
            "completed": st["completed"], "collected": st["collected"], "rejected_busy": st["rejected"],
            "completed_req_per_s": st["completed"] / wall, "value": st["harmonics_done"] / wall, "unit": UNIT,
            "client_lat_p50_ms": st["client_lat_p50_ms"], "client_lat_p99_ms": st["client_lat_p99_ms"],
            "client_lat_max_ms": st["client_lat_max_ms"],
            "sched_lat_p50_ms": st["lat_p50_ms"], "sched_lat_p99_ms": st["lat_p99_ms"],
            "batches": st["batches"], "gpu_busy_frac": st["busy_ms"] / (wall * 1e3), "wall_s": wall,
            "duration_s": args.serve_seconds, "pool_peak_bytes": st["pool_peak"],
            "fp64_rows": "all-binary64 (SHM_REQ_STRICT_FP64)" if strict else "hybrid (float-float m >= 2)",
            "request_errors": len(errors)}
    return res


def extra_spinor(args, shm, torch, inputs, stream, peaks, peaks_src):
    """Spin-1/2 spinor harmonics (Eq. 7) on the 192^3 grid: 2 (lmax+1)^2 two-component
    complex spinors per point (FP64: 6,400 B per point, 45 GB per launch)."""
    res = {}
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    nh = (LMAX + 1) ** 2
    g = inputs.dft_grid_points(N_SIDE)
    for dt, name, es, strict in _xdtypes(torch):
        p = torch.from_numpy(g).to(device="cuda", dtype=dt)
        out = torch.empty((p.shape[0], 2 * nh, 2, 2), dtype=dt, device="cuda")
        fn = lambda: shm.eval_spinor(p, LMAX, out=out, stream=stream, strict=strict)  # noqa: E731
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        per, _ = timed_launches(fn, max(5, min(args.steps, 20)), stream)
        ms = statistics.mean(per)
        gbs = p.shape[0] * (3 + 8 * nh) * es / (ms * 1e-3) / 1e9
        res[f"spinor_dft_grid_192cubed_{name}_lmax9"] = {
            "value": p.shape[0] * 2 * nh / (ms * 1e-3), "unit": "spinor harmonics/s", "kernel_ms": ms,
            **xdtype_label(name),
            "roofline": (({"bound": "alu", **fp64_roofline("spinor", p.shape[0], ms, peaks)}) if strict else
                         {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                          "peak_source": peaks_src}) | {"hbm_frac": gbs / hbm_peak}}
        del out, p
        torch.cuda.empty_cache()
    return res


EXTRA_WORKLOADS: list = [extra_complex, extra_spinor, extra_projectors, extra_serving]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["shm", "reference"], default="shm")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--grid", type=int, default=N_SIDE, help="grid side (192 = the benchmark workload; "
                    "smaller sides only for profiling captures)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--step-budget", type=float, default=None,
                    help="reference arm: seconds of oracle work per step (default: from --steps/--warmup)")
    ap.add_argument("--serve-seconds", type=float, default=30.0,
                    help="length of each Poisson request stream of the serving extra")
    ap.add_argument("--serve-rates", type=lambda v: [float(x) for x in v.split(",")],
                    default=[1000.0, 2000.0, 5000.0, 10000.0, 20000.0, 50000.0])
    ap.add_argument("--serve-fp64", choices=["strict", "hybrid"], default="strict",
                    help="rows of the FP64 requests of the serving extra")
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64",
                    help="f64 is the benchmark workload; f32 only for profiling captures")
    ap.add_argument("--variant", default=None, help="pin a launch variant by name (skips the autotuner)")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: split the one grid into contiguous per-rank parts (strong scaling) instead of "
                         "a grid per rank (replicas, weak scaling)")
    ap.add_argument("--arith", choices=["strict", "hybrid"], default="strict",
                    help="FP64 rows: strict = binary64 throughout (the benchmark workload), hybrid = the "
                         "default rows with float-float m >= 2 columns (profiling captures only)")
    ap.add_argument("--no-tune", dest="tune", action="store_false", default=True,
                    help="skip shm_autotune (use the library's default launch variant)")
    ap.add_argument("--extras", dest="extras", action="store_true", default=True)
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return 0
        else:
            dist.init_process_group("nccl")
    if args.impl == "reference":
        return run_reference(args, rank, world)
    try:
        return run_gpu(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            if dist.is_initialized():
                dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
