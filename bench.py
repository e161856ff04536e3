"""Benchmark: solved DOF/s to a 1e-10 relative residual on the 2-D
terrain-deformed GLL Poisson problem (64x64 elements, p = 8, 263,169 nodes),
FP32 gamma-cycle inside FP64 flexible CG, one GB300.

One step = one complete solve (lifting, outer iterations to tolerance,
u = w + v) with f and g already resident on the device.  The FP64-plain form
is measured the same way and reported beside it.  L2 is flushed (a 256 MB
write) between timed steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own replica of the problem
(independent problems, no collective on the data path); value = all ranks'
DOF / max-over-ranks time.  --impl reference times the FP64 CPU oracle (the
slow plain implementation the GPU path is checked against).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solved DOF/s to 1e-10 rel. residual (FP32-gamma vs FP64 plain)"
WORKLOAD = "terrain2d 64x64 quads p=8 (263,169 nodes), y'=y+0.1 sin(2 pi x)(1-y), 16 random Fourier modes"
GAMMA, ALPHA = 1, 2.0 / 3.0
SMOOTHER = "GLL line blocks R A_p P (Def. 3.2), alpha 2/3"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 256-problem batched and the 3-D 32-RHS measurements")
    ap.add_argument("--roofline-only", action="store_true",
                    help="only the kernel roofline measurements (used for ncu captures of single kernels)")
    ap.add_argument("--roofline-3d", action="store_true",
                    help="only the 3-D fine-level FP32 kernel measurements (small ncu captures)")
    ap.add_argument("--graph", type=int, default=2, choices=[0, 1, 2],
                    help="solve launch mode: 2 = one graph with a device-side loop (default), 1 = one graph "
                         "per iteration (profilers can see its kernels), 0 = plain stream launches")
    ap.add_argument("--profile", action="store_true",
                    help="only the warm-up and timed mixed-precision solves (for an ncu launch list)")
    ap.add_argument("--profile3d", action="store_true",
                    help="as --profile, on the 3-D 16^3 p = 7 workload with one right-hand side")
    ap.add_argument("--serving-only", action="store_true",
                    help="only the serving-stream measurement (prints its JSON object)")
    ap.add_argument("--probe", choices=["line2d", "line3d", "apply64", "setup", "apply3d_multi", "batch_passes",
                                        "batch_worklist", "summation", "apply_ff"],
                    help="launch one kernel a few times on its workload, nothing else (small ncu captures): "
                         "line2d / line3d = the fine-level FP32 line update (MODE 1) of every axis after one "
                         "apply, on the 2-D bench workload / the 3-D 16^3 p = 7 workload; apply64 = the 2-D "
                         "fine-level FP64 apply with fused p.Ap partials, then without")
    return ap.parse_args()


def dist_init(n):
    from paper_2504_10710_gb300 import replicas
    rank, world = replicas.rank_world()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")     # barrier and max-over-ranks only: no data-path collective
    return rank, world


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def make_problem(wl, glls):
    prob, coords = glls.problem_for(wl, glls.SMOOTHER_GLL, glls.RESTRICT_TRANSPOSE)
    f = wl.sample_rhs(coords)[0]
    g = wl.sample_dirichlet(coords)
    return prob, f, g


def run_ours(args, rank, world):
    import torch

    import __graft_entry__
    from paper_2504_10710_gb300 import glls, inputs, replicas

    __graft_entry__.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    wl = inputs.terrain3d(nrhs=1) if args.profile3d else inputs.terrain2d()
    prob, f, g = make_problem(wl, glls)
    N = prob.N
    stream = torch.cuda.current_stream()
    f_d = torch.tensor(f.ravel(), dtype=torch.float64, device="cuda")
    g_d = torch.tensor(g.ravel(), dtype=torch.float64, device="cuda")
    u_d = torch.zeros(N, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    prob.set_rhs(f_d, stream)
    prob.set_dirichlet(g_d, stream)
    tiles = prob.autotune()          # line-solve tiles per level / precision / direction (set-up, untimed)
    if args.roofline_only:
        print(json.dumps({"roofline": fp64_apply_roofline(prob, glls, torch),
                          "roofline_line_update": line_roofline(prob, glls, torch),
                          "roofline_hbm": smoother_rooflines(prob, glls, torch, inputs, flush)}))
        sys.exit(0)
    kernels = [0]

    def timed(precision, steps, warmup, clocks=None):
        o = glls.opts(tol=1e-10, gamma=GAMMA, alpha=ALPHA, precision=precision, use_graph=args.graph)
        its = []
        kernels[0] = 0
        for _ in range(warmup):
            prob.solve(u_d, o, stream)
        torch.cuda.synchronize()
        replicas.barrier(world)
        if clocks:
            clocks.start()
        ms = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = prob.solve(u_d, o, stream)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
            its.append(st.iterations)
            kernels[0] += st.kernels
        torch.cuda.synchronize()
        replicas.barrier(world)
        clk = clocks.stop() if clocks else None
        return ms / steps, its, clk

    clocks = ClockSampler(dev)
    ms_mixed, its_mixed, clk = timed(glls.PREC_MIXED, args.steps, args.warmup, clocks)
    launches = kernels[0]
    if args.profile or args.profile3d:
        print(json.dumps({"profile": True, "workload": wl.name, "ms_per_step": ms_mixed, "iterations": its_mixed}))
        sys.exit(0)
    ms_fp64, its_fp64, _ = timed(glls.PREC_FP64, max(3, args.steps // 2), 2)
    u_mixed = np.zeros(N)
    prob.solve(u_mixed, glls.opts(tol=1e-10, gamma=GAMMA, alpha=ALPHA, precision=glls.PREC_MIXED))
    u_fp64 = np.zeros(N)
    prob.solve(u_fp64, glls.opts(tol=1e-10, gamma=GAMMA, alpha=ALPHA, precision=glls.PREC_FP64))

    # end to end through the C ABI with host buffers (pinned), copies inside
    f_h = torch.tensor(f.ravel(), dtype=torch.float64).pin_memory()
    g_h = torch.tensor(g.ravel(), dtype=torch.float64).pin_memory()
    u_h = torch.zeros(N, dtype=torch.float64).pin_memory()
    o = glls.opts(tol=1e-10, gamma=GAMMA, alpha=ALPHA, precision=glls.PREC_MIXED)
    e2e = []
    for k in range(args.warmup + max(50, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob.set_rhs(f_h.numpy())
        prob.set_dirichlet(g_h.numpy())
        prob.solve(u_h.numpy(), o)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e.append(t1 - t0)
    e2e_s = float(np.mean(e2e))
    lat = np.array(e2e) * 1e3

    # the top kernel of the ncu launch list (the fine-level FP32 line update),
    # the FP64 outer apply, and the FP32 smoother / operator kernels against
    # HBM (bench workload and 3-D)
    roof = line_roofline(prob, glls, torch)
    roof64 = fp64_apply_roofline(prob, glls, torch)
    roof_ff = ff_apply_roofline(prob, glls, torch)
    roof_hbm = smoother_rooflines(prob, glls, torch, inputs, flush)
    serving = serving_run(glls, inputs) if not args.no_serving else None
    if serving is not None:
        # the same mix at an offered load below what the GPU sustains, so that
        # the latencies are not queueing-dominated (a second measurement
        # beside the specified 200/s stream)
        light = serving_run(glls, inputs, nreq=1000, rate=60.0)
        serving["below_capacity"] = {k: light[k] for k in ("requests", "completed", "offered", "achieved",
                                                         "latency_ms", "latency_resident_ms", "service_ms",
                                                         "grouping")}
    batch = batch_run(glls, inputs, torch) if not args.no_batch else None
    smoothers = smoother_compare(glls, inputs, torch)
    summation = summation_compare(glls, inputs, torch)
    multirhs = multirhs_run(glls, inputs, torch) if not args.no_batch else None

    # whole-job throughput: all ranks' DOF over the slowest rank's time
    ms_step = replicas.max_over_ranks(ms_mixed, world)
    value = replicas.aggregate_throughput(N, ms_mixed / 1e3, world)
    res = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 gamma-cycle / f64 outer Krylov, outer apply in float-float (2 x f32)", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "dof": N, "nrhs": 1, "gamma": GAMMA, "alpha": ALPHA, "smoother": SMOOTHER,
                   "restriction": "P^T", "levels": [8, 4, 2, 1], "tol": 1e-10, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "iterations_mixed": int(np.median(its_mixed)),
        "fp64_plain": {"value": world * N / (ms_fp64 / 1e3), "ms_per_step": ms_fp64, "iterations": int(np.median(its_fp64))},
        "mixed_over_fp64": ms_fp64 / ms_mixed,
        "e2e": {"value": world * N / e2e_s, "unit": "DOF/s", "h2d_bytes_per_step": 2 * 8 * N, "d2h_bytes_per_step": 8 * N},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)), "n": int(lat.size),
                       "what": "end to end through glls_set_rhs/set_dirichlet/solve with host buffers"},
        "clocks": clk,
        "smoothers": smoothers,
        "summation": summation,
        "roofline": _top_kernel_roofline(roof_hbm),
        "roofline_outer_apply_ff": roof_ff,
        "roofline_fp64_outer_apply": roof64,
        "roofline_line_update": roof,
        "roofline_hbm": roof_hbm,
        "gpu_launches": int(launches),
        "line_tiles": {f"l{l}_{pn}_ax{a}": c for (l, pn, a), (c, _us) in sorted(tiles.items()) if pn == "f32"},
        "serving": serving,
        "batch": batch,
        "multirhs_3d": multirhs,
    }
    return res, (u_mixed, u_fp64, wl)


def _top_kernel_roofline(roof_hbm):
    """The top kernel of the bench workload's ncu launch list (13 % of the
    solve): the fine-level FP32 apply of the smoothing steps,
    apply_p_kernel<float, 2, 8>, as measured in roofline_hbm (graph replay,
    the level L2-resident as inside a solve)."""
    for e in roof_hbm["kernels"]:
        if e["kernel"] == "apply_p_kernel<float, 2, 8>" and e["workload"] == "terrain2d_64x64_p8":
            r = {"bound": "hbm"}
            r.update({k: e[k] for k in ("kernel", "achieved", "peak", "unit", "frac", "traffic", "ms_per_launch",
                                        "algorithmic_bytes")})
            r["peak_source"] = roof_hbm["peak_source"]
            r["note"] = ("top kernel of the launch list (profiles/launches_terrain2d_64x64_p8_mixed.md); its 6 MB "
                         "level stays in L2 inside a solve, so it is bound by launch and phase latency rather than "
                         "HBM; the same kernels on a level several times L2 (3-D 32^3, p = 8) are in roofline_hbm")
            return r
    return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback 6800 GB/s (of fallback)"


def _traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary, or None when the kernel's source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        f = ln.split()
        if len(f) == 5 and not ln.startswith("#") and f[0] == kernel and f[1] == workload:
            src = os.path.join(ROOT, "paper_2504_10710_gb300", "csrc", f[3])
            try:
                sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
            except OSError:
                return None
            return float(f[2]) if sha == f[4] else None
    return None


def _time_graph(torch, fn, reps=50):
    """Average time of fn(stream) replayed `reps` times from one CUDA graph
    (as inside a solve: data stays in L2 between launches)."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):
            fn(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(reps):
            fn(s)
    g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):          # replay() launches on the current stream
        a.record()
        g.replay()
        b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def _time_cold(torch, fn, flush, reps=30):
    """Median time of single launches of fn(stream), L2 flushed before each
    (data comes from HBM), CUDA events on the launching stream."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):
            fn(s)
    ts = []
    for _ in range(reps):
        with torch.cuda.stream(s):
            # a read-only pass over a buffer twice the L2 evicts the kernel's
            # data without leaving dirty lines to write back during the launch
            flush.sum()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn(s)
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def _interior_random(torch, shape, dtype):
    x = torch.randn(shape, dtype=dtype, device="cuda")
    for ax in range(len(shape)):
        x.narrow(ax, 0, 1).zero_()
        x.narrow(ax, shape[ax] - 1, 1).zero_()
    return x.reshape(-1).contiguous()


def _fp64_peak_gflops(torch):
    """GB300's FP64 rate: 2 FP64 fused multiply-adds per clock per SM (the
    nominal 1.25 TFLOP/s over 152 SMs at 2,070 MHz), times this device's SM
    count and the maximum SM clock in MEASURED_PEAKS.json."""
    peaks, _ = _peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return 4.0 * sms * mhz / 1e3, sms, mhz


def fp64_apply_roofline(prob, glls, torch):
    """The bench workload's top kernel in the ncu launch list (13 % of the
    solve): the FP64 fine-level stiffness apply of the outer iteration, in
    the form the solve launches it: y = A p with the per-CTA partials of
    p.(A p) fused (flexible CG's p.Ap).  FP64-ALU bound.  FLOPs per launch from the
    sum-factorised algorithm: per element 4 (p+1)^3 FMA for the four 1-D
    contraction sweeps and 4 (p+1)^2 for the geometric factors, plus 2 (p+1)^2
    for the dot, 2 FLOP per FMA."""
    L = prob.levels - 1
    shape = prob.level_shape(L)
    p, E = 8, 64 * 64
    x = _interior_random(torch, shape, torch.float64)
    y = torch.zeros_like(x)
    part = torch.zeros(8192, dtype=torch.float64, device="cuda")
    ms = _time_graph(torch, lambda s: prob.apply_partials(L, x, y, part, s))
    flops = 2.0 * E * (4 * (p + 1) ** 3 + 5 * (p + 1) ** 2)
    ach = flops / (ms / 1e3) / 1e9
    peak, sms, mhz = _fp64_peak_gflops(torch)
    return {"bound": "alu", "kernel": "apply_p_kernel<double, 2, 8, DOT> (fine-level FP64 apply with the fused "
                                      "p.Ap partials, as launched by the outer iteration)",
            "achieved": ach, "peak": peak, "unit": "GFLOP/s", "frac": ach / peak,
            "traffic": _traffic("apply_p_kernel<double,2,8,DOT>", "terrain2d_64x64_p8"),
            "ms_per_launch": ms, "algorithmic_flops": flops,
            "peak_source": f"derived: 2 FP64 FMA/clk/SM x {sms} SMs (device properties) x {mhz:.0f} MHz "
                           "(MEASURED_PEAKS.json sm_max_mhz); no FP64 peak is measured",
            "note": "FMA counted as 2 FLOP; 50 launches replayed from a CUDA graph, CUDA events; y is not "
                    "re-zeroed between the timed launches (same work)"}


def ff_apply_roofline(prob, glls, torch):
    """The outer iteration's apply as the mixed-precision solve launches it:
    q = A p with the p.(A p) partials in float-float arithmetic
    (apply_ff_kernel<8>), timed by graph replay.  Bound by the FP32 pipe:
    the algorithm's FP32 instructions per element node are 12 per float-float
    multiply-add (one product, three fused multiply-adds, the six of the
    two-sum, two adds) over 2 (p+1) + 4 + 2 (p+1) of them, plus 3 per
    renormalisation (five), i.e. 48 (p+1) + 63; the peak is 128 FP32 lanes
    per SM per clock.  The FP64 work (splitting p, joining q, the dot) is a
    few operations per node beside it."""
    L = prob.levels - 1
    shape = prob.level_shape(L)
    p, E = prob.info.order[L], 64 * 64
    x = _interior_random(torch, shape, torch.float64)
    y = torch.zeros_like(x)
    part = torch.zeros(8192, dtype=torch.float64, device="cuda")
    ms = _time_graph(torch, lambda s: prob.apply_partials(L, x, y, part, s, ff=True))
    ops = float(E * (p + 1) ** 2 * (48 * (p + 1) + 63))
    ach = ops / (ms / 1e3) / 1e9
    peaks, _ = _peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = 128.0 * sms * mhz / 1e3
    return {"bound": "alu", "kernel": f"apply_ff_kernel<{p}> (fine-level outer apply with the fused p.Ap partials "
                                      "in float-float arithmetic, as launched by the mixed-precision solve)",
            "achieved": ach, "peak": peak, "unit": "G FP32-instructions/s", "frac": ach / peak,
            "traffic": _traffic(f"apply_ff_kernel<{p}>", "terrain2d_64x64_p8"),
            "ms_per_launch": ms, "algorithmic_fp32_instructions": ops,
            "peak_source": f"derived: 128 FP32 lanes/clk/SM x {sms} SMs (device properties) x {mhz:.0f} MHz "
                           "(MEASURED_PEAKS.json sm_max_mhz)",
            "note": "an instruction (FMA included) counted once; 50 launches replayed from a CUDA graph, CUDA "
                    "events; y is not re-zeroed between the timed launches (same work)"}


def line_roofline(prob, glls, torch):
    """The bench workload's second kernel in the ncu launch list: the FP32 line
    update of the fine level (line_block_kernel<float, 8>, MODE 1: x += alpha
    B_s^-1 (r - y) after y = A x), timed as the solve launches it, by graph
    replay (the level stays L2-resident, as inside a solve).  Algorithmic
    bytes per launch: r, y, x read and x written (16 B per node) plus the
    condensed line blocks along the axis (_line_operator_bytes)."""
    L = prob.levels - 1
    shape = prob.level_shape(L)
    N = int(np.prod(shape))
    p = prob.info.order[L]
    x = _interior_random(torch, shape, torch.float32)
    r = _interior_random(torch, shape, torch.float32)
    y = torch.zeros_like(x)
    prob.apply(L, x, y)
    peaks, src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    per_axis = []
    for ax in range(len(shape)):
        ms = _time_graph(torch, lambda s: prob.line_update(L, ax, ALPHA, r, y, x, s))
        byts = 16 * N + _line_operator_bytes(shape, p, ax, True)
        per_axis.append((ms, byts))
    ms = float(np.mean([m for m, _ in per_axis]))
    byts = float(np.mean([b for _, b in per_axis]))
    ach = byts / (ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": f"line_block_kernel<float, {p}> MODE 1 (fine-level line update of the "
                                      "smoothing step, Def. 3.2 line blocks), mean of the axes",
            "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": _traffic(f"line_block_kernel<float,{p}>_m1", "terrain2d_64x64_p8"),
            "ms_per_launch": ms, "algorithmic_bytes": byts,
            "per_axis_ms": [m for m, _ in per_axis], "peak_source": src,
            "note": "50 launches replayed from a CUDA graph per axis, CUDA events on the launching stream; the "
                    "level (9 MB per launch) stays in the 129 MB L2 between launches, as inside a solve"}


def _fp32_apply_kernel(d, p):
    """Name and traffic key of the FP32 apply kernel the library launches for
    a level of dimension d and order p (the dispatch in csrc/apply.cu)."""
    if d == 3 and p >= 4:
        return f"apply_eo3_kernel<float, {p}> (even-odd line apply)", f"apply_eo3_kernel<float,{p}>"
    if d == 3:
        return f"apply_col_kernel<{p}> (column apply)", f"apply_col_kernel<{p}>"
    return f"apply_p_kernel<float, {d}, {p}>", f"apply_p_kernel<float,{d},{p}>"


def _line_operator_bytes(shape, p, s, block):
    """FP32 bytes of the line operator along axis s read by one line solve:
    the Def. 3.2 line blocks (per element segment (p-1)p/2 + 2(p-1) values,
    per element-boundary vertex 2) or the band-1 (diag, off) pairs."""
    d = len(shape)
    n = shape[d - 1 - s]                      # nodes along s
    lines = int(np.prod([shape[d - 1 - a] - 2 for a in range(d) if a != s]))
    if not block:
        return 8 * lines * (n - 2)
    E = (n - 1) // p
    return 4 * lines * E * ((p - 1) * p // 2 + 2 * (p - 1)) + 8 * lines * (E - 1)


def smoother_rooflines(prob, glls, torch, inputs, flush, large=True):
    """FP32 smoother and operator kernels against HBM: the bench workload's
    fine level (L2-resident between launches, as inside a solve) and the 3-D
    16^3 p = 7 fine level (1.44M nodes; L2 flushed before every launch).
    Algorithmic bytes per launch: apply x + G + y (4 + 4 B per node plus
    ncomp (p+1)^d 4 B per element); line solve (B^-1 g) the line operator
    (_line_operator_bytes) + g + x 4 B each per node; smoothing step (apply +
    damped line update, the K2 step of the scope table) x, r read, x written,
    the line operator and G.  With `large`, also the 3-D 32^3 p = 8 fine
    level (17.0 M nodes), whose working set is several times L2."""
    peaks, src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = []

    def entry(kernel, work, ms, byts, cold, tkey):
        ach = byts / (ms / 1e3) / 1e9
        out.append({"kernel": kernel, "workload": work, "ms_per_launch": ms, "algorithmic_bytes": byts,
                    "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "traffic": _traffic(tkey, work) if tkey else None,
                    "l2": "flushed before each launch" if cold else "resident (graph replay)"})

    cases = [("terrain2d_64x64_p8", prob, False)] if prob is not None else []
    wl3 = inputs.terrain3d(nrhs=1)
    p3, _ = glls.problem_for(wl3)
    cases.append(("terrain3d_16x16x16_p7", p3, True))
    if large:
        # working set far above L2: the largest serving mesh (17.0 M nodes,
        # about 0.7 GB per FP32 apply)
        wl4 = inputs.terrain3d(nelem=32, order=8, nrhs=1)
        p4, _ = glls.problem_for(wl4)
        cases.append(("terrain3d_32x32x32_p8", p4, True))
    for work, pb, cold in cases:
        L = pb.levels - 1
        shape = pb.level_shape(L)
        N = int(np.prod(shape))
        d = len(shape)
        p = pb.info.order[L]
        E = int(np.prod([(n - 1) // p for n in shape]))
        G = (3 if d == 2 else 6) * E * (p + 1) ** d * 4
        x = _interior_random(torch, shape, torch.float32)
        y = torch.zeros_like(x)
        r = _interior_random(torch, shape, torch.float32)
        tm = (lambda fn: _time_cold(torch, fn, flush)) if cold else (lambda fn: _time_graph(torch, fn))
        kname, tkey = _fp32_apply_kernel(d, p)
        entry(kname, work, tm(lambda s: pb.apply(L, x, y, s)), 8 * N + G, cold, tkey)
        for ax in range(d):
            ob = _line_operator_bytes(shape, p, ax, True)
            entry(f"line_block_kernel<float, {p}> B^-1 g, axis {ax}", work,
                  tm(lambda s: pb.line_solve(L, ax, r, x, s)), 8 * N + ob, cold,
                  f"line_block_kernel<float,{p}>_ax{ax}")
            entry(f"line_block_kernel<float, {p}> MODE 1 line update, axis {ax}", work,
                  tm(lambda s: pb.line_update(L, ax, ALPHA, r, y, x, s)), 16 * N + ob, cold,
                  f"line_block_kernel<float,{p}>_m1_ax{ax}")
            entry(f"smoothing step (apply + line_block_kernel MODE 1), axis {ax}", work,
                  tm(lambda s: pb.smooth(L, ax, ALPHA, r, x, s)), 12 * N + G + ob, cold, None)
        if pb is not prob:
            pb.close()
    return {"peak_source": src, "kernels": out}


def smoother_compare(glls, inputs, torch, reps=10):
    """The bench workload (2-D 64x64, p = 8) with each line smoother the
    library offers, mixed precision, gamma = 1, to 1e-10: the Def. 3.2 line
    blocks at the paper's alpha = 2/3 (the default), the band-1 part of the
    GLL line systems at alpha = 0.5 (the largest that converges on this
    deformed grid) and the FEM line systems at the paper's alpha = 0.16.
    Iterations and CUDA-event time per solve (outputs on the device)."""
    wl = inputs.terrain2d()
    stream = torch.cuda.current_stream()
    out = {}
    for name, sm, alpha in (("gll_line_blocks", glls.SMOOTHER_GLL, 2.0 / 3.0),
                            ("gll_band1", glls.SMOOTHER_GLL_BAND1, 0.5),
                            ("fem", glls.SMOOTHER_FEM, 0.16)):
        prob, coords = glls.problem_for(wl, sm, glls.RESTRICT_TRANSPOSE)
        prob.set_rhs(wl.sample_rhs(coords)[0])
        prob.set_dirichlet(wl.sample_dirichlet(coords))
        u = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
        o = glls.opts(tol=1e-10, gamma=GAMMA, alpha=alpha, precision=glls.PREC_MIXED, max_iter=300)
        for _ in range(3):
            st = prob.solve(u, o, stream, raise_on_error=False)
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = prob.solve(u, o, stream, raise_on_error=False)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        out[name] = {"alpha": alpha, "iterations": int(st.iterations), "converged": st.status == glls.OK,
                     "ms_per_solve": float(np.median(ms)), "dof_per_s": prob.N / (float(np.median(ms)) / 1e3)}
        prob.close()
    return out


def summation_compare(glls, inputs, torch, reps=10):
    """The bench workload (2-D 64x64, p = 8, line blocks, alpha = 2/3, to
    1e-10) with the two direct stiffness summations: atomic (the default) and
    coloured (bitwise reproducible: one launch per element colour of the
    node-per-thread apply).  Mixed and FP64; iterations, CUDA-event time per
    solve, and whether repeated coloured solves gave the same bits."""
    wl = inputs.terrain2d()
    stream = torch.cuda.current_stream()
    out = {}
    for name, summ in (("atomic", glls.SUM_ATOMIC), ("colored", glls.SUM_COLORED)):
        prob, coords = glls.problem_for(wl, glls.SMOOTHER_GLL, glls.RESTRICT_TRANSPOSE, summation=summ)
        prob.set_rhs(wl.sample_rhs(coords)[0])
        prob.set_dirichlet(wl.sample_dirichlet(coords))
        for pname, prec in (("mixed", glls.PREC_MIXED), ("fp64", glls.PREC_FP64)):
            u = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
            first = None
            o = glls.opts(tol=1e-10, gamma=GAMMA, alpha=ALPHA, precision=prec, max_iter=300)
            same = True
            for _ in range(3):
                st = prob.solve(u, o, stream, raise_on_error=False)
                if first is None:
                    first = u.clone()
                same = same and bool(torch.equal(u, first))
            ms = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                st = prob.solve(u, o, stream, raise_on_error=False)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
                same = same and bool(torch.equal(u, first))
            out[f"{name}_{pname}"] = {"iterations": int(st.iterations), "converged": st.status == glls.OK,
                                      "ms_per_solve": float(np.median(ms)), "same_bits_every_solve": same}
        prob.close()
    return out


def multirhs_run(glls, inputs, torch, reps=3):
    """The 3-D multi-RHS workload: 16^3 hexahedra, p = 7 (1,442,897 nodes),
    32 seeded right-hand sides, FP32 gamma-cycle inside FP64 flexible CG, to
    1e-10, two ways: one problem created with nrhs = 32 (every kernel launch
    covers all right-hand sides, reading the mesh data once), and the problem
    plus 31 clones sharing its mesh data in one glls_solve_batch launch.
    Outputs on the device, CUDA events."""
    wl = inputs.terrain3d()
    stream = torch.cuda.current_stream()
    o = glls.opts(tol=1e-10, gamma=GAMMA, alpha=ALPHA, precision=glls.PREC_MIXED, max_iter=300)

    def timed(fn):
        st = fn()                  # first call captures the graph
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return st, float(np.median(ms))

    # one problem, nrhs = 32
    t0 = time.perf_counter()
    multi, coords = glls.problem_for(wl, glls.SMOOTHER_GLL, nrhs=wl.nrhs)
    F = np.ascontiguousarray(wl.sample_rhs(coords).reshape(wl.nrhs, -1))
    multi.set_rhs(F)
    multi.set_dirichlet(wl.sample_dirichlet(coords).ravel())
    setup_multi = time.perf_counter() - t0
    U = torch.zeros(wl.nrhs * multi.N, dtype=torch.float64, device="cuda")
    st, ms_multi = timed(lambda: multi.solve(U, o, stream, raise_on_error=False))
    its = np.array([x.iterations for x in st])
    dof = multi.N * wl.nrhs
    res = {"workload": wl.name, "nrhs": wl.nrhs, "dof": dof, "ms": ms_multi, "dof_per_s": dof / (ms_multi / 1e3),
           "converged": int(sum(x.status == glls.OK for x in st)),
           "iterations": {"median": float(np.median(its)), "max": int(its.max())}, "setup_s": setup_multi,
           "form": "one problem with nrhs = 32 (each launch covers all right-hand sides)"}
    multi.close()

    # the problem and 31 clones in one batch launch
    t0 = time.perf_counter()
    base, coords = glls.problem_for(wl, glls.SMOOTHER_GLL)
    g = wl.sample_dirichlet(coords)
    probs = [base] + [base.clone() for _ in range(len(F) - 1)]
    for pr, f in zip(probs, F):
        pr.set_rhs(f)
        pr.set_dirichlet(g)
    setup_s = time.perf_counter() - t0
    outs = [torch.zeros(base.N, dtype=torch.float64, device="cuda") for _ in probs]
    st, ms_clones = timed(lambda: glls.solve_batch(probs, outs, o, stream, raise_on_error=False))
    its = np.array([x.iterations for x in st])
    res["clones"] = {"ms": ms_clones, "dof_per_s": dof / (ms_clones / 1e3),
                     "converged": int(sum(x.status == glls.OK for x in st)),
                     "iterations": {"median": float(np.median(its)), "max": int(its.max())}, "setup_s": setup_s,
                     "form": "problem + 31 clones sharing the mesh data, one glls_solve_batch launch"}
    for pr in probs[1:]:
        pr.close()
    base.close()
    return res


def batch_run(glls, inputs, torch, reps=3):
    """The batched uneven workload: 256 independent 2-D problems (n x n
    elements, n ~ U{4..64}, p ~ U{4..12}, amplitude ~ U(0, 0.2); 26.3 M DOF)
    solved together in one graph launch (glls_solve_batch), FP32 gamma-cycle
    with the GLL line-block smoother (alpha = 2/3) inside FP64 flexible CG, to
    1e-10.  Outputs stay on the device; CUDA events around each launch."""
    ws = inputs.batch_uneven()
    t0 = time.perf_counter()
    probs = []
    for w in ws:
        pr, coords = glls.problem_for(w, glls.SMOOTHER_GLL)
        pr.set_rhs(w.sample_rhs(coords)[0])
        pr.set_dirichlet(w.sample_dirichlet(coords))
        probs.append(pr)
    setup_s = time.perf_counter() - t0
    outs = [torch.zeros(p.N, dtype=torch.float64, device="cuda") for p in probs]
    o = glls.opts(tol=1e-10, gamma=GAMMA, alpha=ALPHA, precision=glls.PREC_MIXED, max_iter=300)
    st = glls.solve_batch(probs, outs, o, raise_on_error=False)      # captures the batch graph
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = glls.solve_batch(probs, outs, o, stream, raise_on_error=False)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    its = np.array([x.iterations for x in st])
    dof = sum(p.N for p in probs)
    res = {"problems": len(probs), "dof": dof, "ms": float(np.median(ms)),
           "dof_per_s": dof / (float(np.median(ms)) / 1e3),
           "converged": int(sum(x.status == glls.OK for x in st)),
           "iterations": {"median": float(np.median(its)), "p90": float(np.percentile(its, 90)),
                          "max": int(its.max())},
           "smoother": SMOOTHER, "setup_s": setup_s,
           "form": "one graph launch, one branch per problem (each with its own device-side loop)"}
    # the work-list form: one launch per step over all problems of an order chain
    outs_w = [torch.zeros(p.N, dtype=torch.float64, device="cuda") for p in probs]
    t0 = time.perf_counter()
    st_w = glls.solve_batch(probs, outs_w, o, stream, raise_on_error=False, worklist=True)   # plan + capture
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    ms_w = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st_w = glls.solve_batch(probs, outs_w, o, stream, raise_on_error=False, worklist=True)
        b.record(stream)
        b.synchronize()
        ms_w.append(a.elapsed_time(b))
    its_w = np.array([x.iterations for x in st_w])
    diff = max(float((x - y).abs().max() / y.abs().max()) for x, y in zip(outs_w, outs))
    res["worklist"] = {"ms": float(np.median(ms_w)), "dof_per_s": dof / (float(np.median(ms_w)) / 1e3),
                       "converged": int(sum(x.status == glls.OK for x in st_w)),
                       "iterations": {"median": float(np.median(its_w)), "max": int(its_w.max())},
                       "kernels_per_launch": int(st_w[0].kernels),
                       "groups": len({tuple(p.info.order[:p.info.levels]) for p in probs}),
                       "plan_s": plan_s, "max_rel_diff_vs_branches": diff,
                       "form": "glls_solve_batch_worklist: problems grouped by order chain, one launch per step "
                               "over each group's work list of (problem, level, tile range) items, one graph "
                               "branch and device-side loop per group"}
    for p in probs:
        p.close()
    return res


def serving_run(glls, inputs, nreq=2000, rate=200.0, slots=8, budget_gb=200, max_group=8, max_wait_s=240.0):
    """The serving stream: ``nreq`` Poisson arrivals (mean ``rate`` per
    second) over a pool of 16 2-D meshes (batch-uneven sizes) and 8 3-D meshes
    (n^3 elements, n ~ U{8..32}, p ~ U{4..8}, including 32^3 at p = 8), each
    request one mixed-precision solve to 1e-10.  The meshes are registered
    with the server (coordinates copied once) but nothing is set up before
    the stream starts: the first request on a mesh pays its set-up, later
    concurrent requests on a busy mesh run on clones, and queued requests of
    one mesh are solved together as one multi-right-hand-side solve (up to
    ``max_group``; continuous batching).  Latency is submission
    to the solution in host memory.  The client-side input generation
    (coordinates, right-hand sides) happens before the stream and is not
    part of any figure."""
    from concurrent.futures import ThreadPoolExecutor
    meshes, reqs = inputs.serving_stream(nreq=nreq, rate=rate)
    t0 = time.perf_counter()

    def make(w):
        xi, _ = glls.gll(w.order)
        c = np.ascontiguousarray(w.coords(xi), dtype=np.float64).reshape(w.dim, -1)
        F = [np.ascontiguousarray(f(*c), dtype=np.float64) for f in w.rhs]
        g = np.ascontiguousarray(w.sample_dirichlet(c), dtype=np.float64)
        return c, F, g
    with ThreadPoolExecutor(8) as ex:
        data = list(ex.map(make, meshes))
    inputs_s = time.perf_counter() - t0
    srv = glls.Server(budget_bytes=budget_gb << 30, slots=slots)
    srv.set_max_group(max_group)
    ids = [srv.register(w.dim, w.nelem, w.order, c) for w, (c, _, _) in zip(meshes, data)]
    o = glls.opts(tol=1e-10, gamma=GAMMA, alpha=ALPHA, precision=glls.PREC_MIXED, max_iter=300)
    outs = {}
    tickets = []
    t0 = time.perf_counter()
    lag = []
    for k, (arr, mi, ri) in enumerate(reqs):
        delay = t0 + arr - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        else:
            lag.append(-delay)
        _, F, g = data[mi]
        out = np.empty(F[ri].size)
        tickets.append((srv.submit_mesh(ids[mi], F[ri], g, o, out), mi, time.perf_counter() - t0))
    submit_span = time.perf_counter() - t0
    # collect with a deadline: a request still unfinished then is reported,
    # not waited for
    res_all, pending = [], list(tickets)
    deadline = time.perf_counter() + max_wait_s
    while pending and time.perf_counter() < deadline:
        left = []
        for t, mi, ts in pending:
            st, stats = srv.poll(t, wait=False)
            if st == glls.NOT_READY:
                left.append((t, mi, ts))
            else:
                res_all.append((mi, st, ts, stats.solve_ms, stats.queue_ms, stats.setup_ms, stats.setup_kind,
                                stats.iterations, stats.group))
        pending = left
        if pending:
            time.sleep(0.002)
    for t, _, _ in pending:
        srv.cancel(t)
    info = srv.info()
    srv.close()
    ok = [r for r in res_all if r[1] == glls.OK]
    end = max(ts + lat / 1e3 for _, _, ts, lat, *_ in res_all)
    dof = sum(data[mi][2].size for mi, st, *_ in res_all if st == glls.OK)
    dof_offered = sum(data[mi][2].size for _, mi, _ in reqs)
    span = reqs[-1][0]
    lat = np.array([r[3] for r in ok])
    resident = np.array([r[3] for r in ok if r[6] == 0])
    creates = [(meshes[r[0]].name, r[5]) for r in res_all if r[6] == 1]
    clones = [r[5] for r in res_all if r[6] == 2]
    its = np.array([r[7] for r in ok])
    service = np.array([r[3] - r[4] - r[5] for r in ok])
    gsz = np.array([r[8] for r in ok])

    def pct(a, q):
        return float(np.percentile(a, q)) if len(a) else None
    d3 = [i for i, w in enumerate(meshes) if w.dim == 3]
    return {"requests": nreq, "completed": len(ok), "failed": len(res_all) - len(ok), "unfinished": len(pending),
            "offered": {"requests_per_s": nreq / span, "dof_per_s": dof_offered / span, "arrival_span_s": span},
            "achieved": {"requests_per_s": len(ok) / end, "dof_per_s": dof / end, "wall_s": end},
            "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": float(lat.max()) if len(lat) else None,
                           "what": "submission to solution in host memory (queue, set-up if any, solve)"},
            "latency_resident_ms": {"p50": pct(resident, 50), "p99": pct(resident, 99), "n": int(len(resident)),
                                    "what": "requests served by an instance that was already resident"},
            "setup": {"creates": len(creates), "create_ms": {n: round(ms, 1) for n, ms in creates},
                      "clones": len(clones), "clone_ms_median": pct(np.array(clones), 50),
                      "what": "paid inside the latency of the request that triggered it"},
            "service_ms": {"p50": pct(service, 50), "p99": pct(service, 99),
                           "what": "latency minus queue and set-up: the solve itself, on a GPU shared with the "
                                   "other slots"},
            "grouping": {"max_group": max_group, "grouped_requests": int((gsz > 1).sum()),
                         "group_sizes": {str(k): int((gsz == k).sum()) for k in sorted(set(gsz.tolist()))}},
            "iterations": {"median": pct(its, 50), "max": int(its.max()) if len(its) else None},
            "submit_lag_ms": {"p99": 1e3 * pct(np.array(lag), 99) if lag else 0.0, "late": len(lag)},
            "slots": slots, "budget_gb": budget_gb, "resident_bytes_end": int(info.resident_bytes),
            "server_clones": int(info.clones), "inputs_s": inputs_s,
            "pool": {"2d": [w.name for w in meshes if w.dim == 2], "3d": [meshes[i].name for i in d3],
                     "dof_max": int(max(data[i][2].size for i in d3))}}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_worker(barrier, results):
    """One host core: build the oracle hierarchy (untimed), wait for the
    others, then one full FP64 oracle solve of the bench workload."""
    from oracle import solve as osolve
    from paper_2504_10710_gb300 import inputs
    wl = inputs.terrain2d()
    fine, h = osolve.build(wl, restriction="transpose")
    barrier.wait()
    t0 = time.perf_counter()
    r = osolve.solve(wl, gamma=GAMMA, alpha=ALPHA, tol=1e-10, maxit=200, hierarchy=h)
    results.put((time.perf_counter() - t0, fine.N, r.iterations[0]))


def oracle_baseline(wl, u_ref_gpu=None):
    """The FP64 oracle on the host cores: one solve on one core (with its
    result, used for parity), then one solve per core on all cores at once
    (spawned processes, one BLAS thread each; throughput = cores x DOF / wall
    time from a common start)."""
    import multiprocessing as mp
    from oracle import solve as osolve
    t0 = time.perf_counter()
    fine, h = osolve.build(wl, restriction="transpose")
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = osolve.solve(wl, gamma=GAMMA, alpha=ALPHA, tol=1e-10, maxit=200, hierarchy=h)
    ts = time.perf_counter() - t0
    N = fine.N
    one_core = N / ts
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores + 1)
    results = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(barrier, results)) for _ in range(cores)]
    for pr in procs:
        pr.start()
    all_cores, wall = None, None
    try:
        barrier.wait(timeout=600)
        t0 = time.perf_counter()
        got = [results.get(timeout=600) for _ in procs]
        wall = time.perf_counter() - t0
        all_cores = sum(n for _, n, _ in got) / wall
    except Exception as exc:        # report the one-core figure if the pool fails
        print(f"all-core oracle baseline failed: {exc!r}", file=sys.stderr)
    for pr in procs:
        pr.join(timeout=60)
        if pr.is_alive():
            pr.terminate()
    model = _cpu_model()
    if all_cores is not None:
        out = {"value": all_cores, "unit": "DOF/s", "cores": cores, "kind": "oracle", "cpu_model": model,
               "one_core_value": one_core,
               "sample": f"{cores} concurrent full FP64 solves of the same workload, one per host core "
                         f"({wall:.1f} s wall from a common start; {r.iterations[0]} FCG iterations each); "
                         f"one core alone: {ts:.1f} s per solve; setup {tb:.1f} s excluded"}
    else:
        out = {"value": one_core, "unit": "DOF/s", "cores": 1, "kind": "oracle", "cpu_model": model,
               "sample": f"one full FP64 solve of the same workload ({r.iterations[0]} FCG iterations, "
                         f"{ts:.1f} s; setup {tb:.1f} s excluded)"}
    return out, r


def probe(name, reps=3):
    """Launch one kernel `reps` times per axis on its workload (see --probe);
    `setup` instead creates the 3-D serving meshes, the 2-D bench mesh and the
    3-D 16^3 p = 7 mesh one after another and prints the set-up phases."""
    import torch

    import __graft_entry__
    from paper_2504_10710_gb300 import glls, inputs
    __graft_entry__.build()
    if name == "summation":
        print(json.dumps({"probe": name, "summation": summation_compare(glls, inputs, torch)}))
        return
    if name == "batch_worklist":
        # the batched uneven workload's work-list form with two passes of its
        # loop captured inline (GLLS_WORKLIST_PASSES), so that ncu lists the
        # list kernels of those passes; not a solve to tolerance
        os.environ["GLLS_WORKLIST_PASSES"] = "2"
        ws = inputs.batch_uneven()
        probs = []
        for w in ws:
            pr, coords = glls.problem_for(w, glls.SMOOTHER_GLL)
            pr.set_rhs(w.sample_rhs(coords)[0])
            pr.set_dirichlet(w.sample_dirichlet(coords))
            probs.append(pr)
        outs = [torch.zeros(p.N, dtype=torch.float64, device="cuda") for p in probs]
        o = glls.opts(tol=1e-10, gamma=GAMMA, alpha=ALPHA, precision=glls.PREC_MIXED, max_iter=300)
        for _ in range(reps):
            glls.solve_batch(probs, outs, o, raise_on_error=False, worklist=True)
        torch.cuda.synchronize()
        print(json.dumps({"probe": name, "problems": len(probs), "reps": reps}))
        for p in probs:
            p.close()
        return
    if name == "batch_passes":
        # the batched uneven workload with the iteration cap at 1, 2, 4, 8:
        # the fixed cost and the cost per pass of each batch form
        ws = inputs.batch_uneven()
        probs = []
        for w in ws:
            pr, coords = glls.problem_for(w, glls.SMOOTHER_GLL)
            pr.set_rhs(w.sample_rhs(coords)[0])
            pr.set_dirichlet(w.sample_dirichlet(coords))
            probs.append(pr)
        outs = [torch.zeros(p.N, dtype=torch.float64, device="cuda") for p in probs]
        stream = torch.cuda.current_stream()
        res = {}
        for form in ("branches", "worklist"):
            for cap in (1, 2, 4, 8, 300):
                o = glls.opts(tol=1e-10, gamma=GAMMA, alpha=ALPHA, precision=glls.PREC_MIXED, max_iter=cap)
                glls.solve_batch(probs, outs, o, stream, raise_on_error=False, worklist=form == "worklist")
                ms = []
                for _ in range(3):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    glls.solve_batch(probs, outs, o, stream, raise_on_error=False, worklist=form == "worklist")
                    b.record(stream)
                    b.synchronize()
                    ms.append(a.elapsed_time(b))
                res[f"{form}_cap{cap}"] = float(np.median(ms))
        print(json.dumps({"probe": name, "ms": res}))
        for p in probs:
            p.close()
        return
    if name == "apply3d_multi":
        # the 3-D fine-level FP32 apply for 32 stacked vectors (geometry read
        # once per launch), then for one vector
        wl = inputs.terrain3d(nrhs=1)
        prob, _ = glls.problem_for(wl, glls.SMOOTHER_GLL)
        L = prob.levels - 1
        shape = prob.level_shape(L)
        k = 32
        xs = torch.cat([_interior_random(torch, shape, torch.float32) for _ in range(k)])
        ys = torch.zeros_like(xs)
        for _ in range(reps):
            prob.apply_multi(L, xs, ys, k)
        x1, y1 = xs[:xs.numel() // k].clone(), torch.zeros(xs.numel() // k, dtype=torch.float32, device="cuda")
        for _ in range(reps):
            prob.apply(L, x1, y1)
        torch.cuda.synchronize()
        print(json.dumps({"probe": name, "workload": wl.name, "nrhs": k, "reps": reps}))
        prob.close()
        return
    if name == "setup":
        meshes, _ = inputs.serving_stream(nreq=10)
        wls = [inputs.terrain2d(), inputs.terrain3d(nrhs=1)] + [w for w in meshes if w.dim == 3]
        for w in wls:
            xi, _ = glls.gll(w.order)
            c = np.ascontiguousarray(w.coords(xi)).reshape(w.dim, -1)
            t0 = time.perf_counter()
            pr = glls.Problem(w.dim, w.nelem, w.order, c)
            ms = 1e3 * (time.perf_counter() - t0)
            inf = pr._info()
            print(json.dumps({"workload": w.name, "dof": int(pr.N), "create_ms": round(ms, 1),
                              "phases_ms": dict(zip(["coords", "geometry", "lines", "transfers", "coarse", "upload"],
                                                    [round(v, 1) for v in inf.setup_phase_ms])),
                              "coarse": [int(inf.coarse_unknowns), int(inf.coarse_cr_levels)],
                              "device_gb": round(inf.device_bytes / 2**30, 2)}), flush=True)
            pr.close()
        return
    wl = inputs.terrain3d(nrhs=1) if name == "line3d" else inputs.terrain2d()
    prob, _ = glls.problem_for(wl, glls.SMOOTHER_GLL, glls.RESTRICT_TRANSPOSE)
    L = prob.levels - 1
    shape = prob.level_shape(L)
    if name == "apply_ff":
        # the float-float outer apply launched reps times, then both outer
        # applies timed by graph replay
        x = _interior_random(torch, shape, torch.float64)
        y = torch.zeros_like(x)
        part = torch.zeros(8192, dtype=torch.float64, device="cuda")
        for _ in range(reps):
            y.zero_()
            prob.apply_partials(L, x, y, part, ff=True)
        torch.cuda.synchronize()
        out = {"probe": name, "ff": ff_apply_roofline(prob, glls, torch),
               "fp64": fp64_apply_roofline(prob, glls, torch)}
        prob.close()
        # 3-D 16^3, p = 7: both outer applies by graph replay
        w3 = inputs.terrain3d(nrhs=1)
        p3, _ = glls.problem_for(w3, glls.SMOOTHER_GLL, glls.RESTRICT_TRANSPOSE)
        L3 = p3.levels - 1
        x3 = _interior_random(torch, p3.level_shape(L3), torch.float64)
        y3 = torch.zeros_like(x3)
        part3 = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
        out["ms_3d_16x16x16_p7"] = {
            "ff": _time_graph(torch, lambda s: p3.apply_partials(L3, x3, y3, part3, s, ff=True)),
            "fp64": _time_graph(torch, lambda s: p3.apply_partials(L3, x3, y3, part3, s))}
        p3.close()
        print(json.dumps(out))
        return
    if name == "apply64":
        x = _interior_random(torch, shape, torch.float64)
        y = torch.zeros_like(x)
        part = torch.zeros(8192, dtype=torch.float64, device="cuda")
        for _ in range(reps):
            y.zero_()
            prob.apply_partials(L, x, y, part)
        for _ in range(reps):           # the same apply without the partials
            prob.apply(L, x, y)
    else:
        x = _interior_random(torch, shape, torch.float32)
        r = _interior_random(torch, shape, torch.float32)
        y = torch.zeros_like(x)
        for ax in range(len(shape)):
            for _ in range(reps):
                prob.apply(L, x, y)
                prob.line_update(L, ax, ALPHA, r, y, x)
    torch.cuda.synchronize()
    print(json.dumps({"probe": name, "workload": wl.name, "reps": reps}))
    prob.close()


def main():
    args = parse()
    if args.serving_only:
        import __graft_entry__
        from paper_2504_10710_gb300 import glls, inputs
        __graft_entry__.build()
        print(json.dumps(serving_run(glls, inputs)))
        return
    rank, world = dist_init(args.gpus)
    if args.impl == "reference":
        if rank != 0:
            return
        from paper_2504_10710_gb300 import inputs
        wl = inputs.terrain2d()
        from oracle import solve as osolve
        from oracle.discretize import lift
        fine, h = osolve.build(wl, restriction="transpose")
        # iterations of a full solve (untimed), then one bounded sample per
        # step: one outer FCG iteration (gamma-cycle, FP64 apply, dots, updates)
        its_full = osolve.solve(wl, gamma=GAMMA, alpha=ALPHA, tol=1e-10, maxit=200, hierarchy=h).iterations[0]
        f0, _v = lift(fine, wl.sample_rhs(fine.coords)[0], wl.sample_dirichlet(fine.coords))
        r = f0.copy()
        z = h.precondition(r, GAMMA, ALPHA, 1)
        pdir = z.copy()
        rz = float(np.vdot(r, z))
        times = []
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            q = fine.apply(pdir)
            alpha = rz / float(np.vdot(pdir, q))
            r_new = r - alpha * q
            z_new = h.precondition(r_new, GAMMA, ALPHA, 1)
            rz_new = float(np.vdot(r_new, z_new))
            beta = (rz_new - float(np.vdot(r, z_new))) / rz
            pdir = z_new + beta * pdir
            r, rz = r_new, rz_new
            if k >= args.warmup:
                times.append(time.perf_counter() - t0)
        step_s = float(np.mean(times))
        val = fine.N / (its_full * step_s)
        sample = (f"one outer FCG iteration of the FP64 oracle per step (gamma-cycle + FP64 apply + dots); "
                  f"value = DOF / ({its_full} iterations x {1e3 * step_s:.0f} ms mean step)")
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": val, "unit": "DOF/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "dof": fine.N, "gamma": GAMMA, "alpha": ALPHA, "tol": 1e-10},
            "iterations": int(its_full),
            "cpu_baseline": {"value": val, "unit": "DOF/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return
    if args.probe:
        probe(args.probe)
        return
    if args.roofline_3d:
        import torch

        import __graft_entry__
        from paper_2504_10710_gb300 import glls, inputs
        __graft_entry__.build()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        print(json.dumps({"roofline_hbm": smoother_rooflines(None, glls, torch, inputs, flush)}))
        return
    res, (u_mixed, u_fp64, wl) = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            cb, r = oracle_baseline(wl)
            res["cpu_baseline"] = cb
            ref = r.u[0].ravel()
            res["parity_vs_oracle"] = {
                "fp64_rel_err": float(np.abs(u_fp64 - ref).max() / np.abs(ref).max()),
                "mixed_rel_err": float(np.abs(u_mixed - ref).max() / np.abs(ref).max()),
                "oracle_iterations": r.iterations[0]}
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
