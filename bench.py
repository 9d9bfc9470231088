"""Throughput of the fused RD3Q41 collide-and-stream update on GB300.

One step = one fused pull update (stream + moments + energy-conserving
equilibrium + BGK) of every node of the grid: one kernel launch.

Default workload: 512^3 periodic bcc grid (2 * 512^3 nodes), thermoacoustic
case (Gaussian density pulse of amplitude 1e-2, sigma = 8 cells, at the
centre, plus a seeded 16^3-Fourier-box temperature perturbation of max 1e-3),
nu = 0.01, FP32 arithmetic with populations stored as FP16 deviations
h = f/w - 1.  The other storage precisions are timed on the same workload and
reported under "by_precision".

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--n 512] [--precision f16]
For N > 1 (torchrun), every rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}
DTYPE_NAME = {"f64": "f64", "f32": "f32", "f16": "f32 (f16 storage)", "bf16": "f32 (bf16 storage)"}
NU = 0.01
# Field values in the compute type (4 B, FP64 storage 8 B) one nonideal step moves per node: the
# density pass writes rho, mu, F (3); the field pass reads them and writes mu, F, lap F, the
# isotropic part of I_ab and grad rho (3 + 7); the force pass reads those seven and rho and
# writes g (8 + 3); the step reads g (3).  The populations are gathered twice (density pass,
# step) and written once: 3 x 41 stored values.
NONIDEAL_FIELD_VALUES = 27
STEP_KERNEL_SOURCES = ["lb_common.cuh", "lb_kernels.cuh", "lb_step_tma.cuh", "lb_step_ws.cuh", "lb_step_f32.cu",
                       "lb_step_f64.cu"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=512)
    p.add_argument("--precision", default="f16", choices=list(BYTES))
    p.add_argument("--stochastic", action="store_true",
                   help="with --precision bf16: the stochastic BF16 store (lb_set_stochastic_rounding) in the "
                        "timed runs of that precision")
    p.add_argument("--no-secondary", action="store_true", help="skip the other storage precisions")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-batch", action="store_true", help="skip the batched 64-simulation sweep")
    p.add_argument("--no-walls", action="store_true", help="skip the run with kinetic walls normal to z")
    p.add_argument("--no-nonideal", action="store_true", help="skip the run of the nonideal (van der Waals) fluid")
    p.add_argument("--no-accuracy", action="store_true",
                   help="skip the error of the reduced-precision runs against the GPU FP64 mode")
    p.add_argument("--batch-steps", type=int, default=1000)
    p.add_argument("--batch-sims", type=int, default=64, help="simulations in the batched sweep")
    p.add_argument("--kernel", type=int, default=None,
                   help="step kernel for the headline run (LB_KERNEL_* id); default: the fastest that applies")
    p.add_argument("--no-surrogate", action="store_true", help="skip the surrogate convolution timings")
    p.add_argument("--conv", action="store_true",
                   help="only time the surrogate's convolution kernels (forward and weight gradient) and print "
                        "one JSON object")
    p.add_argument("--conv-impl", default="both", choices=["tcgen05", "mma_sync", "both"])
    p.add_argument("--conv-ops", default="fwd,wgrad", help="comma list of fwd, wgrad")
    p.add_argument("--conv-layers", default="16x32,32x32,32x16")
    p.add_argument("--conv-batch", default="1,4")
    p.add_argument("--conv-reps", type=int, default=20)
    p.add_argument("--conv-warmup", type=int, default=3)
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def _strip_comments(src):
    """C++ source without // and /* */ comments, trailing blanks and blank lines (string and
    character literals kept), so that the hash changes with the code only."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            while i < n and src[i] != "\n":
                i += 1
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = (ln.rstrip() for ln in "".join(out).split("\n"))
    return "\n".join(ln for ln in lines if ln)


def kernel_hash():
    """Hash of the step-kernel sources' code (comments and blank lines ignored)."""
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1909_08406_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(precision, kernel_id, n):
    """dram read+write bytes per launch of the step kernel that ran, from the committed ncu
    summary (keyed "<precision>/<kernel id>"), if it was taken on the current kernel sources;
    else None."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(f"{precision}/{kernel_id}")
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    # scale a smaller capture to this grid by the node count (traffic ~ nodes)
    return e["dram_bytes_per_launch"] * (2 * n ** 3) / e["nodes"]


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        # nvidia-smi's start-up (NVML initialisation) stalls work on the GPU for a few hundred
        # ms: wait for its first sample so that the stall stays out of the timed region
        t0 = time.time()
        while time.time() - t0 < 10.0 and self.proc.poll() is None:
            if os.path.getsize(self.file.name) > 0:
                break
            time.sleep(0.02)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        with open(self.file.name) as fh:
            rows = [r.strip().split(", ") for r in fh if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def time_steps(lb, ctx, torch, steps, warmup):
    """Per-launch device times (ms) of `steps` single-step launches after `warmup`."""
    for _ in range(warmup):
        lb.lb_step(ctx, 1)
    lb.lb_sync(ctx)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for k in range(steps):
        lb.lb_step(ctx, 1)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    lb.lb_sync(ctx)
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    return ev[0].elapsed_time(ev[-1]), per


def cpu_oracle_sample(n_box, target_s=10.0, max_steps=20):
    """The FP64 oracle, as it stands, on a periodic n_box^3 box of the same workload
    recipe, for as many steps as fit in about target_s seconds (at least 1)."""
    import oracle
    from paper_1909_08406_gb300 import workloads as wl
    th0 = oracle.theta0()
    sigma = 8.0 * n_box / 512.0 if n_box < 512 else 8.0
    fl = wl.thermoacoustic_pulse(n_box, th0, sigma=max(sigma, 2.0), kmax=min(8, n_box // 4))
    f = oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy())
    tau = NU / th0
    t0 = time.perf_counter()
    f = oracle.step(f, tau, 1)
    one = time.perf_counter() - t0
    steps = max(1, min(max_steps, int(target_s / max(one, 1e-9)) - 1))
    t0 = time.perf_counter()
    f = oracle.step(f, tau, steps)
    el = time.perf_counter() - t0
    nodes = 2 * n_box ** 3
    return {"mlups": nodes * steps / el / 1e6, "cores": oracle.max_threads(), "steps": steps, "seconds": el,
            "nodes": nodes}


def run_batch(lb, wl, torch, steps, count=64):
    """Batched sweep: `count` independent simulations (cubic edges from {32,48,64,96,128},
    tau in [0.51, 1], standing acoustic waves of log-uniform amplitude, seed 4), FP32,
    `steps` steps, timed as one graph-replayed batched launch sequence, one persistent
    cooperative launch, and per-simulation sequential launches."""
    sims = wl.batch_sweep(count=count)
    th0 = lb.lb_theta0()
    b = lb.lb_batch_init([(s.n, s.n, s.n) for s in sims], [s.tau for s in sims], "f32")
    nodes = sum(2 * s.n ** 3 for s in sims)
    out = {"sims": count, "nodes": nodes, "steps": steps, "edges": sorted({s.n for s in sims})}
    try:
        for k, s in enumerate(sims):
            fl = wl.standing_wave(s.n, s.n, s.n, th0, amplitude=s.amplitude, device="cuda")
            lb.lb_set_fields(lb.lb_batch_sim(b, k), fl["rho"], fl["u"], fl["theta"])
        lb.lb_batch_sync(b)
        tx, ry, ms = lb.lb_batch_tune(b, reps=3)
        # tuned per mode: [tx, ry, rows per thread]; ry = 0: linear tiles of tx consecutive
        # nodes (or node pairs)
        out["plan"] = {"graph": list(lb.lb_batch_get_plan(b, lb.LB_BATCH_GRAPH)),
                       "persistent": list(lb.lb_batch_get_plan(b, lb.LB_BATCH_PERSISTENT))}
        stream = torch.cuda.current_stream()
        for name, mode in (("graph", lb.LB_BATCH_GRAPH), ("persistent", lb.LB_BATCH_PERSISTENT),
                           ("sequential", lb.LB_BATCH_SEQUENTIAL)):
            lb.lb_batch_step(b, 2, mode)  # warm-up (and graph capture for the timed length below)
            lb.lb_batch_step(b, steps, mode) if mode == lb.LB_BATCH_GRAPH else None
            lb.lb_batch_sync(b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lb.lb_batch_step(b, steps, mode)
            e1.record(stream)
            torch.cuda.synchronize()
            lb.lb_batch_sync(b)
            ms = e0.elapsed_time(e1)
            out[name] = {"mlups": nodes * steps / (ms * 1e-3) / 1e6, "seconds": ms * 1e-3,
                         "achieved_gbs": nodes * 328 * steps / (ms * 1e-3) / 1e9}
        out["speedup_graph_vs_sequential"] = out["graph"]["mlups"] / out["sequential"]["mlups"]
        out["speedup_persistent_vs_sequential"] = out["persistent"]["mlups"] / out["sequential"]["mlups"]
    finally:
        lb.lb_batch_destroy(b)
    return out


def conv_timings(torch, sg, layers, batches, impls, ops, reps, warmup):
    """CUDA-event time per launch of the surrogate's convolutions on random BF16 activations of
    batch x 64^3 x cin voxels: the forward convolution with its fused GELU (+ residual when
    cin == cout) epilogue, and the weight + bias gradient (dz of cout channels).  Rate:
    2 * voxels * 27 * cin * cout flops per launch."""
    names = {"tcgen05": sg.CONV_TCGEN05, "mma_sync": sg.CONV_MMA_SYNC}
    out = {}
    for name in impls:
        prev = sg.set_conv_impl(names[name])
        try:
            for cin, cout in layers:
                for batch in batches:
                    shape = (batch, 64, 64, 64)
                    g = torch.Generator(device="cuda").manual_seed(cin * 100 + cout)
                    x = torch.randn(shape + (cin,), device="cuda", generator=g).to(torch.bfloat16)
                    flops = 2.0 * batch * 64 ** 3 * 27 * cin * cout
                    for op in ops:
                        if op == "fwd":
                            w = (torch.randn((cout, 27, cin), device="cuda", generator=g) / math.sqrt(27 * cin)
                                 ).to(torch.bfloat16)
                            b = torch.zeros(cout, device="cuda")
                            y = torch.empty(shape + (cout,), device="cuda", dtype=torch.bfloat16)
                            run = lambda: sg.conv3d_fwd(x, w, b, act=sg.ACT_GELU, res_in=(cin == cout), y=y)  # noqa
                        else:
                            dz = torch.randn(shape + (cout,), device="cuda", generator=g).to(torch.bfloat16)
                            dw = torch.empty((cout, 27, cin), device="cuda")
                            db = torch.empty(cout, device="cuda")
                            scr = sg.wgrad_scratch(x, cin, cout)
                            run = lambda: sg.conv3d_wgrad(x, dz, dw, db, scr)  # noqa
                        for _ in range(warmup):
                            run()
                        torch.cuda.synchronize()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record()
                        for _ in range(reps):
                            run()
                        e1.record()
                        e1.synchronize()
                        ms = e0.elapsed_time(e1) / reps
                        out[f"{op} {name} {cin}->{cout} b{batch}"] = {
                            "us": round(ms * 1e3, 2), "tflops": round(flops / (ms * 1e-3) / 1e12, 1)}
            sg.status()
        finally:
            sg.set_conv_impl(prev)
    return out


def bf16_peak():
    """Measured dense BF16 peak (TFLOP/s, burst) and where it came from."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def workload_config(args, world):
    """The `config` of both arms' JSON lines: the workload the main arm times."""
    n = args.n
    nodes = 2 * n ** 3
    sr = getattr(args, "stochastic", False) and args.precision == "bf16"
    cfg = {"workload": f"thermoacoustic pulse, {n}^3 periodic bcc grid ({nodes} nodes), nu = {NU}, "
                       f"{args.precision} storage" + (", stochastic rounding" if sr else ""),
           "grid": n, "nodes": nodes, "precision": args.precision,
           "l2": "inputs larger than L2 (population buffers of "
                 f"{nodes * 41 * BYTES[args.precision] / 1e9:.1f} GB each)",
           "parallelism": f"replicas x{world}"}
    if sr:
        cfg["rounding"] = "stochastic"
    return cfg


def run_reference(args, rank, world):
    if rank != 0:
        return
    box = 64
    import oracle
    from paper_1909_08406_gb300 import workloads as wl
    th0 = oracle.theta0()
    fl = wl.thermoacoustic_pulse(box, th0, sigma=2.0, kmax=8)
    f = oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy())
    tau = NU / th0
    f = oracle.step(f, tau, max(args.warmup, 0))
    steps = max(1, args.steps)
    t0 = time.perf_counter()
    f = oracle.step(f, tau, steps)
    el = time.perf_counter() - t0
    nodes = 2 * box ** 3
    v = nodes * steps / el / 1e6
    sample = (f"bounded sample of the workload: a {box}^3 periodic box of the thermoacoustic recipe (pulse "
              f"sigma 2 cells), FP64 oracle, {steps} steps after {args.warmup} warm-up steps, MLUPS of that box")
    line = {"impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"thermoacoustic pulse, {box}^3 periodic bcc grid ({nodes} nodes), pulse sigma "
                                   f"2 cells, nu = {NU}, FP64 oracle on the host cores (a bounded sample of the "
                                   f"{args.n}^3 workload of the main line)",
                       "grid": box, "nodes": nodes, "precision": "f64",
                       "parallelism": f"host threads x{oracle.max_threads()}"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if args.conv:
        from paper_1909_08406_gb300 import sg
        impls = ["tcgen05", "mma_sync"] if args.conv_impl == "both" else [args.conv_impl]
        layers = [tuple(int(v) for v in L.split("x")) for L in args.conv_layers.split(",")]
        batches = [int(b) for b in args.conv_batch.split(",")]
        res = conv_timings(torch, sg, layers, batches, impls, args.conv_ops.split(","), args.conv_reps,
                           args.conv_warmup)
        if rank == 0:
            print(json.dumps({"conv": res, "bf16_peak_tflops": bf16_peak()[0]}), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1909_08406_gb300 import lb
    from paper_1909_08406_gb300 import workloads as wl

    from paper_1909_08406_gb300 import decomp

    def barrier():
        decomp.barrier()

    def max_over_ranks(x):
        return decomp.max_over_ranks(x, device="cuda")

    n = args.n
    nodes = 2 * n ** 3
    th0 = lb.lb_theta0()
    tau = NU / th0

    # CPU baseline first (rank 0, N = 1 only): plain C oracle, no GPU involved.
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        box = 96 if n >= 96 else n
        cpu = cpu_oracle_sample(box)

    fields = wl.thermoacoustic_pulse(n, th0, device="cuda")
    precs = [args.precision] + ([] if args.no_secondary else [p for p in ("f32", "bf16", "f16", "f64")
                                                              if p != args.precision])
    results = {}
    by_kernel = {}
    clocks = None

    def timed_run(prec, kernel, steps, warm, sample_clocks, walls=False, nonideal=False):
        ctx = lb.lb_init((n, n, n), tau, prec)
        try:
            lb.lb_set_fields(ctx, fields["rho"], fields["u"], fields["theta"])
            if walls:  # a Couette channel: still wall below, moving wall above, 2e-4 theta0 apart
                lb.lb_set_walls(ctx, (0.0, 0.0, th0 * (1 - 1e-4)), (0.02, 0.0, th0 * (1 + 1e-4)))
            if nonideal:  # van der Waals at theta0 / theta_c = 1.1 (one phase), rho_c = 1
                theta_c = th0 / 1.1
                lb.lb_set_nonideal(ctx, 27.0 / 3.0 * theta_c / 8.0, 1.0 / 3.0, 0.05, 0.5)
            elif args.stochastic and prec == "bf16" and not walls:
                lb.lb_set_stochastic_rounding(ctx, 20191909)
            if kernel is None:
                lb.lb_tune(ctx, reps=3)
            else:
                lb.lb_set_step_kernel(ctx, kernel)
            used = lb.lb_step_variant(ctx)
            lb.lb_sync(ctx)
            barrier()
            torch.cuda.synchronize()
            sampler = ClockSampler(local) if sample_clocks else None
            if sampler:
                sampler.__enter__()
            total_ms, per = time_steps(lb, ctx, torch, steps, warm)
            if sampler:
                sampler.__exit__(None, None, None)
            barrier()
            total_ms = max_over_ranks(total_ms)
        finally:
            lb.lb_destroy(ctx)
        torch.cuda.empty_cache()
        alg = nodes * 41 * 2 * BYTES[prec]
        avg_ms = sum(per) / len(per)
        return {"mlups": world * nodes * steps / (total_ms * 1e-3) / 1e6, "ms_per_step": total_ms / steps,
                "kernel_ms": avg_ms, "achieved_gbs": alg / (avg_ms * 1e-3) / 1e9, "alg_bytes_per_launch": alg,
                "steps": steps, "warmup": warm, "kernel_id": used, "kernel": lb.KERNEL_NAMES[used]}, sampler

    # headline precision: every step kernel that applies to this grid, a short run each; the
    # fastest is then timed in full (the same choice lb_tune makes)
    head = args.precision
    kernels = [args.kernel] if args.kernel is not None else [lb.LB_KERNEL_DIRECT1, lb.LB_KERNEL_DIRECT2,
                                                            lb.LB_KERNEL_DIRECT2R, lb.LB_KERNEL_STAGED,
                                                            lb.LB_KERNEL_WARPSPEC, lb.LB_KERNEL_DIRECT2X,
                                                            lb.LB_KERNEL_DIRECT2XL]
    probe_ctx = lb.lb_init((n, n, n), tau, head)
    applicable = []
    for k in kernels:
        lb.lb_set_step_kernel(probe_ctx, k)
        if lb.lb_step_variant(probe_ctx) == k and k not in applicable:
            applicable.append(k)
    lb.lb_destroy(probe_ctx)
    torch.cuda.empty_cache()
    if len(applicable) > 1:
        for k in applicable:
            r, _ = timed_run(head, k, max(5, args.steps // 3), 2, False)
            by_kernel[lb.KERNEL_NAMES[k]] = {"mlups": r["mlups"], "achieved_gbs": r["achieved_gbs"],
                                             "ms_per_step": r["ms_per_step"]}
        best = max(applicable, key=lambda k: by_kernel[lb.KERNEL_NAMES[k]]["mlups"])
    else:
        best = applicable[0]
    results[head], sampler = timed_run(head, best, args.steps, args.warmup, True)
    clocks = sampler.summary()
    walls = None
    if not args.no_walls:
        r, _ = timed_run(head, best, max(5, args.steps // 5), 3, False, walls=True)
        walls = {"mlups": r["mlups"], "ms_per_step": r["ms_per_step"], "steps": r["steps"],
                 "vs_periodic": r["mlups"] / results[head]["mlups"],
                 "note": "kinetic walls normal to z (Couette channel), same grid, precision and step kernel; "
                         "adds the wall sums and the update of the 2 outermost cell layers at each wall"}
    nonideal = None
    if not args.no_nonideal:
        r, _ = timed_run(head, best, max(5, args.steps // 10), 3, False, nonideal=True)
        per_node = 3 * 41 * BYTES[head] + NONIDEAL_FIELD_VALUES * (8 if head == "f64" else 4)
        ni_gbs = nodes * per_node / (r["kernel_ms"] * 1e-3) / 1e9
        hbm, hbm_kind = measured_peaks()
        nonideal = {"mlups": r["mlups"], "ms_per_step": r["ms_per_step"], "steps": r["steps"],
                    "vs_energy_conserving": r["mlups"] / results[head]["mlups"],
                    "roofline": {"bound": "hbm", "alg_bytes_per_node": per_node, "achieved": ni_gbs, "peak": hbm,
                                 "unit": "GB/s", "frac": ni_gbs / hbm, "peak_kind": hbm_kind},
                    "kernels_per_step": 4,
                    "note": "isothermal van der Waals fluid (theta/theta_c = 1.1, kappa 0.05) on the same fields, "
                            "grid and storage: density, stencil-field and force passes in the storage's compute "
                            "type, then the forced step; all four on x pairs (the density pass and the step with "
                            "16-bit storage, the stencil passes with FP32 fields)"}
    if not args.no_secondary:
        for prec in precs[1:]:
            steps = max(3, args.steps // 10) if prec == "f64" else max(5, args.steps // 2)
            results[prec], _ = timed_run(prec, None, steps, 3, False)

    # the error at which each timed precision runs: the same fields and steps against the GPU FP64
    # mode (itself matched to the FP64 oracle to 1e-12), with the kernel that was timed
    accuracy = None
    if not args.no_accuracy and rank == 0 and world == 1:
        from paper_1909_08406_gb300 import accuracy_report
        precs_acc = [p for p in results if p != "f64"]
        acc = accuracy_report.compare(n, args.steps, precs_acc, fields,
                                      {p: results[p]["kernel_id"] for p in precs_acc})
        accuracy = {"vs": "GPU FP64 mode, same fields and steps", "steps": args.steps,
                    **{p: {k: acc[p][k] for k in ("rel_l2_rho_fluct", "rel_l2_theta_fluct", "max_abs_rho_err",
                                                  "mass_drift", "energy_drift")} for p in precs_acc}}

    batch = None
    if not args.no_batch and world == 1:
        del fields
        torch.cuda.empty_cache()
        batch = run_batch(lb, wl, torch, args.batch_steps, count=args.batch_sims)
        fields = wl.thermoacoustic_pulse(n, th0, device="cuda")

    # end to end through the C ABI with host buffers: upload fields, K steps, read back all fields
    e2e = None
    if not args.no_e2e:
        prec = args.precision
        host = {k: torch.empty(v.shape, dtype=torch.float64, pin_memory=True) for k, v in fields.items()}
        for k in host:
            host[k].copy_(fields[k])
        del fields
        torch.cuda.empty_cache()
        ctx = lb.lb_init((n, n, n), tau, prec)
        try:
            lb.lb_set_fields(ctx, host["rho"], host["u"], host["theta"])
            lb.lb_step(ctx, 2)
            lb.lb_sync(ctx)
            barrier()
            t0 = time.perf_counter()
            lb.lb_set_fields(ctx, host["rho"], host["u"], host["theta"])
            lb.lb_step(ctx, args.steps)
            lb.lb_get_moments(ctx, host["rho"], host["u"], host["theta"])
            lb.lb_sync(ctx)
            el = max_over_ranks(time.perf_counter() - t0)
        finally:
            lb.lb_destroy(ctx)
        io = 5 * nodes * 8
        e2e = {"value": world * nodes * args.steps / el / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": io / args.steps, "d2h_bytes_per_step": io / args.steps,
               "seconds": el, "note": "lb_set_fields from pinned host (rho,u,theta f64, read by the "
                                      "kernel over the host link), K x lb_step, lb_get_moments to pinned "
                                      "host"}

    surrogate = None
    if not args.no_surrogate and rank == 0:
        from paper_1909_08406_gb300 import sg
        pk, pk_kind = bf16_peak()
        ct = conv_timings(torch, sg, [(32, 32)], [4], ["tcgen05"], ["fwd", "wgrad"], 10, 3)
        surrogate = {"layer": "32->32, batch 4 x 64^3, BF16 in, FP32 accumulate, tcgen05",
                     "peak_tflops": pk, "peak_kind": pk_kind,
                     **{op: {**ct[f"{op} tcgen05 32->32 b4"], "frac": ct[f"{op} tcgen05 32->32 b4"]["tflops"] / pk}
                        for op in ("fwd", "wgrad")}}

    if rank != 0:
        return
    r = results[args.precision]
    peak, peak_kind = measured_peaks()
    traffic = ncu_traffic(args.precision + ("sr" if args.stochastic and args.precision == "bf16" else ""),
                          r["kernel_id"], n)
    line = {
        "metric": "MLUPS", "value": r["mlups"], "unit": "MLUPS", "n_gpus": world, "steps": r["steps"],
        "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_NAME[args.precision], "data": "synthetic",
        "config": workload_config(args, world),
        "roofline": {"bound": "hbm", "achieved": r["achieved_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": r["achieved_gbs"] / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": r["kernel"], "alg_bytes_per_launch": r["alg_bytes_per_launch"]},
        # FP64 arithmetic bounds the FP64 mode (its pipe is 85% busy, DRAM 6%), HBM the others
        "by_precision": {p: {"mlups": v["mlups"], "achieved_gbs": v["achieved_gbs"],
                             "frac_of_hbm": v["achieved_gbs"] / peak, "ms_per_step": v["ms_per_step"],
                             "steps": v["steps"], "kernel": v["kernel"],
                             "bound": "fp64" if p == "f64" else "hbm"} for p, v in results.items()},
        "by_kernel": by_kernel,
        "accuracy": accuracy,
        "walls": walls,
        "nonideal": nonideal,
        "batch": batch,
        "surrogate_conv": surrogate,
        "gpu_launches": r["steps"],
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": None if cpu is None else {
            "value": cpu["mlups"], "unit": "MLUPS", "cores": cpu["cores"], "kind": "oracle",
            "sample": f"FP64 oracle on a {round((cpu['nodes'] / 2) ** (1 / 3))}^3 periodic box of the same "
                      f"thermoacoustic recipe, {cpu['steps']} steps ({cpu['seconds']:.1f} s)"},
        "kernel_hash": kernel_hash(),
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
