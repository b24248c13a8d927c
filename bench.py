"""Throughput benchmark of the EXPRK3DS_REAL step on one GB300 (or N replicas).

Default workload: 3D FitzHugh-Nagumo on a 256^3 grid (tau = 1e-3, 200-step
horizon) in DS_PREC_F16X10: the Tucker group on F with fixed-head FP16
operands on the tensor cores (~35-bit operands), the groups on D2, D3 in
split BF16, the state in FP64; the error against the FP64 GPU path is
measured over the full horizon.  --workload schnak2d_1024 runs the 2D
Schnakenberg 1024^2 case, --workload batch64 the 64-instance batch.  A
"step" is one time step of the scheme (Kronecker-sum action + reaction, the
three Tucker-operator groups and the stage updates); the phi-matrix setup
runs once before timing and is reported separately.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload fhn3d_256|schnak2d_1024|batch64|...]
                  [--precision f16x10|bf16x6|bf16x6c|f32|f64]
                  [--err-steps E]   (default: the workload's horizon; 0 skips)

Under torchrun each rank runs an independent replica on its own GPU (the
split step has no data-path exchange), timing is the max over ranks and the
value is the whole-job rate.  --impl reference times the FP64 CPU oracle's
step on a bounded slab of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point*steps/s"
UNIT = "grid-point*steps/s"

PREC_NOTE = {
    "f16x10": ("Tucker group on F: fixed-head FP16 four-part operands, 10 tensor-core products in four "
               "accumulators by weight class (exact head accumulation); groups on D2, D3: split BF16 "
               "(6 products); stencil and reaction in double-float; state FP64"),
    "f16x13": ("all three Tucker groups: fixed-head FP16 four-part operands, 13 tensor-core products in four "
                "accumulators by weight class; increments kept as double-floats, stage differences and the final "
                "update in double-float; stencil and reaction in double-float; state FP64"),
    "bf16x6": "split BF16 (3 parts, 6 tensor-core products, FP32 accumulation); state FP64",
    "bf16x6c": "split BF16 with the main product in its own accumulator; state FP64",
    "f32": "FP32 CUDA-core mode products; state FP64",
    "f64": "FP64 throughout",
}

# DRAM traffic per launch of the tensor-core mode-product kernel (mean over one
# step's launches), from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by "<hash of the kernel source>:<workload>";
# a changed kernel reports null.
NCU_TRAFFIC = {
    # FitzHugh-Nagumo, DS_PREC_F16X10: mean over one step's nine k_mode_tc
    # launches, captured on the (256, 256, 128) half-size case (868 MB per
    # launch; every tensor term scales with the points) and doubled
    "c8bdec4652f80be5:fhn3d_256:f16x10": 1.736e9,
}


def _source_hash() -> str:
    """Hash of the tensor-core kernel's code: tc.cu up to its pointwise
    section (PTX wrappers, descriptors, k_mode_tc), comments and white space
    left out, so that measured counters stay attached to unchanged code."""
    with open(os.path.join(ROOT, "paper_2310_07551_gb300", "csrc", "tc.cu"), "r") as fh:
        src = fh.read()
    cut = src.find("// Pointwise kernels of the split-BF16 step.")
    src = src[:cut] if cut > 0 else src
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = " ".join(src.split())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0: float | None = None, t1: float | None = None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if t0 is not None:
            inside = [x for x in lines if t0 - 0.05 <= x[0] <= t1 + 0.15]
            lines = inside if inside else lines[-2:]
        for _, ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_rate(t_local: float, points_per_rank: int, steps: int, dist=None, device=None):
    """Whole-job rate of N independent replicas: every rank times its own K
    steps; the job time is the max over ranks, the work the sum over ranks.
    Returns (value, t_max)."""
    import torch
    world = 1
    t = t_local
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        tt = torch.tensor([t_local], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return world * points_per_rank * steps / t, t


def partition_instances(sizes, world: int):
    """Split independent problems over `world` ranks with no exchange: largest
    first, each to the rank with the least work so far (ties: lowest rank).
    Returns one sorted index list per rank."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def job_rate_sum(t_local: float, work_local: float, dist=None, device=None):
    """Whole-job rate of ranks with unequal shares of independent problems:
    the job time is the max over ranks, the work the sum over ranks.
    Returns (value, t_max, work_total)."""
    import torch
    t, work = t_local, work_local
    if dist is not None and dist.is_initialized():
        tt = torch.tensor([t_local], dtype=torch.float64, device=device)
        ww = torch.tensor([work_local], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dist.all_reduce(ww, op=dist.ReduceOp.SUM)
        t, work = float(tt.item()), float(ww.item())
    return work / t, t, work


def _problem(w):
    from paper_2310_07551_gb300 import inputs
    Ds = [inputs.fd_neumann(n, w.lo, w.hi) for n in w.dims]
    return [[dl * D for D in Ds] for dl in w.delta]


def _tucker_ops_per_step(d: int) -> int:
    # both components: 10 (d = 2) or 15 (d = 3) Tucker operators each
    return 2 * (10 if d == 2 else 15)


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for key in ("Model name", "Model", "Vendor ID"):
            for ln in out.splitlines():
                if ln.split(":")[0].strip() == key and ln.split(":", 1)[1].strip() not in ("", "-"):
                    return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(w, thick: int, steps: int = 1):
    """Time the FP64 oracle's EXPRK3DS step (Algorithm 1/2: Kronecker-sum
    action, reaction, the three Tucker groups, the stage sums) on a slab of
    the workload: the full grid with its last direction cut to `thick`
    points, same model, tau and initial-data recipe.  The oracle's work per
    grid point is proportional to the summed mode sizes (each Tucker
    operator costs 2 N sum_mu n_mu), so the full grid's rate is the slab's
    times sum(n_slab) / sum(n_full).  Returns (full-grid estimate in
    grid-point*steps/s, slab rate, seconds of CPU work, description)."""
    from oracle import oracle as O
    from paper_2310_07551_gb300 import inputs
    dims = tuple(w.dims[:-1]) + (min(thick, w.dims[-1]),)
    Ds = [inputs.fd_neumann(n, w.lo, w.hi) for n in dims]
    As = [[dl * D for D in Ds] for dl in w.delta]
    P = O.phi_set(dims, As, w.tau)
    U = inputs.initial_state(w.model, dims, seed=w.seed)
    npts = 1
    for n in dims:
        npts *= n
    t0 = time.perf_counter()
    O.step(dims, As, P, w.model, w.params, w.tau, U, steps)
    t = time.perf_counter() - t0
    slab_rate = npts * steps / t
    est = slab_rate * sum(dims) / sum(w.dims)
    desc = (f"{steps} oracle step(s) on the {'x'.join(map(str, dims))} slab of the "
            f"{'x'.join(map(str, w.dims))} workload ({t:.1f} s); full-grid rate = slab rate x "
            f"sum(n_slab)/sum(n_full) = {sum(dims)}/{sum(w.dims)}")
    return est, slab_rate, t, desc


def _slab(w) -> int:
    """Last-direction thickness of the CPU sample: about a quarter of the
    3D grid, about an eighth of the 2D one (~10-20 s of oracle work on a
    16-core host)."""
    return max(8, w.dims[-1] // (4 if len(w.dims) == 3 else 8))


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    cores = O.set_threads(0)
    # each step: one oracle step on a slab small enough that the whole
    # --steps K --warmup W run ends within a few minutes
    thick = max(4, min(_slab(w), w.dims[-1] * 16 // max(1, 4 * (args.steps + args.warmup))))
    for _ in range(max(0, args.warmup)):
        oracle_sample(w, thick)
    vals, secs, desc = [], 0.0, ""
    for _ in range(args.steps):
        v, _, s_, desc = oracle_sample(w, thick)
        vals.append(v)
        secs += s_
    value = args.steps / sum(1.0 / v for v in vals)   # harmonic mean = total work / total time
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": w.npoints / value * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.dims), "tau": w.tau, "model": w.model,
                   "scheme": "exprk3ds_real", "precision": "f64",
                   "oracle": "FP64 CPU oracle (plain loops, OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu": _cpu_model(),
                         "sample": desc + f"; {args.steps} samples, {secs:.1f} s of CPU work"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world):
    """64 independent Schnakenberg instances with uneven grids, stepped
    together by CUDA graphs of 10 steps (grouped launches over all of a
    rank's instances).  Under torchrun the instances are partitioned over the
    ranks (largest first, to the least-loaded rank; no data-path exchange).
    value = sum over ranks of the instances' grid points x steps / the
    slowest rank's time."""
    import numpy as np
    import torch

    from paper_2310_07551_gb300 import configs, ds, inputs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    every = configs.batch_instances()
    mine = partition_instances([int(np.prod(i.dims)) for i in every], world)[rank]
    insts = [every[k] for k in mine]
    As = []
    for inst in insts:
        Ds = [inputs.fd_neumann(n, 0.0, 1.0) for n in inst.dims]
        As.append([[dl * D for D in Ds] for dl in inst.delta])
    t0 = time.perf_counter()
    batch = ds.Batch([i.dims for i in insts], As, [i.tau for i in insts], "schnakenberg",
                     [i.params for i in insts], args.precision)
    setup_s = time.perf_counter() - t0
    U0 = [inputs.initial_state("schnakenberg", i.dims, seed=7 + k, a=i.params[1], b=i.params[2])
          for k, i in zip(mine, insts)]
    Us = [torch.from_numpy(u.copy()).cuda() for u in U0]
    npts = sum(int(np.prod(i.dims)) for i in insts)
    batch.integrate(Us, args.warmup)
    batch.sync()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.steps <= 0:
        barrier()
        e0.record(stream)
        batch.integrate(Us, 10)
        e1.record(stream)
        barrier()
        per = e0.elapsed_time(e1) / 1e4
        steps = torch.tensor([max(30, int(1.5 / max(per, 1e-6)) // 10 * 10)], device="cuda")
        if dist is not None:
            dist.all_reduce(steps, op=dist.ReduceOp.MIN)
        args.steps = int(steps.item())
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.3)
    barrier()
    t_wall0 = time.time()
    e0.record(stream)
    batch.integrate(Us, args.steps)
    e1.record(stream)
    barrier()
    t_wall1 = time.time()
    clk = clocks.stop(t_wall0, t_wall1)
    batch.sync()
    t_local = e0.elapsed_time(e1) / 1e3
    value, t, work = job_rate_sum(t_local, float(npts) * args.steps, dist, "cuda")
    # the timed graphs' fused-or-separate choices (ms 0: replayed from DS_TUNE_CACHE)
    fusion = order = None
    if args.precision != "f64":
        fusion = {("F", "D2", "D3")[g]: {"fused": f, "ms_fused": a, "ms_separate": b}
                  for g, f, a, b in batch.fusion()}
        order = {("F", "D2", "D3")[g]: {"order": o, "ms_order0": a, "ms_order1": b}
                 for g, o, a, b in batch.tile_order()}
    # useful flops per batch step: 20 Tucker operators (2D: F group 6 per
    # component, D2 and D3 2 each) of 2 N (n_1 + n_2) flops
    useful = sum(40.0 * np.prod(i.dims) * sum(i.dims) for i in insts)
    err = None
    if args.precision != "f64" and args.err_steps != 0:
        m = configs.BATCH_STEPS if args.err_steps < 0 else args.err_steps
        b64 = ds.Batch([i.dims for i in insts], As, [i.tau for i in insts], "schnakenberg",
                       [i.params for i in insts], "f64")
        Ua = [torch.from_numpy(u.copy()).cuda() for u in U0]
        Ub = [torch.from_numpy(u.copy()).cuda() for u in U0]
        batch.integrate(Ua, m)
        b64.integrate(Ub, m)
        batch.sync()
        b64.sync()
        per_inst = [max(float((a[c] - b[c]).abs().max() / b[c].abs().max()) for c in range(2))
                    for a, b in zip(Ua, Ub)]
        b64.close()
        e = torch.tensor([max(per_inst)], dtype=torch.float64, device="cuda")
        if dist is not None:
            dist.all_reduce(e, op=dist.ReduceOp.MAX)
        err = {"value": float(e.item()), "steps": m, "reduction": "max over instances and components",
               "median_over_instances_this_rank": float(np.median(per_inst)),
               "instances_above_1e-6_this_rank": int(sum(x > 1e-6 for x in per_inst))}
    peaks, peak_src = _peaks()
    # tensor instructions per useful product: 6 BF16 (split BF16); in f16x10
    # the F group (6 of 10 operators per component) takes 10 FP16 products
    per_prod = {"bf16x6": 6.0, "bf16x6c": 6.0, "f16x10": 0.6 * 10.0 + 0.4 * 6.0, "f16x13": 13.0}.get(args.precision)
    tensor_tf = per_prod * useful * args.steps / t_local / 1e12 if per_prod else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak" if world == 1 else "strong", "vs_baseline": None, "dtype": args.precision,
        "data": "synthetic",
        "config": {"workload": "batch64", "instances": len(every), "instances_this_rank": len(insts),
                   "grid_points": int(sum(np.prod(i.dims) for i in every)),
                   "parallelism": f"instances partitioned over {world} ranks" if world > 1 else "single",
                   "precision": args.precision, "state": "fp64", "phi_setup_s": setup_s,
                   "arithmetic": PREC_NOTE.get(args.precision, args.precision),
                   "l2": "L2 not flushed (batch state 2.3 GB of FP64 > L2)"},
        "rel_err_vs_fp64": err,
        "roofline": {"bound": "tensor", "achieved": tensor_tf, "peak": peaks["bf16_tflops_sustained"],
                     "unit": "TFLOP/s", "frac": tensor_tf / peaks["bf16_tflops_sustained"] if tensor_tf else None,
                     "traffic": None, "kernel": "whole batch step of rank 0 (all its instances' kernels)",
                     "peak_source": f"{peak_src} bf16_tflops_sustained"},
        "gpu_launches": batch.kernels_per_step * args.steps,
        "clocks": clk,
    }
    if fusion is not None:
        line["config"]["epilogue_fusion"] = fusion
        line["config"]["mode1_tile_order"] = order
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0,
                    help="timed steps (default: enough for about 1.5 s of timed work)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fhn3d_256")
    ap.add_argument("--precision", default=None, choices=["f16x10", "f16x13", "bf16x6", "bf16x6c", "f32", "f64"],
                    help="default: f16x10 (f16x13 for batch64)")
    ap.add_argument("--err-steps", type=int, default=-1)
    ap.add_argument("--scheme", default="exprk3ds_real", choices=["exprk3ds_real", "etd2rkds"],
                    help="etd2rkds: the second-order split ETD2RK (FP64 plans)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.precision is None:
        args.precision = "f16x13" if args.workload == "batch64" else "f16x10"

    from paper_2310_07551_gb300 import configs
    if args.workload == "batch64":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "reference arm covers the single-instance workloads"}))
            return
        run_batch(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    w = configs.WORKLOADS[args.workload]
    if args.err_steps < 0:
        args.err_steps = w.steps

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import numpy as np
    import torch

    from paper_2310_07551_gb300 import ds, inputs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    As = _problem(w)
    if args.scheme != "exprk3ds_real":
        args.precision = "f64"
    t0 = time.perf_counter()
    ps = ds.PhiSet(w.dims, As, w.tau, scheme=args.scheme)
    setup_s = time.perf_counter() - t0
    plan = ds.Plan(ps, w.model, w.params, args.precision)
    U0 = inputs.initial_state(w.model, w.dims, seed=w.seed)
    U = torch.from_numpy(U0).cuda()

    # warm-up (also builds the CUDA graph of the step)
    for _ in range(args.warmup):
        plan.integrate(U, 1)
    plan.sync(U, check_state=True)

    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.steps <= 0:
        barrier()
        e0.record(stream)
        plan.integrate(U, 3)
        e1.record(stream)
        barrier()
        per = e0.elapsed_time(e1) / 3e3
        args.steps = max(30, int(1.5 / max(per, 1e-6)))
    # L2 is flushed between timed steps: a 256 MB buffer (twice L2) is
    # written outside each step's event pair, so no step starts with its
    # inputs resident in L2.
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.3)
    barrier()
    t_wall0 = time.time()
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        plan.integrate(U, 1)
        b.record(stream)
    barrier()
    t_wall1 = time.time()
    clk = clocks.stop(t_wall0, t_wall1)
    plan.sync(U, check_state=True)
    t = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    value, t = job_rate(t, w.npoints, args.steps, dist, "cuda")
    launches_per_step = plan.kernels_per_step

    # per-kernel device times with CUDA events on the launching stream
    kprof = max(3, min(args.steps, 10))
    plan.profile(True)
    for _ in range(kprof):
        flush.zero_()
        plan.step(U)
    prof = plan.profile_read(with_bytes=True)
    plan.profile(False)
    plan.sync(U, check_state=True)

    # end to end through the public API with host buffers: every step copies
    # the state from pinned host memory, steps it and copies the new state
    # back into the same host buffer (the trajectory lives on the host)
    Uh = torch.empty(U.shape, dtype=U.dtype).pin_memory()
    Uh.copy_(U)
    k_e2e = max(3, min(args.steps, 10))
    barrier()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(k_e2e):
        U.copy_(Uh, non_blocking=True)
        plan.integrate(U, 1)
        Uh.copy_(U, non_blocking=True)
    e3.record(stream)
    barrier()
    t_e2e = e2.elapsed_time(e3) / 1e3
    if dist is not None:
        tt = torch.tensor([t_e2e], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
    bytes_state = U.numel() * U.element_size()

    # error of this precision against the FP64 GPU path after a few steps
    err = None
    if args.precision != "f64" and args.err_steps > 0:
        p64 = ds.Plan(ps, w.model, w.params, "f64")
        Ua = torch.from_numpy(U0.copy()).cuda()
        Ub = torch.from_numpy(U0.copy()).cuda()
        plan.integrate(Ua, args.err_steps)
        p64.integrate(Ub, args.err_steps)
        plan.sync()
        p64.sync()
        err = max(float((Ua[c] - Ub[c]).abs().max() / Ub[c].abs().max()) for c in range(2))
        p64.close()

    peaks, peak_src = _peaks()
    tc_ms, tc_n, tc_fl, tc_by = prof["tc"]
    fx_ms, fx_n, fx_fl, fx_by = prof["fx"]
    f64_ms, f64_n, f64_fl, _ = prof["f64"]
    pw_ms, pw_n, _, pw_by = prof["pointwise"]
    prof_ms = tc_ms + fx_ms + f64_ms + pw_ms
    step_ms = t / args.steps * 1e3
    if args.precision == "f32":
        achieved = f64_fl / (f64_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": None, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "kernel": "k_gemm<float> (FP32 CUDA-core mode product)",
                "peak_source": "no measured FP32 peak"}
    elif args.precision in ("bf16x6", "bf16x6c", "f16x10", "f16x13"):
        # The dominant kernel family: every k_mode_tc launch of the step.
        # Tensor-instruction flops: six BF16 products per FP32-class product
        # (split-BF16 launches), ten FP16 products (FX launches; 13 in f16x13).  Their
        # time is their share of the per-launch event profile times the
        # graph-timed step, so it never exceeds ms_per_step.
        fx_prods = 13.0 if args.precision == "f16x13" else 10.0
        tflops_step = (6.0 * tc_fl + fx_prods * fx_fl) / kprof
        share = (tc_ms + fx_ms) / prof_ms if prof_ms > 0 else None
        k_ms = share * step_ms if share else None
        achieved = tflops_step / (k_ms / 1e3) / 1e12 if k_ms else None
        peak = peaks["bf16_tflops_sustained"]
        key = f"{_source_hash()}:{w.name}:{args.precision}"
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None,
                "traffic": NCU_TRAFFIC.get(key),
                "traffic_source": ("ncu capture of this kernel source (mean DRAM read + write per k_mode_tc "
                                   "launch of one step, on the half-size case, scaled to the full grid)"
                                   if key in NCU_TRAFFIC else
                                   "null: no ncu capture of this kernel source on this workload"),
                "alg_bytes_per_launch": (tc_by + fx_by) / (tc_n + fx_n) if tc_n + fx_n else None,
                "launches_per_step": (tc_n + fx_n) // kprof,
                "kernel": ("k_mode_tc (tcgen05 mode products: FX fixed-head FP16 on the F group, "
                           "split BF16 on the D groups)" if fx_n else
                           "k_mode_tc (tcgen05 split-BF16 mode product)"),
                "tensor_flops_per_step": tflops_step,
                "kernel_share_of_step": share,
                "kernel_ms_per_step": k_ms,
                "peak_source": f"{peak_src} bf16_tflops_sustained (FP16 and BF16 share the dense rate)",
                "useful_fp32_class_tflops": (tc_fl + fx_fl) / kprof / (k_ms / 1e3) / 1e12 if k_ms else None,
                "fx_launches": {"launches_per_step": fx_n // kprof,
                                "tensor_tflops": fx_prods * fx_fl / (fx_ms / 1e3) / 1e12,
                                "event_ms_per_step": fx_ms / kprof} if fx_n else None,
                "bf16_launches": {"launches_per_step": tc_n // kprof,
                                  "tensor_tflops": 6.0 * tc_fl / (tc_ms / 1e3) / 1e12,
                                  "event_ms_per_step": tc_ms / kprof} if tc_n else None,
                "pointwise": {"bound": "hbm", "achieved": pw_by / (pw_ms / 1e3) / 1e9 if pw_ms else None,
                              "peak": peaks["hbm_gbs"], "unit": "GB/s",
                              "frac": pw_by / (pw_ms / 1e3) / 1e9 / peaks["hbm_gbs"] if pw_ms else None,
                              "alg_bytes_per_step": pw_by / kprof,
                              "kernels": "k_rhs_tiled (F = K U + g(U)) and the stage kernels the tuner kept "
                                         "separate",
                              "peak_source": f"{peak_src} hbm_gbs"}}
    else:
        achieved = f64_fl / (f64_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s",
                "frac": achieved / 1.25, "traffic": None,
                "kernel": "k_dgemm (FP64 mode product)",
                "peak_source": "nominal GB300 FP64 (1.25 TFLOP/s; not a measured peak)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.dims), "tau": w.tau, "model": w.model,
                   "scheme": args.scheme, "precision": args.precision, "state": "fp64",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": (f"L2 flushed between timed steps (256 MB buffer written outside each step's "
                          f"events); FP64 state {16 * w.npoints / 1e6:.0f} MB"),
                   "arithmetic": PREC_NOTE.get(args.precision, args.precision),
                   "phi_setup_s": setup_s},
        "rel_err_vs_fp64": {"value": err, "steps": args.err_steps} if err is not None else None,
        "roofline": roof,
        "e2e": {"value": world * w.npoints * k_e2e / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state},
        "gpu_launches": launches_per_step * args.steps,
        "kernel_event_ms_per_step": {"tensor_core_bf16": tc_ms / kprof, "tensor_core_fx": fx_ms / kprof,
                                     "fp64_gemm": f64_ms / kprof, "pointwise": pw_ms / kprof},
        "clocks": clk,
    }
    if args.precision in ("bf16x6", "bf16x6c", "f16x10", "f16x13"):
        line["autotuner"] = [{"group": ["F", "D2", "D3"][g], "mode": mu, "split_k": k or None, "stream_k": k == 0,
                              "tiles": t, "tile_n": tn, "tile_order": c.pop("order", 0), "candidates_ms": c}
                             for g, mu, k, t, tn, c in plan.tuning()]
        line["epilogue_fusion"] = [{"group": ["F", "D2", "D3"][g], "fused": fz,
                                    "ms_fused": round(a, 4), "ms_separate": round(b, 4)}
                                   for g, fz, a, b in plan.fusion()]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        threads = O.set_threads(0)
        v, slab_rate, secs, desc = oracle_sample(w, _slab(w))
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": _cpu_model(),
                                "sample": desc, "slab_rate": slab_rate}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    ps.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
