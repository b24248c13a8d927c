"""Throughput benchmark of the EXPRK3DS_REAL step on one GB300 (or N replicas).

Default workload: 3D FitzHugh-Nagumo on a 256^3 grid (tau = 1e-3), split-BF16
tensor-core mode products with the FP64 state.  A "step" is one time step of
the scheme (Kronecker-sum action + reaction, the three Tucker-operator groups
and the stage updates); the phi-matrix setup runs once before timing and is
reported separately.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload fhn3d_256] [--precision bf16x6|f64]

Under torchrun each rank runs an independent replica on its own GPU (the
split step has no data-path exchange), timing is the max over ranks and the
value is the whole-job rate.  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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

# DRAM traffic per launch of the tensor-core mode-product kernel, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the hash of
# the kernel source it was measured on; a changed kernel reports null.
NCU_TRAFFIC = {}


def _source_hash() -> str:
    with open(os.path.join(ROOT, "paper_2310_07551_gb300", "csrc", "tc.cu"), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


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
            self.lines.append(line.strip())

    def stop(self):
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
        for ln in self.lines:
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


def _problem(w):
    from paper_2310_07551_gb300 import inputs
    Ds = [inputs.fd_neumann(n, w.lo, w.hi) for n in w.dims]
    return [[dl * D for D in Ds] for dl in w.delta]


def _tucker_ops_per_step(d: int) -> int:
    # both components: 10 (d = 2) or 15 (d = 3) Tucker operators each
    return 2 * (10 if d == 2 else 15)


def oracle_sample(w, reps: int = 1):
    """Time the FP64 oracle on a bounded sample of the workload: one mu-mode
    product per direction on the full tensor (one Tucker operator's worth of
    contraction work), scaled by the Tucker operators of a step.  Returns
    (grid-point*steps/s, seconds of CPU work, description)."""
    import numpy as np

    from oracle import oracle as O
    from paper_2310_07551_gb300 import inputs
    X = inputs.initial_state(w.model, w.dims, seed=w.seed)[0]
    A = _problem(w)[1]
    P = [O.phi(w.tau * Am, 1)[1] for Am in A]
    t0 = time.perf_counter()
    for _ in range(reps):
        for mu in range(1, w.d + 1):
            X = O.mode_product(X, mu, P[mu - 1])
    t = (time.perf_counter() - t0) / reps
    t_step = t * _tucker_ops_per_step(w.d)
    del np
    return w.npoints / t_step, t * reps, (
        f"{reps} x one mu-mode product per direction on the full {'x'.join(map(str, w.dims))} tensor "
        f"(= one Tucker operator), scaled by the {_tucker_ops_per_step(w.d)} Tucker operators of a step")


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count()
    # warm-up samples
    for _ in range(max(0, args.warmup)):
        oracle_sample(w, 1)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        v, s, desc = oracle_sample(w, 1)
        vals.append(v)
        secs += s
    value = args.steps / sum(1.0 / v for v in vals)   # harmonic mean = total work / total time
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": w.npoints / value * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.dims), "tau": w.tau, "model": w.model,
                   "oracle": "FP64 CPU oracle (plain loops, OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc + f"; {args.steps} samples, {secs:.1f} s of CPU work"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fhn3d_256")
    ap.add_argument("--precision", default="bf16x6", choices=["bf16x6", "f64"])
    ap.add_argument("--err-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2310_07551_gb300 import configs
    w = configs.WORKLOADS[args.workload]

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
    t0 = time.perf_counter()
    ps = ds.PhiSet(w.dims, As, w.tau)
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
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.3)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        plan.integrate(U, 1)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    plan.sync(U, check_state=True)
    t = e0.elapsed_time(e1) / 1e3
    if dist is not None:
        tt = torch.tensor([t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    value = world * w.npoints * args.steps / t
    launches_per_step = plan.kernels_per_step

    # per-kernel device times with CUDA events on the launching stream
    kprof = max(3, min(args.steps, 10))
    plan.profile(True)
    for _ in range(kprof):
        plan.step(U)
    prof = plan.profile_read()
    plan.profile(False)
    plan.sync(U, check_state=True)

    # end to end through the public API with host buffers: H2D of the state,
    # one step, D2H of the new state, every step
    Uh = torch.from_numpy(U0.copy()).pin_memory()
    Uo = torch.empty_like(Uh).pin_memory()
    k_e2e = max(3, min(args.steps, 10))
    plan.integrate(U, 1)
    barrier()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(k_e2e):
        U.copy_(Uh, non_blocking=True)
        plan.integrate(U, 1)
        Uo.copy_(U, non_blocking=True)
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
    tc_ms, tc_n, tc_fl = prof["tc"]
    f64_ms, f64_n, f64_fl = prof["f64"]
    pw_ms, pw_n, _ = prof["pointwise"]
    if args.precision == "bf16x6":
        # tensor-instruction flops: six BF16 products per FP32-class product
        achieved = 6.0 * tc_fl / (tc_ms / 1e3) / 1e12
        peak = peaks["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": NCU_TRAFFIC.get(_source_hash()),
                "kernel": "k_mode_tc (tcgen05 split-BF16 mode product)",
                "peak_source": f"{peak_src} bf16_tflops_sustained",
                "useful_fp32_tflops": tc_fl / (tc_ms / 1e3) / 1e12,
                "kernel_share_of_step": tc_ms / (tc_ms + pw_ms) if tc_ms + pw_ms > 0 else None}
    else:
        achieved = f64_fl / (f64_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s",
                "frac": achieved / 1.25, "traffic": None,
                "kernel": "k_dgemm (FP64 mode product)", "peak_source": "nominal GB300 FP64"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.dims), "tau": w.tau, "model": w.model,
                   "precision": args.precision, "state": "fp64",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2 (FP64 state 268 MB; >10 GB moved per step)"
                   if w.npoints >= 1 << 24 else "L2 not flushed (small workload)",
                   "phi_setup_s": setup_s},
        "rel_err_vs_fp64": {"value": err, "steps": args.err_steps} if err is not None else None,
        "roofline": roof,
        "e2e": {"value": world * w.npoints * k_e2e / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state},
        "gpu_launches": launches_per_step * args.steps,
        "kernel_ms_per_step": {"tensor_core": tc_ms / kprof, "fp64_gemm": f64_ms / kprof,
                               "pointwise": pw_ms / kprof},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, secs, desc = oracle_sample(w, 1)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": desc + f" ({secs:.1f} s of CPU work)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    ps.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
