"""Run one EXPRK3DS_REAL step of a FitzHugh-Nagumo or Schnakenberg problem between
cudaProfilerStart and cudaProfilerStop, after warm-up steps, for profilers that
capture only that range (ncu --profile-from-start off).

  python -m paper_2310_07551_gb300.profile_step --model fhn --dims 256 256 128 \\
      --precision f16x10 --warmup 2

The problem is the workloads' recipe (the FD Neumann Laplacian on [-1, 1]^d for
FitzHugh-Nagumo, [0, 1]^d for Schnakenberg, white-noise or near-equilibrium
initial data) at the given grid.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--model", default="fhn", choices=["fhn", "schnakenberg"])
    ap.add_argument("--dims", type=int, nargs="+", default=[256, 256, 128])
    ap.add_argument("--precision", default="f16x10")
    ap.add_argument("--warmup", type=int, default=2)
    args = ap.parse_args()

    import torch

    from paper_2310_07551_gb300 import configs, ds, inputs

    dims = tuple(args.dims)
    if args.model == "fhn":
        lo, hi, delta, tau, p = -1.0, 1.0, (1.0, 42.1887), 1e-3, configs.FHN
    else:
        lo, hi, delta, tau, p = 0.0, 1.0, (1.0, 10.0), 1e-4, configs.SCHNAK
    Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
    As = [[dl * D for D in Ds] for dl in delta]
    ps = ds.PhiSet(dims, As, tau)
    plan = ds.Plan(ps, args.model, p, args.precision)
    U = torch.from_numpy(inputs.initial_state(args.model, dims, seed=1)).cuda()
    plan.integrate(U, args.warmup)
    plan.sync()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    plan.integrate(U, 1)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    plan.sync(U, check_state=True)
    print("ok", dims, args.precision)


if __name__ == "__main__":
    main()
