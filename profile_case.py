"""Run one transform configuration a few times (for profilers) and report the
device status word; exits non-zero if the status is not 0.

    python profile_case.py --log2n 20 --log2k 12 --batch 4096 --reps 4
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--log2n", type=int, default=20)
    ap.add_argument("--log2k", type=int, default=12)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=4)
    ap.add_argument("--prec", default="c64", choices=["c64", "c128"])
    ap.add_argument("--fp64-df", action="store_true", help="complex128 in double-float arithmetic")
    ap.add_argument("--strategy", default="", choices=["", "levels", "queue"],
                    help="multi-level plans: per-level launches or one work-queue launch")
    ap.add_argument("--uneven", type=int, default=0,
                    help="run the uneven workload's recipe with this many instances instead")
    ap.add_argument("--sas", default="", choices=["", "ap", "subset"],
                    help="run Shift-and-Sample on that support kind (N = 2^20, k = 3000) instead")
    args = ap.parse_args()
    if args.uneven:
        return uneven(args)
    if args.sas:
        return sas(args)

    import torch

    import workloads as W
    from paper_2211_15299_gb300 import Plan

    inst, _ = W.workload_shared(M=args.log2n, s=args.log2k, batch=1, coeffs=False)
    plan = Plan(args.log2n, inst.J, args.prec, fp64_df=args.fp64_df)
    if args.strategy:
        plan.set_strategy(args.strategy)
    dt = torch.complex64 if args.prec == "c64" else torch.complex128
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    x = torch.randn((args.batch, inst.k), dtype=dt, device="cuda", generator=g)
    y = torch.empty_like(x)
    for _ in range(args.reps):
        plan.execute_strided(x, y)
    torch.cuda.synchronize()
    st = plan.device_status()
    print(f"profile_case log2n={args.log2n} log2k={args.log2k} batch={args.batch} {args.prec} "
          f"strategy={args.strategy or 'default'} reps={args.reps} device_status={st:#x}", flush=True)
    return 0 if st == 0 else 3


def uneven(args) -> int:
    import torch

    import workloads as W
    from paper_2211_15299_gb300 import Batch, Plan

    insts = W.workload_uneven(count=args.uneven)
    plans = [Plan(i.M, i.J, args.prec) for i in insts]
    b = Batch(plans)
    dt = torch.complex64 if args.prec == "c64" else torch.complex128
    x = torch.randn(b.total, dtype=dt, device="cuda")
    y = torch.empty_like(x)
    for _ in range(args.reps):
        b.execute(x, y)
    torch.cuda.synchronize()
    st = b.device_status()
    n_items, n_ctr, grid = b.stats()
    print(f"profile_case uneven={args.uneven} coeffs={b.total} items={n_items} counters={n_ctr} grid={grid} "
          f"reps={args.reps} device_status={st:#x}", flush=True)
    return 0 if st == 0 else 3


def sas(args) -> int:
    import torch

    import workloads as W
    from paper_2211_15299_gb300 import Sas

    J = W.workload_sas(args.sas)
    p = Sas(20, J, args.prec)
    dt = torch.complex64 if args.prec == "c64" else torch.complex128
    x = torch.randn((args.batch, p.n_samples), dtype=dt, device="cuda")
    w = torch.empty_like(x)
    y = torch.empty((args.batch, p.k), dtype=dt, device="cuda")
    for _ in range(args.reps):
        p.execute(x, y, work=w)
    torch.cuda.synchronize()
    print(f"profile_case sas={args.sas} k={p.k} R={p.R} mu*={p.mu_star} batch={args.batch} reps={args.reps}",
          flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
