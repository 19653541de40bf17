"""Run one stage of the ESMP2 hot path repeatedly on a seeded synthetic instance.

Meant as the target command of a profiler capture (one kernel family, a few launches, a
few GB on the device):

    python -m paper_2003_12923_gb300.profile_stage --No 10 --Nv 400 --stage virt-bf16 --reps 3

Stages:
    virt-bf16     bf16 x bf16 -> fp32 virtual-index contraction (tcgen05), all slices
    virt-fp64tc   float64-exact virtual-index contraction from digit products (tcgen05)
    virt-fp64     the same with float64 GEMMs
    sigma-fp64    float64 sigma build
    sigma-fp64tc  float64 sigma build with the tensor-core virtual-index terms
    sigma-mixed   sigma with bf16 virtual-index terms, float64 elsewhere
    sigma-inner   the inner (float32 vector) sigma of the mixed solve, per-stage timed
    solve-mixed   a mixed-precision solve to --tol (create excluded)
  (--inner bf16 | tf32 | reduced picks the inner sigma of the last two)
"""
from __future__ import annotations

import argparse
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--No", type=int, default=10)
    ap.add_argument("--Nv", type=int, default=400)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--sigma-off", type=float, default=1e-3)
    ap.add_argument("--stage", default="virt-bf16",
                    choices=["virt-bf16", "virt-fp64tc", "virt-fp64", "sigma-fp64", "sigma-fp64tc", "sigma-mixed",
                             "sigma-inner", "solve-mixed"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--inner", default="bf16", choices=["bf16", "tf32", "reduced"],
                    help="sigma-inner / solve-mixed: bf16 or tf32 contraction, or the reduced-cost basis")
    args = ap.parse_args(argv)

    import torch
    import synth
    from paper_2003_12923_gb300 import esmp2

    inst = synth.make_instance(args.No, args.Nv, args.seed, sigma_off=args.sigma_off)
    d = {k: torch.from_numpy(inst[k]).cuda() for k in ("F", "ovov", "ooov", "ovvv", "C")}
    h = esmp2.Handle(d["F"], d["ovov"], d["ooov"], d["ovvv"], d["C"])
    x = h.rhs()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    inner = {"bf16": esmp2.MIXED_BF16, "tf32": esmp2.MIXED_TF32, "reduced": esmp2.REDUCED_MIXED}[args.inner]
    if args.stage == "solve-mixed":
        info = h.solve(tol=args.tol, maxit=3000, precision=inner)
        print("solve", info)
    elif args.stage == "sigma-inner":
        ms = h.profile_sigma(x, precision=inner, reps=args.reps)
        print("inner sigma stage ms (to bf16, virtual, -, couplings, total):", [round(float(v), 3) for v in ms[:5]])
    else:
        out = torch.empty_like(x)
        for _ in range(args.reps):
            if args.stage == "virt-bf16":
                h.virtual_contraction(x, esmp2.MIXED_BF16, out=out)
            elif args.stage == "virt-fp64tc":
                h.virtual_contraction(x, esmp2.FP64_TC, out=out)
            elif args.stage == "virt-fp64":
                h.virtual_contraction(x, esmp2.FP64, out=out)
            elif args.stage == "sigma-fp64":
                h.sigma(x, esmp2.FP64, out=out)
            elif args.stage == "sigma-fp64tc":
                h.sigma(x, esmp2.FP64_TC, out=out)
            else:
                h.sigma(x, esmp2.MIXED_BF16, out=out)
    torch.cuda.synchronize()
    print(f"stage {args.stage} No={args.No} Nv={args.Nv} reps={args.reps}: {time.perf_counter() - t0:.3f} s")
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
