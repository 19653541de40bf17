#!/usr/bin/env python3
"""Writes the stored oracle values the GPU tests compare against (calls only oracle/ and the
seeded input generator synth/; nothing here reads the CUDA path).

Each task is one file tests/golden/o2_<task>.json:

  e2_4_130, e2_3_300, e2_c2   O2 plain-CG solve (Sec. III.A: CG) of the first-order equation of
                              one synthetic instance and its energy parts: E2_D + E2_L by the
                              Hylleraas functional 2 b.x + x.Ax (error quadratic in the
                              residual), E2_S by the direct S-space sum (Sec. II.D).
  grad_c5                     the same solve at No=16 Nv=160 and the derivatives of E2 along
                              sampled steps of F and of (ia|jb), from the first-order equation
                              at that solution (oracle.grad.analytic_F / analytic_ovov).

These runs take minutes to hours of host time (O2 is plain loops), which is why their results
are stored rather than recomputed inside the GPU tests.

usage: python tests/golden/make_o2_reference.py TASK [TASK ...]
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import grad, o2, top  # noqa: E402

# task: (No, Nv, seed, sigma_off, tol)
E2_TASKS = {
    "e2_4_130": (4, 130, 21, 1e-3, 1e-9),
    "e2_3_300": (3, 300, 22, 1e-3, 1e-9),
    "e2_c2": (20, 200, 1, 1e-3, 1e-7),
}
# the derivatives are first order in the solution's error (2 x.db + x.dA x at an approximate x),
# so the C5 solve is taken to 1e-11, well below the 1e-6 relative accuracy they are compared at
C5 = (16, 160, 5, 1e-3, 1e-11)
GRAD_F = [(0, 0), (3, 3), (20, 20), (0, 1), (2, 9), (0, 16), (5, 40), (17, 30), (16, 170), (100, 101)]
GRAD_OVOV = [(0, 0, 0, 0), (0, 0, 1, 1), (2, 5, 7, 9), (1, 0, 1, 0), (3, 17, 0, 2), (15, 159, 14, 158),
             (4, 40, 9, 3), (6, 100, 6, 11), (0, 7, 12, 150), (11, 60, 2, 60), (8, 1, 8, 1), (13, 31, 5, 77)]


def _cpu():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _meta(task, No, Nv, seed, sigma_off, tol, t0, res):
    return {"task": task, "command": f"python tests/golden/make_o2_reference.py {task}",
            "instance": {"No": No, "Nv": Nv, "seed": seed, "sigma_off": sigma_off,
                         "generator": "synth.make_instance"},
            "tol": tol, "cg_iterations": int(res["iters"]),
            "final_rel_residual": float(res["hist"][-1]) if res["hist"] else None,
            "seconds": time.time() - t0, "threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
            "host_cpu": _cpu()}


def run_e2(task):
    No, Nv, seed, so, tol = E2_TASKS[task]
    t0 = time.time()
    prep = top.prepare(synth.make_instance(No, Nv, seed, sigma_off=so))
    res = o2.solve(prep, tol=tol, maxit=1000)
    out = _meta(task, No, Nv, seed, so, tol, t0, res)
    out.update({k: float(res[k]) for k in ("E2", "E2_D", "E2_L", "E2_S")})
    out["n_S"] = int(res["n_S"])
    return out


def run_grad_c5(task):
    No, Nv, seed, so, tol = C5
    t0 = time.time()
    inst = synth.make_instance(No, Nv, seed, sigma_off=so)
    prep = top.prepare(inst)
    res = o2.solve(prep, tol=tol, maxit=3000)
    out = _meta(task, No, Nv, seed, so, tol, t0, res)
    out.update({k: float(res[k]) for k in ("E2", "E2_D", "E2_L", "E2_S")})
    x = res["x"]
    out["convention"] = ("derivative of E2 along the step that moves F_pq and F_qp together (once if p == q), "
                         "and (ia|jb) with (jb|ia) (once if they coincide); orbital indices of the ESMF basis, "
                         "F over No+Nv orbitals, ovov as [i][a][j][b] with a, b virtual indices")
    out["dF_step"] = [[p, q, grad.analytic_F(inst, x, p, q, prep=prep)] for (p, q) in GRAD_F]
    out["dOVOV_step"] = [[i, a, j, b, grad.analytic_ovov(inst, x, i, a, j, b, prep=prep)]
                         for (i, a, j, b) in GRAD_OVOV]
    out["seconds"] = time.time() - t0
    return out


def main(argv):
    tasks = argv or sorted(E2_TASKS) + ["grad_c5"]
    for task in tasks:
        if task in E2_TASKS:
            out = run_e2(task)
        elif task == "grad_c5":
            out = run_grad_c5(task)
        else:
            raise SystemExit(f"unknown task {task}")
        path = os.path.join(HERE, f"o2_{task}.json")
        with open(path + ".tmp", "w") as f:
            json.dump(out, f, indent=1)
        os.replace(path + ".tmp", path)
        print(f"{task}: wrote {path} ({out['seconds']:.0f} s)", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
