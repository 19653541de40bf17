#!/usr/bin/env python3
"""ESMP2-TOP(1) benchmark: time-to-solution of the first-order equation on one GB300.

One step = the whole hot path on one synthetic instance with its inputs already
resident in HBM: esmp2_create (TOP basis, integral transforms, right-hand side),
esmp2_solve to a true relative residual below --tol, esmp2_energy (E2_D + E2_L by the
Hylleraas functional, E2_S by the direct S-space sum), esmp2_destroy.
value = mean seconds per step (time-to-solution, lower is better).
e2e   = the same through the public API from pinned HOST buffers (host->device copy
        of every input and the device->host read of the energy inside the timed region),
        mean of two steps after one untimed one.
Multi-GPU: instances are independent, so N ranks run N replicas (weak scaling, no
collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ESMP2 time-to-solution (res<1e-8) & sigma TFLOP/s at No=30 Nv=400, mixed vs FP64"
WORKLOADS = {
    # name: (No, Nv, seed, sigma_off, default precision, default tol)
    "c3": (30, 400, 3, 1e-3, "mixed", 1e-8),
    "c3_off1e-4": (30, 400, 2, 1e-4, "mixed", 1e-8),   # conditioning sweep of the off-diagonal Fock
    "c3_off1e-2": (30, 400, 4, 1e-2, "mixed", 1e-8),
    "c2": (20, 200, 1, 1e-3, "fp64", 1e-10),
    "c1": (6, 30, 0, 1e-3, "fp64", 1e-10),
}
# stored oracle energies (written by tests/golden/make_o2_reference.py from oracle/ alone)
GOLDEN = {"c2": "tests/golden/o2_e2_c2.json"}
# DRAM traffic per launch of a kernel, from one ncu capture of the named profile summary;
# valid only while the kernel's source file is byte-identical to the captured one (sha256
# prefix), else reported as null
TRAFFIC = {
    "digits": {"source": "paper_2003_12923_gb300/csrc/tc_bf16.cu", "sha256_16": "a13c20289dbe36a5",
               "profile": "profiles/k_virt_digit_levels_No30_Nv400.md",
               "bytes_per_launch": 24.7e9},   # the eight k_virt launches of one step, averaged
}


def comb2(n):
    return n * (n - 1) // 2


def unique_amplitudes(No, Nv):
    """Unique D+L amplitudes of TOP(1) (S counted once per spin-flip pair)."""
    T = comb2(No) * comb2(Nv)
    S = No * No * Nv * Nv / 2.0
    X = comb2(No - 1) * comb2(Nv - 1)
    Y = comb2(No) * comb2(Nv)
    Z = (No * Nv - 1) * (No - 1) * (Nv - 1)
    return T + S + X + Y + Z


def sigma_flops(No, Nv):
    n = unique_amplitudes(No, Nv)
    return {"alg_total": 4.0 * n * (No + Nv), "alg_virtual": 4.0 * n * Nv,
            "exec_virtual": 20.0 * No * No * Nv ** 3, "exec_total": 20.0 * No * No * Nv * Nv * (No + Nv)}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def measure_fp64_peak(dev):
    """Float64 GEMM rate of this GPU (cuBLAS through torch.matmul, 4096^3, best of 3, CUDA
    events): the denominator for kernels bound by the float64 pipe."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        best = t if best is None else min(best, t)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


def kernel_traffic(kernel):
    ent = TRAFFIC.get(kernel)
    if not ent:
        return None, None
    import hashlib
    path = os.path.join(ROOT, ent["source"])
    try:
        h = hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    except OSError:
        return None, None
    if h != ent["sha256_16"]:
        return None, f"{ent['profile']} (kernel changed since the capture: traffic not reported)"
    return ent, ent["profile"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(No, Nv, seed, sigma_off):
    import synth
    return synth.make_instance(No, Nv, seed, sigma_off=sigma_off)


def _golden(config):
    path = GOLDEN.get(config)
    if not path or not os.path.exists(os.path.join(ROOT, path)):
        return None
    with open(os.path.join(ROOT, path)) as f:
        return json.load(f)


def cpu_baseline(No, Nv, seed, sigma_off, budget_s=12.0, inst=None, tol=1e-8, config=None):
    """The oracle (O2, as it stands) on this host's cores.  Small workloads (at most 2e6
    amplitudes): one whole O2 solve (create + plain CG to tol + energy), timed.  Larger ones:
    O2 sigma on randomly sampled elements of the same workload for about budget_s seconds,
    extrapolated to one full sigma build, times the number of sigma builds of an O2 solve of
    the same recipe (the stored oracle solve of this workload when there is one, else the
    No=6 Nv=30 seed 0 solve run here) -- an extrapolation, reported as such."""
    from oracle import o2, top
    import synth
    t0 = time.time()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    n = 5 * No * No * Nv * Nv
    if n <= 2_000_000:
        full = inst if inst is not None else synth.make_instance(No, Nv, seed, sigma_off=sigma_off)
        ts = time.perf_counter()
        res = o2.solve(top.prepare(full), tol=tol)
        t = time.perf_counter() - ts
        return {"value": t, "unit": "s", "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
                "extrapolated": False, "E2": res["E2"], "cg_iterations": res["iters"],
                "sample": f"whole O2 solve of the No={No} Nv={Nv} seed={seed} instance to {tol} (timed)",
                "wall_s": time.time() - t0}
    if inst is None:
        F = synth.fock(No, Nv, seed, sigma_off)
        C = synth.singles_coefficients(F, No, Nv, seed)
    else:
        F, C = inst["F"], inst["C"]
    U, lam, Wv = top.top_basis(top.normalise_singles(C))
    Ft = top.transform_fock(F, U, Wv)
    prep = {"No": No, "Nv": Nv, "F": Ft, "lam": lam,
            "ovov": np.zeros((No, Nv, No, Nv)), "ooov": np.zeros((No, No, No, Nv)),
            "ovvt": np.zeros((No, Nv, Nv, No))}   # sigma needs no integrals
    o = o2.O2(prep)
    x = np.full(n, 1e-3)
    rng = np.random.default_rng(0)
    done, t_spent, batch = 0, 0.0, 256
    while t_spent < budget_s:
        idx = rng.integers(0, n, batch)
        ts = time.perf_counter()
        o.sigma_at(x, idx)
        t_spent += time.perf_counter() - ts
        done += batch
        batch = min(batch * 2, 65536)
    t_elem = t_spent / done
    g = _golden(config) if config else None
    if g is not None:
        n_sigma = g["cg_iterations"] + 2
        src = f"the stored O2 solve of this workload ({g['task']}: {g['cg_iterations']} CG iterations to {g['tol']})"
    else:
        small = synth.make_instance(6, 30, 0)
        res = o2.solve(top.prepare(small), tol=tol)
        n_sigma = res["iters"] + 2
        src = f"the O2 solve of No=6 Nv=30 seed 0 to {tol} ({res['iters']} CG iterations)"
    t_sigma = t_elem * n
    return {"value": t_sigma * n_sigma, "unit": "s", "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
            "extrapolated": True,
            "sample": (f"O2 sigma at {done} random elements of the No={No} Nv={Nv} block vector "
                       f"({t_spent:.1f} s), extrapolated to {n} elements = {t_sigma:.1f} s per sigma build, "
                       f"x {n_sigma} builds as in {src}"),
            "t_sigma_s": t_sigma, "n_sigma": n_sigma, "wall_s": time.time() - t0}


def lanczos_ritz(esmp2, dins, names, steps=24):
    """The extreme Ritz values of `steps` Lanczos steps on the operator (the library's float64
    sigma, weighted inner product of the layout, started from the right-hand side)."""
    import torch
    h = esmp2.Handle(*(dins[k] for k in names))
    # A is symmetric in the determinant inner product (block weights of the layout)
    wt = torch.tensor(h.weights, dtype=torch.float64, device=dins["F"].device).view(5, 1, 1, 1, 1)
    wnorm = lambda v: float((wt * v * v).sum()) ** 0.5
    b = h.rhs()
    q = b / wnorm(b)
    q_prev = torch.zeros_like(q)
    alphas, betas, beta = [], [], 0.0
    for _ in range(steps):
        w = h.sigma(q, esmp2.FP64)
        a = float((wt * w * q).sum())
        w = w - a * q - beta * q_prev
        alphas.append(a)
        beta = wnorm(w)
        if beta < 1e-14:
            break
        betas.append(beta)
        q_prev, q = q, w / beta
    h.close()
    k = len(alphas)
    T = np.diag(alphas)
    if k > 1:
        T = T + np.diag(betas[:k - 1], 1) + np.diag(betas[:k - 1], -1)
    ritz = np.linalg.eigvalsh(T)
    return {"steps": k, "ritz_min": float(ritz[0]), "ritz_max": float(ritz[-1]),
            "ritz_low": [float(v) for v in ritz[:4]]}


def max_over_ranks(value, dist, device):
    """Largest per-rank float over the process group: the whole job's time."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    if args.config not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm covers the single-instance configs"}))
        return 0
    No, Nv, seed, so, _, tol0 = WORKLOADS[args.config]
    tol = args.tol if args.tol is not None else tol0
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    vals = []
    last = None
    for _ in range(args.warmup + args.steps):
        last = cpu_baseline(No, Nv, seed, so, budget_s=args.ref_budget, tol=tol, config=args.config)
        vals.append(last["value"])
    v = statistics.mean(vals[args.warmup:])
    cb = dict(last)
    cb["value"] = v
    line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{args.config}: No={No} Nv={Nv} seed={seed} sigma_off={so} TOP(1) tol={tol}"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batch(args):
    """Batched workload: 64 uneven instances (No ~ U{8..32}, Nv = round(r No), r ~ U[8,14]),
    solved through esmp2_batch_solve (mixed precision, `--concurrency` workers, one stream
    each) from host inputs, in waves of `--wave` instances (the whole batch's OVVV blocks
    total 230 GB, so inputs are generated wave by wave; generation is not timed).
    value = instances solved per second of batch_solve wall time (host inputs: the value is
    also the end-to-end number).  The float64 comparison times sequential plain-FP64 solves
    (create + solve + energy, host inputs) on every `--fp64-every`-th instance and scales to
    the whole batch by No^2 Nv^3; the oracle baseline is extrapolated the same way from
    sampled O2 sigma elements of four instances."""
    import torch
    import synth
    from paper_2003_12923_gb300 import esmp2
    rank = int(os.environ.get("RANK", "0"))
    shapes = synth.batch_shapes(64)
    prec = {"mixed": esmp2.MIXED_BF16, "tf32": esmp2.MIXED_TF32, "reduced": esmp2.REDUCED_MIXED,
            "auto": esmp2.MIXED_BF16}.get(args.precision, esmp2.MIXED_BF16)
    t_batch, t_seq64, w_seq64, w_all = 0.0, 0.0, 0.0, 0.0
    n_done, worst_res, e2_diffs, iters, launches, h2d = 0, 0.0, [], [], 0, 0
    e2_by_seed = {}
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    except Exception:
        pass
    # warm-up: one small wave (the first two shapes), untimed
    warm = [synth.make_instance(No, Nv, sd, sigma_off=1e-3) for (No, Nv, sd) in shapes[:2]]
    esmp2.batch_solve(warm, tol=args.tol, maxit=args.maxit, precision=prec, concurrency=args.concurrency)
    del warm
    esmp2.kernel_timing(True)
    esmp2.kernel_times()
    clk = ClockSampler(uuid)
    clk.start()
    for w0 in range(0, len(shapes), args.wave):
        wave = shapes[w0:w0 + args.wave]
        insts = [synth.make_instance(No, Nv, sd, sigma_off=1e-3) for (No, Nv, sd) in wave]
        h2d += sum(inst[k].nbytes for inst in insts for k in ("F", "ovov", "ooov", "ovvv", "C"))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, res = esmp2.batch_solve(insts, tol=args.tol, maxit=args.maxit, precision=prec,
                                    concurrency=args.concurrency)
        torch.cuda.synchronize()
        t_batch += time.perf_counter() - t0
        if st != esmp2.OK:
            raise RuntimeError("batch_solve failed: " + "; ".join(r["message"] for r in res if r["status"]))
        for (No, Nv, sd), inst, r in zip(wave, insts, res):
            w = No * No * float(Nv) ** 3
            w_all += w
            n_done += 1
            worst_res = max(worst_res, r["rel_residual"])
            iters.append(r["iterations"])
            launches += int(r["kernel_launches"])
            e2_by_seed[sd] = r["E2"]
        del insts
    clocks = clk.stop()
    ktimes = esmp2.kernel_times()
    esmp2.kernel_timing(False)
    # sequential plain-FP64 solves of every fp64_every-th instance, outside the kernel-timing window
    for idx in range(0, len(shapes), args.fp64_every):
        No, Nv, sd = shapes[idx]
        inst = synth.make_instance(No, Nv, sd, sigma_off=1e-3)
        t0 = time.perf_counter()
        h = esmp2.Handle(*(torch.from_numpy(inst[k]).cuda() for k in ("F", "ovov", "ooov", "ovvv", "C")))
        h.solve(tol=args.tol, maxit=args.maxit, precision=esmp2.FP64)
        e64 = h.energy()["E2"]
        h.close()
        torch.cuda.synchronize()
        t_seq64 += time.perf_counter() - t0
        w_seq64 += No * No * float(Nv) ** 3
        e2_diffs.append(abs(e2_by_seed[sd] - e64))
        del inst
    est64 = t_seq64 * (w_all / w_seq64) if w_seq64 > 0 else None
    # the reduced-cost basis form of the same batch (no virtual-index contraction), reported
    # beside the tensor-core form
    red = None
    if not args.no_variants and prec != esmp2.REDUCED_MIXED:
        t_red, worst_red, d_red = 0.0, 0.0, 0.0
        e_main = {}
        for w0 in range(0, len(shapes), args.wave):
            wave = shapes[w0:w0 + args.wave]
            insts = [synth.make_instance(No, Nv, sd, sigma_off=1e-3) for (No, Nv, sd) in wave]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, res = esmp2.batch_solve(insts, tol=args.tol, maxit=args.maxit, precision=esmp2.REDUCED_MIXED,
                                        concurrency=args.concurrency)
            torch.cuda.synchronize()
            t_red += time.perf_counter() - t0
            if st != esmp2.OK:
                raise RuntimeError("batch_solve (reduced) failed: " + "; ".join(r["message"] for r in res if r["status"]))
            for (No, Nv, sd), r in zip(wave, res):
                worst_red = max(worst_red, r["rel_residual"])
                e_main[sd] = r["E2"]
            del insts
        red = {"value": len(shapes) / t_red, "unit": "solves/s", "batch_seconds": t_red, "worst_rel_residual": worst_red}
    if red is not None:
        red["max_abs_E2_minus_main"] = max(abs(e_main[sd] - e2_by_seed[sd]) for sd in e_main)
    peaks, peak_src = load_peaks()
    fp64_peak = measure_fp64_peak(torch.device("cuda", 0))
    fams = {k: family_roofline(k, v, peaks, peak_src, fp64_peak, 1) for k, v in ktimes.items()}
    roofline = None
    if ktimes:
        dom = max(ktimes, key=lambda k: ktimes[k]["ms"])
        roofline = dict(fams[dom])
        roofline["family"] = dom
        # the stored dram capture is of the No=30 Nv=400 workload, not of these instances
        roofline["traffic"] = None
        roofline["traffic_source"] = None
        roofline["note"] = "kernel families over the batch's timed waves"
    cb = None
    if rank == 0 and not args.no_cpu_baseline:
        # O2 on four instances of the batch (sampled sigma elements, extrapolated), scaled to all 64
        t_cpu, w_cpu, parts = 0.0, 0.0, []
        for (No, Nv, sd) in shapes[::16]:
            c1 = cpu_baseline(No, Nv, sd, 1e-3, budget_s=max(2.0, args.ref_budget / 4), tol=args.tol)
            t_cpu += c1["value"]
            w_cpu += No * No * float(Nv) ** 3
            parts.append({"No": No, "Nv": Nv, "seed": sd, "seconds": c1["value"]})
        t_all = t_cpu * (w_all / w_cpu)
        cb = {"value": n_done / t_all, "unit": "solves/s", "cores": c1["cores"], "cpu_model": c1["cpu_model"],
              "kind": "oracle", "extrapolated": True,
              "sample": ("O2 solves of instances 0, 16, 32, 48 of the batch, each extrapolated from sampled sigma "
                         "elements, summed and scaled to all 64 by No^2 Nv^3"), "instances": parts}
    line = {"metric": "ESMP2 batched solves/s, 64 uneven instances (No 8-32, Nv 8-14 x No), res<1e-8, mixed",
            "value": n_done / t_batch, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": t_batch * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f64" if prec != esmp2.MIXED_TF32 else "tf32+f64", "data": "synthetic",
            "config": {"workload": "c4: synth.batch_shapes(64) seeds 100-163, sigma_off 1e-3", "tol": args.tol,
                       "precision": args.precision, "concurrency": args.concurrency, "wave": args.wave,
                       "step": "esmp2_batch_solve per wave (create from host inputs + solve + energy + destroy)",
                       "l2": "no flush: instances are solved once each"},
            "roofline": roofline, "kernel_families": fams, "cpu_baseline": cb,
            "e2e": {"value": n_done / t_batch, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(n_done * 8 * 4)},
            "gpu_launches": launches, "clocks": clocks,
            "instances": n_done, "batch_seconds": t_batch, "worst_rel_residual": worst_res,
            "inner_iterations_total": int(sum(iters)), "reduced_basis_form": red,
            "fp64_sequential": {"seconds_measured": t_seq64, "instances_measured": len(e2_diffs),
                                "seconds_estimated_all": est64,
                                "solves_per_s_estimated": (n_done / est64) if est64 else None,
                                "max_abs_E2_mixed_minus_fp64": max(e2_diffs) if e2_diffs else None,
                                "scaling": "measured seconds x (sum No^2 Nv^3 over all / over measured)"}}
    if rank == 0:
        print(json.dumps(line))
    return 0


def family_roofline(name, kt, peaks, peak_src, fp64_peak, steps):
    """Achieved rate of one kernel family from its own CUDA events over the timed region."""
    sec = kt["ms"] * 1e-3
    out = {"launches": kt["launches"], "kernel_ms_per_step": kt["ms"] / steps,
           "avg_launch_ms": kt["ms"] / max(1, kt["launches"])}
    if sec <= 0:
        return out
    if name == "precond":
        out.update({"bound": "tensor", "unit": "TFLOP/s", "peak": peaks["bf16_tflops_sustained"],
                    "achieved": kt["exec_units"] / sec / 1e12, "achieved_executed": kt["exec_units"] / sec / 1e12,
                    "kernel": "vg::k_vgemm, bf16 rotations of the inner preconditioner (executed flops: extra work "
                              "beyond the method's count)",
                    "peak_source": f"bf16 dense sustained, {peak_src} (MEASURED_PEAKS.json)"})
    elif name in ("contraction", "digits"):
        out.update({"bound": "tensor", "unit": "TFLOP/s", "peak": peaks["bf16_tflops_sustained"],
                    "achieved": kt["alg_units"] / sec / 1e12, "achieved_executed": kt["exec_units"] / sec / 1e12,
                    "peak_source": f"bf16 dense sustained, {peak_src} (MEASURED_PEAKS.json)"})
        out["kernel"] = ("vg::k_vgemm, bf16 (or tf32) operands, the packed inner sigma's virtual-index GEMM: achieved = "
                         "the method's flops 4 n_unique Nv per build"
                         if name == "contraction" else
                         "k_virt, exact bf16 digit products (float64-accurate residual, energy, rotations): "
                         "achieved = the method's flops of each contraction once; achieved_executed = every "
                         "digit pair the tensor cores run")
    elif name == "coupling":
        out.update({"bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"], "achieved": kt["alg_units"] / sec / 1e9,
                    "kernel": "kp_couple_anti/s/z (packed float32 inner coupling pass) and k_couple (float64 true "
                              "residual): algorithmic bytes = one read of x and of the products, one write of y",
                    "peak_source": f"copy bandwidth, {peak_src} (MEASURED_PEAKS.json)"})
    elif name == "gemm64":
        out.update({"bound": "alu", "unit": "TFLOP/s", "peak": fp64_peak, "achieved": kt["alg_units"] / sec / 1e12,
                    "kernel": "gemm64_kernel: float64 GEMM on the CUDA cores",
                    "peak_source": "float64 GEMM rate measured in this run (torch.matmul 4096^3, cuBLAS)"})
    else:
        out.update({"bound": "alu", "unit": "Gelem/s", "peak": None, "achieved": kt["alg_units"] / sec / 1e9,
                    "kernel": "k_e2s: S-space energy sum (double-float on the float32 pipes)",
                    "peak_source": "no measured float32 peak"})
    if out.get("achieved") is not None and out.get("peak"):
        out["frac"] = out["achieved"] / out["peak"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="c3", choices=sorted(WORKLOADS) + ["c4"])
    ap.add_argument("--wave", type=int, default=16, help="c4: instances generated and solved per batch call")
    ap.add_argument("--concurrency", type=int, default=3, help="c4: host workers (streams) of the batch")
    ap.add_argument("--fp64-every", type=int, default=8, help="c4: time plain FP64 on every k-th instance")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "mixed", "tf32", "reduced", "minres"])
    ap.add_argument("--no-variants", action="store_true", help="skip the tf32 and reduced-basis forms")
    ap.add_argument("--minres-probe", type=int, default=150, help="MINRES iterations tried on an indefinite workload")
    ap.add_argument("--tol", type=float, default=None, help="default: the workload's (1e-8 mixed, 1e-10 fp64)")
    ap.add_argument("--maxit", type=int, default=3000)
    ap.add_argument("--ref-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the single plain-fp64 solve reported beside the mixed headline")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "c4":
        if args.tol is None:
            args.tol = 1e-8
        return run_batch(args)

    import torch
    import torch.distributed as dist
    from paper_2003_12923_gb300 import esmp2

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    No, Nv, seed, so, prec0, tol0 = WORKLOADS[args.config]
    tol = args.tol if args.tol is not None else tol0
    seed = seed + 1000 * rank
    inst = make_inputs(No, Nv, seed, so)
    names = ("F", "ovov", "ooov", "ovvv", "C")
    dins = {k: torch.from_numpy(inst[k]).to(dev) for k in names}
    esmp2.load()
    prec_name = prec0 if args.precision == "auto" else args.precision
    prec = {"mixed": esmp2.MIXED_BF16, "tf32": esmp2.MIXED_TF32, "reduced": esmp2.REDUCED_MIXED,
            "fp64": esmp2.FP64, "minres": esmp2.REDUCED_MINRES}[prec_name]
    stream = torch.cuda.current_stream()
    fp64_peak = measure_fp64_peak(dev)

    hkw = {}   # problem-statement options of the handles (the level shift of an indefinite workload)

    def step(inputs, precision=None):
        h = esmp2.Handle(*(inputs[k] for k in names), **hkw)
        info = h.solve(tol=tol, maxit=args.maxit, precision=prec if precision is None else precision)
        e = h.energy()
        n_l = h.kernel_launches
        h.close()
        return info, e, n_l

    indefinite = None
    try:
        step(dins)
    except esmp2.Esmp2Error as err:
        if err.status != esmp2.ERR_INDEFINITE:
            raise
        # CG does not apply (Sec. III.A uses CG, which needs a positive definite operator): the
        # lowest Ritz values of a short Lanczos run are the evidence.  Preconditioned MINRES is
        # probed with a bounded number of iterations; the timed solve applies the level shift
        # (the intruder-state remedy) just large enough to make the operator positive definite.
        lz = lanczos_ritz(esmp2, dins, names)
        hm = esmp2.Handle(*(dins[k] for k in names))
        t0 = time.perf_counter()
        im = hm.solve(tol=tol, maxit=args.minres_probe, precision=esmp2.REDUCED_MINRES, raise_on_error=False)
        torch.cuda.synchronize()
        probe = {"iterations": im["iterations"], "rel_residual": im["rel_residual"],
                 "seconds": time.perf_counter() - t0, "status": im["status"]}
        hm.close()
        shift = float(np.ceil((-lz["ritz_min"] + 0.1) * 10.0) / 10.0)
        indefinite = {"cg_status": "indefinite", "message": str(err), "lanczos": lz, "minres_probe": probe,
                      "level_shift": shift,
                      "note": "the timed solve is the mixed CG solve of A + level_shift (E2 of the shifted operator)"}
        hkw["level_shift"] = shift
        step(dins)
    for _ in range(args.warmup - 1):
        step(dins)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    esmp2.kernel_timing(True)     # event pairs around every launch of the hot-path kernel families
    esmp2.kernel_times()          # clear
    clk = ClockSampler(uuid)
    clk.start()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos, launches = [], 0
    for _ in range(args.steps):
        info, e, n_l = step(dins)
        infos.append((info, e))
        launches += n_l
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ktimes = esmp2.kernel_times()
    esmp2.kernel_timing(False)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    if world > 1:
        elapsed = max_over_ranks(elapsed, dist, dev)
    tts = elapsed / args.steps

    # every kernel family of the timed region from its own CUDA events; the headline roofline
    # is the family with the largest device time
    peaks, peak_src = load_peaks()
    fams = {k: family_roofline(k, v, peaks, peak_src, fp64_peak, args.steps) for k, v in ktimes.items()}
    for k in fams:
        fams[k]["share_of_step"] = ktimes[k]["ms"] / 1e3 / elapsed
    dom = max(ktimes, key=lambda k: ktimes[k]["ms"])
    roofline = dict(fams[dom])
    roofline["family"] = dom
    ent, prof = kernel_traffic(dom)
    roofline["traffic"] = ent["bytes_per_launch"] if ent else None
    roofline["traffic_source"] = prof

    # per-stage view of one sigma build of this precision (outside the timed region)
    h = esmp2.Handle(*(dins[k] for k in names), **hkw)
    x = h.rhs()
    # (MINRES runs the float64 sigma of the reduced-cost basis, not profiled per stage: the
    # float64 stages of the TOP-basis sigma are shown instead)
    ms = h.profile_sigma(x, precision=esmp2.FP64 if prec == esmp2.REDUCED_MINRES else prec, reps=3)
    fl = sigma_flops(No, Nv)
    nu = unique_amplitudes(No, Nv)
    roofline["sigma_stage_ms"] = [float(v) for v in ms[:5]]
    sigma_alg_tflops = fl["alg_total"] / (ms[4] * 1e-3) / 1e12
    sigma_alg_gbs = (16.0 if prec in (esmp2.FP64, esmp2.REDUCED_MINRES) else 6.0) * nu / (ms[4] * 1e-3) / 1e9
    h.close()

    e2e = None
    if not args.no_e2e:
        pinned = {}
        for k in names:
            t = torch.empty(inst[k].shape, dtype=torch.float64, pin_memory=True)
            t.numpy()[...] = inst[k]
            pinned[k] = t.numpy()
        h2d = sum(pinned[k].nbytes for k in names)
        step(pinned)   # untimed: the staging buffers of host inputs are the device pool's first use
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(2):
            info_e, e_e, _ = step(pinned)
        torch.cuda.synchronize()
        t_e2e = (time.perf_counter() - t0) / 2
        d2h = 8 * 32 * (info_e["iterations"] + 4 * info_e["outer"] + 8) + 8 * 32 * 6
        e2e = {"value": t_e2e, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    fp64_cmp = None
    if prec not in (esmp2.FP64, esmp2.REDUCED_MINRES) and not args.no_fp64_compare:
        # the plain float64 GPU form on the same instance, timed once with CUDA events
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h64 = esmp2.Handle(*(dins[k] for k in names), **hkw)
        info64 = h64.solve(tol=tol, maxit=args.maxit, precision=esmp2.FP64)
        en64 = h64.energy()
        h64.close()
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_cmp = {"time_to_solution_s": e0.elapsed_time(e1) / 1e3, "iterations": info64["iterations"],
                    "rel_residual": info64["rel_residual"], "E2": en64["E2"]}

    # the other inner forms on the same instance, each timed once after one untimed run (CUDA
    # events, create + solve + energy like the step): tf32 contraction, and the reduced-cost basis
    # (no virtual-index contraction at all; reported beside the tensor-core form, not instead)
    variants = {}
    if prec not in (esmp2.FP64, esmp2.REDUCED_MINRES) and No <= 32 and not args.no_variants:
        for name, pv in (("tf32_form", esmp2.MIXED_TF32), ("reduced_basis_form", esmp2.REDUCED_MIXED)):
            if pv == prec:
                continue
            step(dins, pv)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info_v, e_v, _ = step(dins, pv)
            e1.record(stream)
            torch.cuda.synchronize()
            variants[name] = {"time_to_solution_s": e0.elapsed_time(e1) / 1e3, "iterations": info_v["iterations"],
                              "outer": info_v["outer"], "rel_residual": info_v["rel_residual"], "E2": e_v["E2"],
                              "E2_minus_main": e_v["E2"] - infos[-1][1]["E2"]}

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(No, Nv, seed, so, inst=inst, tol=tol, config=args.config)

    info, e = infos[-1]
    line = {"metric": METRIC, "value": tts, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tts * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec in (esmp2.FP64, esmp2.REDUCED_MINRES) else "bf16+f64",
            "data": "synthetic",
            "config": {"workload": f"{args.config}: No={No} Nv={Nv} seed={seed} sigma_off={so} TOP(1)",
                       "tol": tol, "precision": prec_name, "step": "create+solve+energy, inputs resident",
                       "l2": "no flush: every block vector (5.8 GB at No=30 Nv=400) is larger than L2"},
            "roofline": roofline, "kernel_families": fams, "fp64_gemm_peak_tflops": fp64_peak,
            "cpu_baseline": cb, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
            "sigma_builds_per_s": 1e3 / ms[4], "sigma_tflops_alg": sigma_alg_tflops, "sigma_gbs_alg": sigma_alg_gbs,
            "iterations": info["iterations"], "outer": info["outer"], "sigma_fp64": info["sigma_fp64"],
            "sigma_lowp": info["sigma_lowp"], "rel_residual": info["rel_residual"], "E2": e["E2"],
            "E2_parts": e}
    g = _golden(args.config)
    if g is not None and seed == g["instance"]["seed"]:
        line["E2_error_vs_oracle"] = {k: e[k] - g[k] for k in ("E2", "E2_D", "E2_L", "E2_S")}
        line["E2_error_vs_oracle"]["oracle"] = GOLDEN[args.config]
    line.update(variants)
    if indefinite is not None:
        line["indefinite_for_cg"] = indefinite
    if fp64_cmp is not None:
        fp64_cmp["E2_mixed_minus_fp64"] = e["E2"] - fp64_cmp["E2"]
        fp64_cmp["speedup_mixed_over_fp64"] = fp64_cmp["time_to_solution_s"] / tts
        line["fp64_form"] = fp64_cmp
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def _mixed_available():
    from paper_2003_12923_gb300 import esmp2
    return getattr(esmp2, "MIXED_READY", False)


if __name__ == "__main__":
    sys.exit(main())
