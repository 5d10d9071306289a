#!/usr/bin/env python
"""DF-EA-ADC(3) sigma throughput and time-to-roots on GB300.

Workload (default): canonical EA-ADC(3), o=20 occupied, v=200 virtual,
naux=600 auxiliary functions, 4 roots, synthetic inputs from ``synth``
(seeded SplitMix64/Box-Muller generator; occupied energies uniform in
[-1.2,-0.4] Eh, virtual energies log-spaced 0.02-20 Eh, symmetric Gaussian
B^Q with decay exp(-Q/150), scaled to max |t| = 0.05).

One timed step = one sigma = M c over the 4 root vectors in mixed precision
(DF ladder, ring and second-order coupling GEMMs on tcgen05 BF16 tensor cores
with FP32 accumulation; DF coupling pieces in FP32; diagonal and 1p/1p block
in FP64), the unit Davidson repeats every iteration.  L2 is flushed (256 MB
write) between timed steps.  Time-to-roots is measured once beside it: the
mixed-precision Davidson (to its noise floor) with a final sigma-and-Ritz step
in FP64 (or in split BF16), against the plain FP64 GPU Davidson (diagonal
correction) converged to ||r|| <= 1e-4, all from built states, with the
errors against the oracle's roots (tests/golden/canonical-200.npz).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DF-EA-ADC(3) sigma TFLOP/s + time-to-roots vs FP64 GPU at ≤1e-5 Eh"
WORKLOAD = "canonical-200"
NROOTS = 4


def sigma_flops(o, v, naux, nvec):
    """Algorithmic flops of one sigma: DF ladder 4 o v^3 naux, ring 3 x 2 (ov)^2 v,
    second-order coupling 6 x 2 (ov)^2 v, DF coupling pieces 8 x 2 naux o v^2."""
    return nvec * (4.0 * o * v ** 3 * naux + 18.0 * o * o * v ** 3 + 16.0 * naux * o * v * v)


def ladder_flops(o, v, naux, nvec):
    return nvec * 4.0 * o * v ** 3 * naux


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("bf16_tflops", 1900.0), d.get("hbm_gbs", 6800.0), "measured"
    return 1900.0, 6800.0, "fallback"


def source_sha():
    h = hashlib.sha256()
    for f in ("tc_gemm.cuh", "tc_common.cuh", "tc_gemm2.cuh", "tc_gemm2.cu"):
        h.update(open(os.path.join(ROOT, "paper_2511_05897_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ladder_traffic():
    """DRAM bytes per ladder call from the committed ncu summary, if it was
    taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "ladder_canonical-200.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    return d.get("dram_bytes_per_call") if d.get("source_sha") == source_sha() else None


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(pr, nvec=1):
    """The CPU oracle's sigma (numpy FP64, all host cores) on a bounded sample:
    nvec vectors of the same workload (the 1p/1p intermediate, a one-off
    construction, is replaced by its diagonal: the per-vector cost is the same)."""
    from oracle import restricted as R

    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    sig = R.Sigma.__new__(R.Sigma)
    sig.p, sig.order = p, 3
    sig.M11 = np.diag(p.ev)
    sig.D2p1h = R.diag_2p1h(p)
    dim = p.v + p.o * p.v * p.v
    x = np.random.default_rng(0).standard_normal((nvec, dim))
    t0 = time.perf_counter()
    sig(x)
    dt = time.perf_counter() - t0
    fl = sigma_flops(p.o, p.v, p.naux, nvec)
    return {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{nvec} sigma vector(s) of {WORKLOAD} (numpy FP64, BLAS on all host cores), {dt:.1f} s"}


def job_rate(local_ms, flops_per_rank_step, world, device):
    """Whole-job rate of weak-scaled replicas: every rank does the same work
    per step; the step time is the slowest rank's (max over ranks).  Returns
    (ms_per_step, TFLOP/s of all ranks together)."""
    ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * flops_per_rank_step / (ms * 1e-3) / 1e12


def bench_config(o, v, naux):
    """The workload both arms report (the reference arm times one vector of it per step)."""
    return {"workload": f"{WORKLOAD}: canonical EA-ADC(3), o={o}, v={v}, naux={naux}, {NROOTS} roots",
            "nvec_per_step": NROOTS, "l2": "flushed (256 MB write) between timed steps",
            "precision": "BF16 tensor-core operands, FP32 accumulation; DF coupling pieces FP32; "
                         "diagonal and 1p/1p block FP64"}


FNO_STATES, FNO_THRESH, NAF_THRESH = 4, 0.15, 0.1


def fno_states(E, ctx):
    """Per-state truncated spaces (Sec. III) for the 4 lowest canonical ADC(2)
    roots: build (canonical ADC(2) roots, densities, natural orbitals, NAFs,
    intermediates), the 3 lowest roots of every state (BF16 Davidson with a
    split-BF16 Ritz step) and Eq. 30 (FP64 ADC(2) in each truncated space).
    Thresholds 0.15 (occupation) and 0.1 (auxiliary metric) keep about 60 %
    of the virtuals and half of the auxiliary functions of this problem."""
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E.eaadc_build_states(ctx, FNO_STATES, FNO_THRESH, NAF_THRESH, 3, 1.0, can_opts=dict(tol=1e-6, maxit=300))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    om, rn, it, st = E.eaadc_davidson(ctx, 3, tol=1e-5, prec=E.EAADC_MIXED_BF16, refine=3, max_sub=40, maxit=300)
    t2 = time.perf_counter()
    en = E.eaadc_ea_energies(ctx, dict(tol=1e-6, maxit=300))
    t3 = time.perf_counter()
    info = [E.eaadc_state_info(ctx, k) for k in range(FNO_STATES)]
    return {"nstates": FNO_STATES, "fno_thresh": FNO_THRESH, "naf_thresh": NAF_THRESH,
            "vprime": [i[0] for i in info], "nauxprime": [i[1] for i in info],
            "build_s": t1 - t0, "davidson_s": t2 - t1, "eq30_s": t3 - t2, "davidson_iterations": [int(i) for i in it],
            "omega_uncorr_eh": [float(w) for w in en["omega_uncorr"]],
            "omega_corr_eh": [float(w) for w in en["omega_corr"]],
            "omega2_can_eh": [float(w) for w in en["omega2_can"]],
            "mode": "states sequential; BF16 Davidson + split-BF16 Ritz step per state; Eq. 30 in FP64"}


def end_to_end(E, pr, device, stream, fp64_build_s, fp64_solve_s):
    """From host inputs to the 4 roots within 1e-5 Eh: upload, build (amplitude
    ladder on the tensor cores, split BF16), BF16 Davidson with a split-BF16
    Ritz step; against the FP64 upload + build + FP64 GPU Davidson."""
    import torch

    gold = golden_roots()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = E.eaadc_init(pr["o"], pr["v"], pr["naux"], pr["eps_occ"], pr["eps_vir"], pr["B"], device, stream)
    try:
        E.eaadc_set_build_precision(ctx, E.EAADC_MIXED_BF16X3)
        E.eaadc_build_canonical(ctx, 3, 1.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        om, rn, it, st = E.eaadc_davidson(ctx, NROOTS, tol=1e-5, prec=E.EAADC_MIXED_BF16, refine=3, max_sub=40,
                                          maxit=300)
        t2 = time.perf_counter()
    finally:
        E.eaadc_destroy(ctx)
    out = {"ours": {"seconds": t2 - t0, "init_build_s": t1 - t0, "solve_s": t2 - t1,
                    "mode": "split-BF16 amplitude ladder in the build; BF16 Davidson + split-BF16 Ritz step"},
           "fp64_gpu": {"seconds": fp64_build_s + fp64_solve_s, "init_build_s": fp64_build_s,
                        "solve_s": fp64_solve_s}}
    if gold is not None:
        out["ours"]["max_err_vs_oracle_eh"] = float(np.abs(om[0] - gold).max())
    out["speedup_vs_fp64_gpu"] = out["fp64_gpu"]["seconds"] / out["ours"]["seconds"]
    return out


def golden_roots():
    p = os.path.join(ROOT, "tests", "golden", "canonical-200.npz")
    return np.load(p)["omega3"] if os.path.exists(p) else None


def time_to_roots(E, ctx, fp64_baseline=True):
    """Seconds from built state to the 4 lowest roots within 1e-5 Eh: ours
    (BF16 tensor-core sigma to the noise floor, then one sigma-and-Ritz step in
    FP64 or in split BF16) and the plain FP64 GPU Davidson; errors against the
    oracle's roots."""
    import torch

    gold = golden_roots()
    out = {}
    runs = [("mixed_bf16_fp64_ritz", dict(tol=1e-5, prec=E.EAADC_MIXED_BF16, refine=2)),
            ("mixed_bf16_x3_ritz", dict(tol=1e-5, prec=E.EAADC_MIXED_BF16, refine=3))]
    if fp64_baseline:
        runs.append(("fp64_gpu", dict(tol=1e-4, etol=1e-6, prec=E.EAADC_FP64, refine=0)))
    for name, kw in runs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        om, rn, it, st = E.eaadc_davidson(ctx, NROOTS, max_sub=40, maxit=300, **kw)
        dt = time.perf_counter() - t0
        out[name] = {"seconds": dt, "iterations": int(it[0]), "status": int(st),
                     "omega_eh": [float(w) for w in om[0]], "resnorm": [float(r) for r in rn[0]]}
        if gold is not None:
            out[name]["max_err_vs_oracle_eh"] = float(np.abs(om[0] - gold).max())
    if "fp64_gpu" in out:
        for k in ("mixed_bf16_fp64_ritz", "mixed_bf16_x3_ritz"):
            out[k]["speedup_vs_fp64_gpu"] = out["fp64_gpu"]["seconds"] / out[k]["seconds"]
    return out


def run_reference(args, rank):
    if rank != 0:
        return
    from synth import config_problem

    pr = config_problem(WORKLOAD)
    times = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(pr, 1)
        if i >= args.warmup:
            times.append(cb)
    val = statistics.mean(t["value"] for t in times)
    o, v, naux = pr["o"], pr["v"], pr["naux"]
    fl = sigma_flops(o, v, naux, 1)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": fl / (val * 1e12) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(o, v, naux),
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "1 sigma vector per step (numpy FP64 oracle on all host cores)"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-roots", action="store_true", help="skip the time-to-roots solves")
    ap.add_argument("--no-fp64-baseline", action="store_true", help="skip the FP64 GPU Davidson baseline")
    ap.add_argument("--no-fno", action="store_true", help="skip the per-state FNO/NAF run")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    args.warmup = max(3, args.warmup)

    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import paper_2511_05897_gb300 as E

    if not os.path.exists(E.LIB_PATH):
        import __graft_entry__ as g

        g.build()
    from synth import config_problem

    pr = config_problem(WORKLOAD)
    o, v, naux = pr["o"], pr["v"], pr["naux"]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    torch.cuda.synchronize()
    t_init0 = time.perf_counter()
    ctx = E.eaadc_init(o, v, naux, pr["eps_occ"], pr["eps_vir"], pr["B"], local, sh)
    try:
        E.eaadc_build_canonical(ctx, 3, 1.0)
        torch.cuda.synchronize()
        init_build_fp64_s = time.perf_counter() - t_init0
        _, _, dim = E.eaadc_state_info(ctx, 0)
        nvec = NROOTS
        x = torch.randn(nvec, dim, dtype=torch.float64, device="cuda")
        x /= x.norm(dim=1, keepdim=True)
        y = torch.empty_like(x)
        lad = torch.empty(nvec, o, v, v, dtype=torch.float32, device="cuda")
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        fl_step = sigma_flops(o, v, naux, nvec)

        def step():
            E.eaadc_sigma(ctx, 0, nvec, x.data_ptr(), y.data_ptr(), E.EAADC_MIXED_BF16, sh)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with Clocks(local) as clk:
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            n0 = E.eaadc_kernel_launches()
            for i in range(args.steps):
                flush.zero_()
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            n1 = E.eaadc_kernel_launches()
            if world > 1:
                dist.barrier()
            ms = [a.elapsed_time(b) for a, b in ev]
            # dominant kernel: the DF ladder alone, same stream
            lev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            torch.cuda.nvtx.range_push("roofline_ladder")  # lets a profiler select these launches
            for i in range(args.steps):
                flush.zero_()
                lev[i][0].record(stream)
                E.eaadc_ladder(ctx, 0, nvec, x.data_ptr(), lad.data_ptr(), sh)
                lev[i][1].record(stream)
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            lms = statistics.mean(a.elapsed_time(b) for a, b in lev)
            # the split-BF16 (three-product) sigma, same workload (after an untimed
            # call: the first one of a shape tunes the ladder chunk size)
            E.eaadc_sigma(ctx, 0, nvec, x.data_ptr(), y.data_ptr(), E.EAADC_MIXED_BF16X3, sh)
            xev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(max(2, args.steps // 2))]
            for a, b in xev:
                flush.zero_()
                a.record(stream)
                E.eaadc_sigma(ctx, 0, nvec, x.data_ptr(), y.data_ptr(), E.EAADC_MIXED_BF16X3, sh)
                b.record(stream)
            torch.cuda.synchronize()
            x3_ms = statistics.mean(a.elapsed_time(b) for a, b in xev)
            # end to end through the host-buffer entry point (pinned memory, copies timed)
            xh = torch.empty((nvec, dim), dtype=torch.float64, pin_memory=True)
            yh = torch.empty((nvec, dim), dtype=torch.float64, pin_memory=True)
            xh.copy_(x)
            xn, yn = xh.numpy(), yh.numpy()
            e2e_t = []
            for i in range(max(2, args.steps // 2)):
                t0 = time.perf_counter()
                E.eaadc_sigma_host(ctx, 0, xn, E.EAADC_MIXED_BF16, out=yn)
                e2e_t.append(time.perf_counter() - t0)
        mean_ms, value = job_rate(statistics.mean(ms), fl_step, world, "cuda")
        e2e_val = fl_step / statistics.mean(e2e_t) / 1e12
        bf16_peak, hbm_peak, src = peaks()
        achieved = ladder_flops(o, v, naux, nvec) / (lms * 1e-3) / 1e12
        roots = None
        if not args.no_roots and rank == 0:
            roots = time_to_roots(E, ctx, not args.no_fp64_baseline)
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": bench_config(o, v, naux),
            "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": nvec * dim * 8,
                    "d2h_bytes_per_step": nvec * dim * 8},
            "gpu_launches": int(n1 - n0),
            "sigma_bf16x3": {"value": fl_step / (x3_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": x3_ms,
                             "note": "each operand split into two BF16 parts, three products per GEMM"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": achieved / bf16_peak, "traffic": ladder_traffic(),
                         "kernel": "DF particle-particle ladder (tcgen05 BF16 GEMM stages), one call",
                         "ms_per_launch": lms, "peak_source": f"{src} bf16 dense burst"},
            "clocks": clk.summary(),
        }
        if roots is not None:
            line["time_to_roots"] = roots
        if roots is not None and "fp64_gpu" in roots:
            line["end_to_end"] = end_to_end(E, pr, local, sh, init_build_fp64_s, roots["fp64_gpu"]["seconds"])
        if not args.no_fno and rank == 0:
            line["fno_states"] = fno_states(E, ctx)
        if rank == 0 and world == 1:
            line["cpu_baseline"] = cpu_baseline(pr, 1)
        if rank == 0:
            print(json.dumps(line), flush=True)
    finally:
        E.eaadc_destroy(ctx)
        if world > 1:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
