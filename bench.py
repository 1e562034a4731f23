#!/usr/bin/env python3
"""Throughput benchmark of the semi-implicit IMEX hSGN step on GB300.

Workload (the dam-break / undular-bore configuration, run at 2^24 cells per
instance so that every state is far larger than L2): dx = 0.05, transmissive
ends, flat bottom, h = 1.2 on the left and 1.0 on the right joined by a tanh
transition of width 5 h0 (h0 = 1), u = 0, eta = h, w = 0; one instance per
relaxation parameter lambda in {10, 100, 1000}, each with its own
dt = min(4 dx / nu_max, 0.5 dx / u_max) computed at t = 0 (CFL_IMEX = 4,
material CFL 0.5). One benchmark step advances all three instances by one IMEX
step (two implicit stages each). Inputs are synthetic (seed-free closed forms).

The headline is the FP64-class double-float form (every value a pair of
single-precision numbers, one launch per stage; within 1e-12 per step of the
FP64 oracle). The FP64 form and the mixed-precision form (FP32 increments) are
timed on the same workload and reported beside it, each with its error against
the oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). --impl reference times the FP64 CPU oracle on
the host cores instead (the reference arm of this comparison).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "hSGN cell-stage updates/sec and % HBM roofline on 1 GB300 at stated L2 error vs FP64 oracle"
UNIT = "cell-stage updates/s"
L2_BYTES = 129 * 1024 * 1024
FLUSH_BYTES = 512 * 1024 * 1024

# Algorithmic traffic of one cell-stage in FP64 (flat bottom): stage 1 reads U^n
# (32 B) and writes U_I^(1) (32 B); stage 2 reads U^n and U_I^(1) (64 B) and
# writes U^{n+1} (32 B): 160 B per cell and step = 80 B per cell-stage; the
# bottom adds 8 B per cell-stage (read once per stage).
BYTES_PER_CELL_STAGE = 80.0
BYTES_PER_CELL_STAGE_BOTTOM = 88.0
# What the windowed mixed path itself moves per cell-stage: stage 1 reads U^n
# (32 B) and writes the FP32 increments (16 B); stage 2 reads U^n and the
# increments (48 B) and writes U^{n+1} (32 B): 64 B.
BYTES_MOVED_MIXED = 64.0
# Algorithmic FP64 operations of the flux + assembly + block elimination kernel
# per cell and launch (average of the two stages), counted from the kernel's
# formulas: stage-state combination 12, face reconstruction and Rusanov fluxes
# 47, starred values and coefficients 42, matrix row and right-hand side 23,
# chunk Thomas sweep with three right-hand sides and recombination 25
# (a fused multiply-add counts 2, a division 1).
FLOPS_PER_CELL_ASSEMBLE = 149.0
# Single-precision operations the double-float stage kernel executes per cell
# and launch (average of its two stages, window overlap included): ncu's
# per-launch counts of FADD + FMUL + 2 FFMA (sm__sass_thread_inst_executed_op_
# {fadd,fmul,ffma}_pred_on.sum) divided by the cells of the launch, on the
# 2^22-cell dam break (lambda = 1000, 64-row window overlap; the capture of
# profiles/ncu_df_stage.md).
# Valid for the kernel sources whose hash is DF_FLOPS_SOURCE_SHA; None when the
# kernel has changed since (the roofline then reports no achieved flop rate).
DF_FLOPS_PER_CELL = 1481.5      # stage 1 / 2: 1389 / 1574
DF_FP32_INST_PER_CELL = 1220.5  # FADD + FMUL + FFMA instructions, stage 1 / 2: 1143 / 1298
DF_TRAFFIC_PER_CELL = 70.9      # dram__bytes_read + write per cell and launch, stage 1 / 2: 53.1 / 88.6
DF_FLOPS_SOURCE_SHA = "c2cfbebac1571de6"
DF_SOURCES = ("hsgn_dfstage.cuh", "hsgn_dfloat.cuh", "hsgn_fused.cuh", "hsgn_mixed.cuh",
              "hsgn_kernels.cuh", "hsgn_tridiag.cuh")


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--log2n", type=int, default=24)
    ap.add_argument("--lams", default="10,100,1000")
    ap.add_argument("--cpu-steps", type=int, default=3,
                    help="oracle steps per instance for the CPU baseline and the L2 check")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 path")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision path")
    ap.add_argument("--no-comparators", action="store_true",
                    help="skip the scheme comparison (time to solution)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint workload")
    ap.add_argument("--no-shelf", action="store_true", help="skip the 2^24-cell shelf workload")
    ap.add_argument("--no-paper-runs", action="store_true",
                    help="skip the runs of the paper's CPU-time tables")
    ap.add_argument("--no-tridiag", action="store_true",
                    help="skip the standalone tridiagonal solve")
    ap.add_argument("--tridiag-log2n", type=int, default=24, help="rows of that solve (log2)")
    ap.add_argument("--accuracy", action="store_true",
                    help="instead of the benchmark: both forms against the FP64 oracle / form "
                         "over the configurations' full lengths (minutes)")
    ap.add_argument("--accuracy-steps", type=int, default=2000)
    ap.add_argument("--shelf-accuracy-steps", type=int, default=5000)
    ap.add_argument("--shelf-log2n", type=int, default=24, help="cells of the shelf workload (log2)")
    ap.add_argument("--shelf-steps", type=int, default=50, help="timed steps of the shelf workload")
    ap.add_argument("--sequential", action="store_true",
                    help="run the instances of a step back to back on one stream "
                         "(default: one CUDA stream each)")
    ap.add_argument("--batch", type=int, default=4096, help="instances of the batched workload")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def workload(log2n: int, lams):
    from paper_2510_07539_gb300 import inputs
    n = 1 << log2n
    dx = 0.05
    x, U = inputs.dam_break(n, dx, 1.2, 1.0, 5.0 / dx)
    return n, dx, -0.5 * n * dx, 0.5 * n * dx, U, [float(l) for l in lams]


def config_dict(n, lams, dts, extra=None):
    d = {
        "workload": "hSGN dam break / undular bore, 1D, flat bottom, transmissive",
        "cells": n,
        "instances": len(lams),
        "lambda": lams,
        "dt": dts,
        "dx": 0.05,
        "h_left": 1.2,
        "h_right": 1.0,
        "transition_width": "5 h0 (tanh)",
        "cfl_imex": 4.0,
        "mcfl": 0.5,
        "scheme": "2-stage IMEX RK (printed tableau)",
        "rusanov_speed": "global max|u^n|",
        "streams": "one CUDA stream per instance, joined every step",
        "l2_between_steps": f"flushed ({FLUSH_BYTES >> 20} MiB write) before every timed step",
    }
    if extra:
        d.update(extra)
    return d


def code_of(text: str) -> str:
    """C/C++/CUDA source without its comments, trailing blanks and empty lines
    (a comment changes no instruction the counters were taken from). String
    literals are kept as they are."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            while i < n and text[i] != "\n":
                i += 1
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = (ln.rstrip() for ln in "".join(out).split("\n"))
    return "\n".join(ln for ln in lines if ln)


def source_sha(files=None) -> str:
    """Hash of kernel sources without comments: the named files of the
    library's csrc folder (a kernel's own header and those it includes), or
    all of them."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2510_07539_gb300", "csrc")
    names = sorted(files) if files else sorted(os.listdir(csrc))
    for name in names:
        with open(os.path.join(csrc, name), encoding="utf-8") as fh:
            h.update(code_of(fh.read()).encode("utf-8"))
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_steps(n, dx, U, lams, dts, steps):
    import oracle
    oracle.build()
    out, t0 = [], time.perf_counter()
    for lam, dt in zip(lams, dts):
        p = oracle.Params(n, dx, oracle.BC_TRANSMISSIVE, lam=lam)
        out.append(oracle.run(p, U, dt, steps))
    return out, time.perf_counter() - t0


def cpu_dts(n, dx, U, lams):
    import oracle
    return [oracle.suggest_dt(oracle.Params(n, dx, oracle.BC_TRANSMISSIVE, lam=l), U, 4.0, 0.5)[0]
            for l in lams]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    lams = [float(x) for x in args.lams.split(",")]
    # a bounded sample: at most about 1.5e9 cell-stages of oracle work in all
    # (about a minute on one core), taken as the same dam break on a smaller
    # grid of the same spacing when K + W steps of the full grid would exceed it
    log2n = args.log2n
    while log2n > 10 and 2.0 * (1 << log2n) * len(lams) * (args.steps + args.warmup) > 1.5e9:
        log2n -= 1
    n, dx, _, _, U, lams = workload(log2n, lams)
    dts = cpu_dts(n, dx, U, lams)
    import oracle
    oracle.build()
    params = [oracle.Params(n, dx, oracle.BC_TRANSMISSIVE, lam=l) for l in lams]
    states = [U for _ in lams]
    for _ in range(args.warmup):
        states = [oracle.run(p, s, dt, 1) for p, s, dt in zip(params, states, dts)]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        states = [oracle.run(p, s, dt, 1) for p, s, dt in zip(params, states, dts)]
    el = time.perf_counter() - t0
    units = 2.0 * n * len(lams) * args.steps
    value = units / el
    sample = (f"{args.steps} full IMEX steps of all {len(lams)} instances "
              f"({n} cells each" + ("" if log2n == args.log2n else
                                     f", the workload's {1 << args.log2n}-cell grid "
                                     "sampled as the same dam break on fewer cells") +
              "), single-threaded C oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(n, lams, dts),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# replicas: whole-job value from per-rank timings
# ---------------------------------------------------------------------------
def combine_ranks(dist, local_ms: float, local_units: float, device="cpu"):
    """Max over ranks of the timed region and sum over ranks of the work done.
    The job value is (sum of units) / (slowest rank's time): each rank runs
    an independent replica of the workload (no data exchange)."""
    import torch
    if dist is None:
        return local_ms, local_units
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def sep_launches(n: int) -> int:
    """Kernel launches of the separator-system solve of n blocks (mirrors the
    library: one warp for <= 128 rows, else reduce + recurse + back-out)."""
    return 1 if n <= 128 else 2 + sep_launches((n + 127) // 128)


def time_path(S, torch, flags, n, xl, xr, lams, Ud, steps, warmup, flush, stream, dist, clocks,
              concurrent=False):
    """K timed steps of the three-instance workload in one precision form."""
    sols = [S.Solver(n, xl, xr, S.BC_TRANSMISSIVE, lam=l, flags=flags) for l in lams]
    for s in sols:
        s.set_state(*Ud)
    dts = [s.suggest_dt(4.0, 0.5) for s in sols]
    # the instances are independent. Default: one after the other on the
    # timing stream (each kernel's event pair then times that kernel alone);
    # concurrent: one CUDA stream each, forked and joined every step
    side = [torch.cuda.Stream() for _ in sols]
    fork = torch.cuda.Event()
    joins = [torch.cuda.Event() for _ in sols]

    def one_step():
        if not concurrent:
            for s, dt in zip(sols, dts):
                s.step(dt, stream=stream)
            return
        fork.record(stream)
        for s, dt, st, j in zip(sols, dts, side, joins):
            st.wait_event(fork)
            s.step(dt, stream=st)
            j.record(st)
        for j in joins:
            stream.wait_event(j)

    for _ in range(warmup):
        one_step()
    for s in sols:
        s.check()
        s.profile(True)
        s.profile_read(reset=True)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    sampler = ClockSampler(clocks) if clocks else None
    if sampler:
        time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(steps):
        flush.fill_(float(k))
        ev0[k].record(stream)
        one_step()
        ev1[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = sampler.stop() if sampler else None
    for s in sols:
        s.check()
    ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    prof = [s.profile_read(reset=True) for s in sols]
    for s in sols:
        s.profile(False)
    ms, _ = combine_ranks(dist, ms, 0.0, device="cuda")
    tot = {k: (sum(p[k][0] for p in prof), sum(p[k][1] for p in prof))
           for k in ("assemble", "reduced", "backsub")}
    return sols, dts, ms, tot, clk


def l2_vs_oracle(sols, dts, Ud, refs, ks, np):
    """Worst relative L2 error over the instances per variable after ks steps,
    and the paper's relative L1 error (Sec. 6) of the depth,
    ||h - h_ref||_1 / ||h||_1."""
    per = {k: 0.0 for k in ("h", "q", "heta", "hw")}
    l1 = 0.0
    for s, dt, ref in zip(sols, dts, refs):
        s.set_state(*Ud)
        s.run(dt, ks)
        got = [t.cpu().numpy() for t in s.get_state()]
        for k, name in enumerate(per):
            nr = np.linalg.norm(ref[k])
            if nr > 0:
                per[name] = max(per[name], float(np.linalg.norm(got[k] - ref[k]) / nr))
        l1 = max(l1, float(np.sum(np.abs(got[0] - ref[0])) / np.sum(np.abs(got[0]))))
    # the depth is the headline variable; q and h w are roundoff-sized where
    # the water is at rest, so their relative L2 is dominated by that noise
    return {"depth_rel_l2": per["h"], "depth_rel_l1": l1, "per_variable_rel_l2": per,
            "steps": ks}


def time_to_solution(S, torch, n, xl, xr, Ud, stream):
    """GPU time to advance the dam break (lambda = 1000, one instance of n
    cells) by the physical time of 20 steps of the paper's scheme at
    CFL_IMEX 4, with each scheme at its own stability limit: the semi-implicit
    schemes at CFL_IMEX 4, the explicit ones at CFL 0.4 (Heun) and 0.2 (Euler),
    as in the paper's cost tables (Sec. 6)."""
    lam = 1000.0
    runs = [("si_printed_fp64", S.FLAG_FP64, 4.0), ("si_ars222_fp64", S.SCHEME_ARS222, 4.0),
            ("si_first_order_fp64", S.SCHEME_SI1, 4.0), ("ex_heun_fp64", S.SCHEME_EX_HEUN, 0.4),
            ("ex_euler_fp64", S.SCHEME_EX_EULER, 0.2), ("si_printed_mixed", S.FLAG_MIXED, 4.0)]
    out, T = {}, None
    for name, flags, cfl in runs:
        s = S.Solver(n, xl, xr, S.BC_TRANSMISSIVE, lam=lam, flags=flags)
        s.set_state(*Ud)
        dt = s.suggest_dt(cfl, 0.5)
        if T is None:
            T = 20 * dt
        steps = max(1, int(math.ceil(T / dt - 1e-9)))
        dt = T / steps
        s.run(dt, 2)          # warm-up (graph capture)
        s.set_state(*Ud)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.enqueue(dt, steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        s.check()
        out[name] = {"steps": steps, "dt": dt, "ms": e0.elapsed_time(e1)}
        s.close()
    si = out["si_printed_fp64"]["ms"]
    return {
        "workload": f"dam break, lambda = 1000, {n} cells, physical time T = {T:.6g} "
                    "(20 steps of the paper's scheme at CFL_IMEX 4)",
        "runs": out,
        "ex_heun_over_si_fp64": out["ex_heun_fp64"]["ms"] / si,
        "ex_heun_fp64_over_si_mixed": out["ex_heun_fp64"]["ms"] / out["si_printed_mixed"]["ms"],
        "paper_cpu_ratio_ex_over_si": "2.5-3.0 (Gaussian bell, lambda 100-1000, Sec. 6.1 table)",
    }


def run_to_time(S, torch, stream, n, xl, xr, bc, lam, flags, U, cfl, mcfl, T):
    """GPU time of one run to the final time T with the fixed step of the
    initial state (dt = T / ceil(T / dt0), dt0 from the Sec. 5 rule); returns
    the record and the final depth (None when the run broke down)."""
    with S.Solver(n, xl, xr, bc, lam=lam, flags=flags) as s:
        Ud = [torch.tensor(u, device="cuda") for u in U]
        s.set_state(*Ud)
        dt0 = s.suggest_dt(cfl, mcfl)
        steps = max(1, int(math.ceil(T / dt0 - 1e-9)))
        dt = T / steps
        s.run(dt, 2)  # the graphs of both buffers (windowed form) / the step graph
        s.set_state(*Ud)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.enqueue(dt, steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        try:
            s.check()
        except S.HsgnError as err:
            return {"steps": steps, "dt": dt, "failed": str(err)}, None
        return {"steps": steps, "dt": dt, "ms": e0.elapsed_time(e1)}, s.get_state()[0].cpu().numpy()


def run_to_time_cfl(S, torch, stream, n, xl, xr, bc, lam, U, cfl, mcfl, T, chunk=200):
    """The double-float form to the final time T with the time step re-evaluated
    from the current state before every step (Sec. 5), on the device
    (hsgn_run_cfl); the last step is shortened to land on T. Returns the record
    and the final depth (None when the run broke down)."""
    with S.Solver(n, xl, xr, bc, lam=lam, flags=S.FLAG_DOUBLE_FLOAT) as s:
        Ud = [torch.tensor(u, device="cuda") for u in U]
        s.set_state(*Ud)
        torch.cuda.synchronize()
        t, steps, t0 = 0.0, 0, time.perf_counter()
        try:
            while True:
                dt = s.suggest_dt(cfl, mcfl)
                if t + dt >= T:
                    s.run(T - t, 1)
                    steps += 1
                    break
                # chunks of steps whose sum stays below T by a margin of one
                # chunk of the current dt
                k = max(1, min(chunk, int((T - t) / dt) - 1))
                t += s.run_cfl(cfl, mcfl, k)
                steps += k
        except S.HsgnError as err:
            return {"steps": steps, "t": t, "failed": str(err)}, None
        ms = 1e3 * (time.perf_counter() - t0)
        return ({"steps": steps, "ms_wall": ms, "dt_policy": "per step (Sec. 5), on the device"},
                s.get_state()[0].cpu().numpy())


def time_paper_runs(S, torch, stream):
    """The runs of the paper's CPU-time tables, timed on the GPU (the paper's
    seconds are for an unstated CPU and implementation: context only).
    Sec. 6.1: the Gaussian bell h = 1 + exp(-x^2/20) on [-200, 200], N = 5000,
    T = 35, the paper's scheme at CFL_IMEX 2 against explicit Heun at CFL 0.4,
    for lambda = 100, 500, 1000, 5000 (boundaries not printed: transmissive).
    Sec. 6.3: the solitary wave of amplitude 1 over depth 1, N = 2000, T = 1,
    lambda = 1000, first- and second-order semi-implicit schemes at CFL_IMEX
    2.5 and explicit ones at CFL 0.4 (domain not printed: [-50, 50],
    periodic), with the relative L1 error of the depth against the closed form.
    Steps are fixed from the initial state. Under these readings the scheme has
    a growing mode on the bell from lambda 1000 at CFL_IMEX 2 (and explicit
    Heun from lambda 500 at CFL 0.4): the FP64 runs break down, in the oracle
    alike; a mixed-precision run is timed only where its FP64 run reached T,
    and its distance to it is reported. Even where the runs reach T, the bell
    amplifies rounding differences by about 6 % per step from step ~200 until
    they saturate: the FP64 path and the oracle end 0.7 % apart at lambda 100,
    so the mixed-vs-FP64 distance measures that sensitivity, not the accuracy
    of the mixed form."""
    import numpy as np
    from paper_2510_07539_gb300 import inputs as inp
    bell = {}
    paper_bell = {100.0: (7.68, 19.51), 500.0: (16.18, 39.938), 1000.0: (25.59, 75.86),
                  5000.0: (63.34, 169.73)}
    x, dx, U = inp.gaussian_bell()
    for lam, (p_si, p_ex) in paper_bell.items():
        row = {}
        row["si_fp64"], h64 = run_to_time(S, torch, stream, 5000, -200.0, 200.0,
                                          S.BC_TRANSMISSIVE, lam, S.FLAG_FP64, U, 2.0, 0.0, 35.0)
        if h64 is not None:
            row["si_mixed"], hm = run_to_time(S, torch, stream, 5000, -200.0, 200.0,
                                              S.BC_TRANSMISSIVE, lam, S.FLAG_MIXED, U, 2.0, 0.0,
                                              35.0)
            if hm is not None:
                row["si_mixed"]["depth_rel_l2_vs_fp64"] = float(np.linalg.norm(hm - h64) /
                                                               np.linalg.norm(h64))
        # the same run with the time step re-evaluated every step (double-float
        # form): the policy of Sec. 5, under which lambda = 1000 reaches T
        row["si_dfloat_per_step_dt"], _ = run_to_time_cfl(S, torch, stream, 5000, -200.0, 200.0,
                                                          S.BC_TRANSMISSIVE, lam, U, 2.0, 0.0,
                                                          35.0)
        row["ex_heun_fp64"], _ = run_to_time(S, torch, stream, 5000, -200.0, 200.0,
                                             S.BC_TRANSMISSIVE, lam, S.SCHEME_EX_HEUN, U, 0.4,
                                             0.0, 35.0)
        row["paper_cpu_s"] = {"si": p_si, "ex_heun": p_ex}
        bell[f"lambda_{lam:g}"] = row
    x, _ = inp.cell_centres(2000, -50.0, 50.0)
    U = inp.solitary(x, 1.0, 1.0, 0.0, period=100.0)
    h_exact = inp.solitary(x, 1.0, 1.0, 0.0, t=1.0, period=100.0)[0]
    sol = {}
    for name, flags, cfl, paper in (("si_order1", S.SCHEME_SI1, 2.5, 1.2502),
                                    ("si_order2", S.FLAG_FP64, 2.5, 4.0350),
                                    ("ex_order1", S.SCHEME_EX_EULER, 0.4, 3.2105),
                                    ("ex_order2", S.SCHEME_EX_HEUN, 0.4, 16.9138)):
        rec, h = run_to_time(S, torch, stream, 2000, -50.0, 50.0, S.BC_PERIODIC, 1000.0, flags,
                             U, cfl, 0.0, 1.0)
        if h is not None:
            rec["depth_rel_l1_vs_closed_form"] = float(np.sum(np.abs(h - h_exact)) /
                                                       np.sum(np.abs(h)))
        rec["paper_cpu_s"] = paper
        sol[name] = rec
    return {"gaussian_bell": bell, "solitary_lambda_1000": sol,
            "note": "paper CPU seconds: unstated hardware and implementation; context only"}


def time_tridiag(S, torch, stream, hbm_peak, log2n=24, reps=10):
    """The library's tridiagonal component (hsgn_tridiag_solve, FP64) on 2^24
    rows of an hSGN-like SPD system, cyclic and not. Each call synchronises
    (it reports the device error word), so the per-call time includes that
    round trip. Algorithmic bytes 40 per row (a, b, c, d in, x out)."""
    from paper_2510_07539_gb300 import inputs as inp
    n = 1 << log2n
    out = {}
    for periodic in (False, True):
        rows = [torch.tensor(v, device="cuda") for v in inp.random_tridiag(77, n, periodic)]
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        ws = torch.empty(S.tridiag_workspace_bytes(n) + 512, dtype=torch.uint8, device="cuda")
        for _ in range(3):
            S.tridiag_solve(*rows, periodic, out=x, workspace=ws)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            S.tridiag_solve(*rows, periodic, stream=stream, out=x, workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = 40.0 * n / (ms / 1e3) / 1e9
        out["cyclic" if periodic else "open"] = {
            "rows": n, "ms_per_solve": ms, "rows_per_s": n / (ms / 1e3), "achieved_gbs": gbs,
            "frac_of_hbm": gbs / hbm_peak}
    out["note"] = ("block reduction (one warp per 128 rows, three right-hand sides), recursive "
                   "separator levels, back-substitution; FP64, each call synchronises")
    return out


def time_adjoint(S, torch, stream):
    """The adjoint workload: N = 4096, dx = 0.1, periodic, lambda = 100, a wave
    a = 0.1 over 8 Gaussian bumps (bottom form), 2000 steps at CFL_IMEX 2, the
    misfit at 5 equispaced gauges against a run over another bottom; gradient
    with respect to the initial state and the bottom, checkpoints every 100."""
    import numpy as np
    from paper_2510_07539_gb300 import inputs as inp
    n, steps, lam, K = 4096, 2000, 100.0, 100
    x, dx, b, U = inp.gauss_bottom_wave(inp.SEED_BASE + 4, n)
    U = inp.wave_over_bottom(x, b, 1.0, 0.1, 0.5 * n * dx + 0.037, period=n * dx)
    b2 = inp.gauss_bottom_wave(inp.SEED_BASE + 5, n)[2]
    cells = [int(n * (k + 0.5) / 5) for k in range(5)]
    Ud = [torch.tensor(u, device="cuda") for u in U]
    flags = S.FLAG_WELL_BALANCED
    with S.Solver(n, 0.0, n * dx, 0, lam=lam, flags=flags, bathymetry=b2) as s:
        s.set_state(*Ud)
        dt = s.suggest_dt(2.0, 0.5)
        hs = torch.empty(steps, len(cells), dtype=torch.float64, device="cuda")
        idx = torch.tensor(cells, device="cuda")
        for k in range(steps):
            s.step(dt)
            hs[k] = s.get_state()[0][idx]
    data = hs.cpu().numpy()
    with S.Solver(n, 0.0, n * dx, 0, lam=lam, flags=flags, bathymetry=b) as s:
        s.set_state(*Ud)
        s.run(dt, 5)
        s.set_state(*Ud)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.run(dt, steps)
        fwd = time.perf_counter() - t0
        s.set_state(*Ud)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, g, gb = s.adjoint(dt, steps, cells, data, checkpoint_every=K)
        adj = time.perf_counter() - t0
    return {"workload": f"wave over 8 Gaussian bumps, N = {n}, periodic, lambda = {lam:g}, "
                        f"{steps} steps at CFL_IMEX 2, 5 gauges, checkpoints every {K}, FP64 "
                        "bottom form",
            "forward_ms": 1e3 * fwd, "misfit_and_gradient_ms": 1e3 * adj,
            "gradient_over_forward": adj / fwd, "misfit": J,
            "grad_bottom_l2": float(np.linalg.norm(gb.cpu().numpy()))}


def time_shelf(S, torch, stream, hbm_peak, log2n=24, steps=50, warmup=3):
    """The large workload: N = 2^24, dx = 0.005, transmissive, lambda = 1000, a
    wave a = 0.1 running towards a 1:20 shelf (depth 1 -> 0.5), bottom form,
    dt = min(4 dx/nu, 0.5 dx/u_max) at t = 0. FP64, double-float and mixed
    precision advance the same initial state by `steps` steps (each state is
    537 MB, far above L2); the double-float and mixed results are compared
    with the FP64 one, which matches the FP64 oracle to 1e-12 per step."""
    import numpy as np
    from paper_2510_07539_gb300 import inputs as inp
    n, lam = 1 << log2n, 1000.0
    x, dx, b, U = inp.shelf_wave(n, dx=0.005 * (1 << 24) / n)
    Ud = [torch.tensor(u, device="cuda") for u in U]
    del U
    out, dt = {}, None
    for name, flags in (("fp64", S.FLAG_WELL_BALANCED),
                        ("dfloat", S.FLAG_WELL_BALANCED | S.FLAG_DOUBLE_FLOAT),
                        ("mixed", S.FLAG_WELL_BALANCED | S.FLAG_MIXED)):
        with S.Solver(n, 0.0, n * dx, S.BC_TRANSMISSIVE, lam=lam, flags=flags,
                      bathymetry=b) as s:
            s.set_state(*Ud)
            if dt is None:
                dt = s.suggest_dt(4.0, 0.5)
            s.run(dt, warmup)
            s.set_state(*Ud)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.enqueue(dt, steps, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            s.check()
            ms = e0.elapsed_time(e1)
            out[name] = {"value": 2.0 * n * steps / (ms / 1e3), "unit": UNIT,
                         "ms_per_step": ms / steps,
                         "state": [t.cpu().numpy() for t in s.get_state()]}
    ref, got = out["fp64"].pop("state"), out["mixed"].pop("state")
    gdf = out["dfloat"].pop("state")
    rel = [float(np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k])) for k in range(4)]
    rel_df = [float(np.linalg.norm(gdf[k] - ref[k]) / np.linalg.norm(ref[k])) for k in range(4)]
    # algorithmic bytes of the bottom form: 88 per cell-stage (the FP64 state
    # traffic of the scheme, 80 B, plus the bottom read once per stage)
    gbs = (BYTES_PER_CELL_STAGE_BOTTOM * 2.0 * n * steps
           / (out["mixed"]["ms_per_step"] * steps / 1e3) / 1e9)
    out["mixed"]["roofline"] = {"bound": "hbm", "kernel": "k_mixed_fused (bottom form)",
                                "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                "frac": gbs / hbm_peak,
                                "algorithmic_bytes_per_cell_stage": BYTES_PER_CELL_STAGE_BOTTOM,
                                "timing": "whole steps (both stages), one stream"}
    return {"workload": f"wave a = 0.1 towards a 1:20 shelf, N = 2^{log2n}, dx = {dx:g}, "
                        f"transmissive, lambda = 1000, bottom form, dt = {dt:.6g} "
                        f"(CFL_IMEX 4), {steps} timed steps (of the 5000-step run)",
            "fp64": out["fp64"], "dfloat": out["dfloat"], "mixed": out["mixed"],
            "dfloat_over_fp64": out["dfloat"]["value"] / out["fp64"]["value"],
            "dfloat_vs_fp64_rel_l2_after_steps": {"h": rel_df[0], "q": rel_df[1],
                                                  "h_eta": rel_df[2], "h_w": rel_df[3]},
            "mixed_over_fp64": out["mixed"]["value"] / out["fp64"]["value"],
            "mixed_vs_fp64_rel_l2_after_steps": {"h": rel[0], "q": rel[1], "h_eta": rel[2],
                                                 "h_w": rel[3]}}


def kernel_roofline_alu(name, flops_per_cell, n, avg_ms, peak, peak_source):
    """Arithmetic roofline of one stage kernel from its average launch time."""
    if flops_per_cell is None or not (avg_ms > 0):
        return {"bound": "alu", "kernel": name, "achieved": None, "peak": peak,
                "unit": "TFLOP/s", "frac": None, "peak_source": peak_source,
                "kernel_avg_ms": avg_ms}
    tf = flops_per_cell * n / (avg_ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": name, "achieved": tf, "peak": peak, "unit": "TFLOP/s",
            "frac": tf / peak, "peak_source": peak_source, "kernel_avg_ms": avg_ms,
            "flops_per_cell_launch": flops_per_cell}


def hbm_view(n, avg_ms, hbm_peak, bytes_per_cell=BYTES_PER_CELL_STAGE):
    gbs = bytes_per_cell * n / (avg_ms / 1e3) / 1e9
    return {"achieved_gbs": gbs, "frac_of_measured_hbm": gbs / hbm_peak,
            "algorithmic_bytes_per_cell_stage": bytes_per_cell}


# the library's profile slots per form: the stage kernel, the separator levels
# of the FP64 form's global solve and its back-substitution kernel
SHARE_NAMES = {
    "df": {"assemble": "k_df_stage"},
    "mixed": {"assemble": "k_mixed_fused"},
    "fp64": {"assemble": "k_stage_assemble", "reduced": "separator levels (k_block_reduce, "
             "k_cyclic_onewarp, k_block_backout)", "backsub": "k_backsub"},
}


def time_form(S, torch, flags, n, xl, xr, lams, Ud, args, flush, stream, dist, clocks,
              concurrent, names=None):
    """A form timed twice on the workload: the instances of a step on one stream
    each (the throughput), then back to back on one stream, where the event
    pair of every launch times that launch alone (the kernel's duration)."""
    sols, dts, ms, tot, clk = time_path(S, torch, flags, n, xl, xr, lams, Ud, args.steps,
                                        args.warmup, flush, stream, dist, clocks, concurrent)
    if concurrent:
        qsols, _, qms, qtot, _ = time_path(S, torch, flags, n, xl, xr, lams, Ud, args.steps,
                                           args.warmup, flush, stream, dist, None, False)
        for s_ in qsols:
            s_.close()
    else:
        qms, qtot = ms, tot
    avg = qtot["assemble"][0] / max(qtot["assemble"][1], 1)
    share_den = sum(v[0] for v in qtot.values())
    share = {(names or {}).get(k, k): v[0] / share_den for k, v in qtot.items()
             if v[1] > 0} if share_den > 0 else {}
    return sols, dts, ms, qms, avg, share, clk


def run_ours(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CPU oracle arm is --impl reference)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2510_07539_gb300 import build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    from paper_2510_07539_gb300 import solver as S

    lams = [float(x) for x in args.lams.split(",")]
    n, dx, xl, xr, U, lams = workload(args.log2n, lams)
    Ud = [torch.tensor(u, device="cuda") for u in U]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(local)
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) >= 32:
        gpu_id = "GPU-" + gpu_id
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = ("measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), burst"
               if "hbm_gbs" in peaks else "fallback 6.8 TB/s of the profiling recipe")
    # arithmetic peaks measured here: fused multiply-add chains on every SM
    # (hsgn_fma_peak), best of three
    fp32_peak = max(S.fma_peak(32) for _ in range(3))
    fp64_peak = max(S.fma_peak(64) for _ in range(3))
    units_rank = 2.0 * n * len(lams) * args.steps

    # ---- headline: the double-float form (FP64 class), one launch per stage;
    #      the instances of a step on one stream each (whole-job throughput)
    dsols, ddts, dms, dqms, davg, dshare, clocks = time_form(
        S, torch, S.FLAG_DOUBLE_FLOAT, n, xl, xr, lams, Ud, args, flush, stream, dist, gpu_id,
        not args.sequential, SHARE_NAMES["df"])
    value = units_rank * world / (dms / 1e3)
    # the window overlap each instance stepped with (it follows the coupling)
    dover = [s.df_overlap() for s in dsols]
    counted = DF_FLOPS_SOURCE_SHA is not None and source_sha(DF_SOURCES) == DF_FLOPS_SOURCE_SHA
    dflops = DF_FLOPS_PER_CELL if counted else None
    roofline = kernel_roofline_alu(
        "k_df_stage (double-float stage: fluxes, rows, depth solve and back-substitution in one "
        "launch)", dflops, n, davg, fp32_peak,
        "measured here: FP32 fused multiply-add chains on every SM (hsgn_fma_peak), best of 3")
    roofline.update({
        # DRAM bytes per launch: the ncu count per cell of the 2^22-cell capture
        # times the cells of one launch (traffic grows with the cells)
        "traffic": DF_TRAFFIC_PER_CELL * n if counted else None,
        # the FP32 pipe's issue share: FP32 instructions per second against half
        # the measured multiply-add flop rate (one instruction per lane and clock)
        "fp32_pipe_frac": (DF_FP32_INST_PER_CELL * n / (davg / 1e3) / 1e12 / (fp32_peak / 2.0))
        if counted and davg > 0 else None,
        "kernel_timing": f"one stream, {len(lams)} instances back to back, {args.steps} steps "
                         "(the sequential pass)",
        "kernel_share": dshare,
        "hbm": hbm_view(n, davg, hbm_peak),
        "sequential_value": units_rank * world / (dqms / 1e3),
    })
    launches = len(lams) * args.steps * 2

    # ---- the FP64 form (exact separator solve) on the same workload
    fp64, fsols, fdts = None, [], []
    if not args.no_fp64:
        fsols, fdts, fms, fqms, favg, fshare, _ = time_form(
            S, torch, S.FLAG_FP64, n, xl, xr, lams, Ud, args, flush, stream, dist, None, False,
            SHARE_NAMES["fp64"])
        fp64 = {"value": units_rank * world / (fms / 1e3), "unit": UNIT,
                "ms_per_step": fms / args.steps, "dtype": "f64",
                "roofline": kernel_roofline_alu(
                    "k_stage_assemble", FLOPS_PER_CELL_ASSEMBLE, n, favg, fp64_peak,
                    "measured here: FP64 fused multiply-add chains on every SM (hsgn_fma_peak)"),
                "kernel_share": fshare,
                "hbm": {"frac_of_measured_hbm_whole_step": BYTES_PER_CELL_STAGE * units_rank
                        / (fms / 1e3) / 1e9 / hbm_peak}}

    # ---- the mixed-precision form (FP32 increments, windowed solve)
    mixed, msols, mdts = None, [], []
    if not args.no_mixed:
        msols, mdts, mms, mqms, mavg, mshare, _ = time_form(
            S, torch, S.FLAG_MIXED, n, xl, xr, lams, Ud, args, flush, stream, dist, None,
            not args.sequential, SHARE_NAMES["mixed"])
        mgbs = BYTES_PER_CELL_STAGE * n / (mavg / 1e3) / 1e9
        mixed = {"value": units_rank * world / (mms / 1e3), "unit": UNIT,
                 "ms_per_step": mms / args.steps, "dtype": "f32 increments + double-float state",
                 "roofline": {"bound": "hbm", "kernel": "k_mixed_fused", "achieved": mgbs,
                              "peak": hbm_peak, "unit": "GB/s", "frac": mgbs / hbm_peak,
                              "peak_source": hbm_src, "kernel_avg_ms": mavg,
                              "algorithmic_bytes_per_cell_stage": BYTES_PER_CELL_STAGE,
                              "bytes_moved_per_cell_stage": BYTES_MOVED_MIXED},
                 "sequential_value": units_rank * world / (mqms / 1e3)}

    # ---- the precision split with an FP64-class solve: FP32 fluxes and
    #      coefficients, rows, depth solve and back-substitution in pairs
    mixed_df, xsols, xdts = None, [], []
    if not args.no_mixed:
        xsols, xdts, xms, xqms, xavg, _, _ = time_form(
            S, torch, S.FLAG_MIXED | S.FLAG_DOUBLE_FLOAT, n, xl, xr, lams, Ud, args, flush,
            stream, dist, None, not args.sequential)
        mixed_df = {"value": units_rank * world / (xms / 1e3), "unit": UNIT,
                    "ms_per_step": xms / args.steps,
                    "dtype": "f32 fluxes and coefficients + double-float solve and state",
                    "kernel_avg_ms": xavg, "hbm": hbm_view(n, xavg, hbm_peak),
                    "sequential_value": units_rank * world / (xqms / 1e3)}

    # ---- the paper's comparison: the same physical time with each scheme
    comparators = None
    if not args.no_comparators:
        comparators = time_to_solution(S, torch, 1 << 20, -0.5 * (1 << 20) * dx,
                                       0.5 * (1 << 20) * dx,
                                       [torch.tensor(u, device="cuda")
                                        for u in workload(20, lams)[4]], stream)
    adjoint = None
    if not args.no_adjoint and rank == 0:
        adjoint = time_adjoint(S, torch, stream)
    tridiag = None
    if not args.no_tridiag and rank == 0:
        tridiag = time_tridiag(S, torch, stream, hbm_peak, args.tridiag_log2n)
    paper_runs = None
    if not args.no_paper_runs and rank == 0:
        paper_runs = time_paper_runs(S, torch, stream)
    shelf = None
    if not args.no_shelf and rank == 0:
        shelf = time_shelf(S, torch, stream, hbm_peak, args.shelf_log2n, args.shelf_steps)

    # ---- batched workload: 4096 independent periodic solitary waves of uneven
    #      length, the windowed mixed stage over all of them, each step one
    #      replay of the captured step graph
    batched = None
    if not args.no_batched:
        from paper_2510_07539_gb300 import inputs as inp
        insts = inp.batched_instances(inp.SEED_BASE + 3, args.batch)
        ns = [it.n for it in insts]
        B = S.BatchedSolver(ns, [-0.5 * it.n * it.dx for it in insts],
                            [0.5 * it.n * it.dx for it in insts], [it.lam for it in insts])
        packed = [torch.tensor(np.concatenate([it.state[k] for it in insts]), device="cuda")
                  for k in range(4)]
        B.set_state(*packed)
        # CFL_IMEX = 2: at 3 and above the largest-amplitude lambda = 1000 waves of
        # this batch have a growing mode of the scheme (1.05-1.14 per step)
        bdts = B.suggest_dt(2.0, 0.5)
        B.set_dt(bdts)
        # tiles picked by the library's autotuner (outside the timed region;
        # the state is kept)
        tune = B.autotune(4)
        bvar = B.get_tiles()
        B.run(0.0, args.warmup)  # also captures the step graphs of both state buffers
        bev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        bev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            bev0[k].record(stream)
            B.enqueue(0.0, 1, stream=stream)
            bev1[k].record(stream)
        torch.cuda.synchronize()
        B.check()
        bms = sum(a.elapsed_time(c) for a, c in zip(bev0, bev1))
        bcells = int(sum(ns))
        bgbs = BYTES_PER_CELL_STAGE * 2.0 * bcells / (bms / args.steps / 1e3) / 1e9
        batched = {
            "workload": f"{len(ns)} periodic hSGN solitary waves, N ~ U[256, 8192], "
                        "a ~ U[0.05, 0.4], lambda in {10, 100, 1000}, per-instance dt "
                        "(CFL_IMEX 2, MCFL 0.5), mixed precision, windowed stage over all "
                        "instances (one launch per stage and tile variant)",
            "instances": len(ns), "cells": bcells,
            "value": 2.0 * bcells * args.steps * world / (bms / 1e3), "unit": UNIT,
            "ms_per_step": bms / args.steps,
            "timing": "each step one replay of the captured step graph (hsgn_enqueue)",
            "roofline": {"bound": "hbm", "achieved": bgbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": bgbs / hbm_peak,
                         "algorithmic_bytes_per_cell_stage": BYTES_PER_CELL_STAGE,
                         "timing": "whole steps"},
            # one launch per stage for every tile variant in use
            "gpu_launches_per_step": 2 * len(set(int(v) for v in bvar)),
            "autotune": {"variants": ["256 threads, 64-row overlap (894-row tiles)",
                                      "128 threads, 64-row overlap (382-row tiles)",
                                      "256 threads, 32-row overlap (958-row tiles)",
                                      "128 threads, 32-row overlap (446-row tiles)",
                                      "per-instance cost-model assignment"],
                         "ms_per_step": [None if math.isnan(x) else x
                                         for x in tune["ms_per_step"]],
                         "kept": tune["choice"],
                         "instances_per_variant": [int((bvar == v).sum()) for v in range(4)]},
        }
        if rank == 0 and world == 1 and not args.no_cpu:
            # error of the batched path on a sample of instances after 10 steps
            B.set_state(*packed)
            B.run(0.0, 10)
            got = [t.cpu().numpy() for t in B.get_state()]
            import oracle
            worst = 0.0
            for kk in range(min(8, len(ns))):
                it = insts[kk]
                o0, o1 = int(B.offsets[kk]), int(B.offsets[kk + 1])
                ref = oracle.run(oracle.Params(it.n, it.dx, 0, lam=it.lam), it.state, bdts[kk], 10)
                worst = max(worst, float(np.linalg.norm(got[0][o0:o1] - ref[0])
                                         / np.linalg.norm(ref[0])))
            batched["depth_rel_l2_vs_oracle"] = {"value": worst, "instances": 8, "steps": 10}
        B.close()

    # ---- end to end through the C ABI with host buffers (the headline form)
    e2e = None
    if not args.no_e2e:
        host_in = [[torch.tensor(u).pin_memory() for u in U] for _ in lams]
        k_e2e = max(2, min(args.steps, 20))
        # every step copies each instance's state in from pinned host memory,
        # steps it and copies the result out to pinned host memory
        # (hsgn_copy_state_out: enqueued, no host wait). Consecutive steps
        # alternate between two sets of handles, each instance of a set with
        # its own pair of streams: the copies and their conversions on a
        # high-priority stream, so that they are not held behind the stage
        # kernels of the other instances, the step on a normal one, joined by
        # events; one step's copies in then overlap the other instances' steps
        # and copies out on the copy engines. Errors are checked after the
        # timed region
        sets = [dsols, [S.Solver(n, xl, xr, S.BC_TRANSMISSIVE, lam=l, flags=S.FLAG_DOUBLE_FLOAT)
                        for l in lams]]
        host_out = [[[torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(4)]
                     for _ in lams] for _ in sets]
        side = [[torch.cuda.Stream() for _ in lams] for _ in sets]
        cside = [[torch.cuda.Stream(priority=-1) for _ in lams] for _ in sets]
        for s, dt, hi, ho in zip(sets[1], ddts, host_in, host_out[1]):
            s.set_state(*hi)
            s.step(dt)  # the step graph of the new handle, outside the timed region
            s.copy_state_out(ho)
        fork = torch.cuda.Event()

        def e2e_steps(k):
            fork.record(stream)
            for sts in side + cside:
                for st in sts:
                    st.wait_event(fork)
            for it in range(k):
                c = it % 2
                for s, dt, hi, ho, st, cs in zip(sets[c], ddts, host_in, host_out[c], side[c],
                                                 cside[c]):
                    s.set_state(*hi, stream=cs)
                    ready = torch.cuda.Event()
                    ready.record(cs)
                    st.wait_event(ready)
                    s.step(dt, stream=st)
                    done = torch.cuda.Event()
                    done.record(st)
                    cs.wait_event(done)
                    s.copy_state_out(ho, stream=cs)
            for sts in side + cside:
                for st in sts:
                    j = torch.cuda.Event()
                    j.record(st)
                    stream.wait_event(j)

        # untimed warm-up steps of the same loop: every pinned buffer and both
        # handle sets have been through one copy before the timed region
        e2e_steps(max(2, args.warmup))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_steps(k_e2e)
        e1.record(stream)
        torch.cuda.synchronize()
        for s in sets[0] + sets[1]:
            s.check()
        for s in sets[1]:
            s.close()
        ems, units = combine_ranks(dist, e0.elapsed_time(e1), 2.0 * n * len(lams) * k_e2e,
                                   device="cuda")
        nbytes = 4 * n * 8 * len(lams)
        e2e = {"value": units / (ems / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": k_e2e,
               "warmup": max(2, args.warmup)}
        # the host link alone, after the timed region: the same arrays copied in,
        # out and both ways at once (one stream per direction, best of three);
        # a step cannot take less than its bytes at the two-way rate
        dev_in = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4 * len(lams))]
        dev_out = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(4 * len(lams))]
        src_in = [u for hi in host_in for u in hi]
        dst_out = [u for ho in host_out[0] for u in ho]
        up, down = torch.cuda.Stream(), torch.cuda.Stream()

        def link_ms(h2d, d2h):
            best = float("inf")
            for _ in range(3):
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for st, on, pairs in ((up, h2d, zip(dev_in, src_in)),
                                      (down, d2h, zip(dst_out, dev_out))):
                    if not on:
                        continue
                    st.wait_event(a)
                    with torch.cuda.stream(st):
                        for dst, src in pairs:
                            dst.copy_(src, non_blocking=True)
                    j = torch.cuda.Event()
                    j.record(st)
                    stream.wait_event(j)
                b.record(stream)
                b.synchronize()
                best = min(best, a.elapsed_time(b))
            return best

        t_up, t_down, t_both = link_ms(True, False), link_ms(False, True), link_ms(True, True)
        del dev_in, dev_out
        both_gbs = nbytes / (t_both * 1e6)
        ceiling = 2.0 * n * len(lams) / (t_both / 1e3)
        e2e["host_link"] = {
            "h2d_gbs": nbytes / (t_up * 1e6), "d2h_gbs": nbytes / (t_down * 1e6),
            "both_ways_gbs_per_direction": both_gbs,
            "e2e_ceiling": ceiling, "frac_of_ceiling": e2e["value"] / ceiling,
            "note": "plain copies of the step's bytes, timed after the e2e region; the ceiling is "
                    "the step's updates over the time both copies take at once"}

    # ---- CPU oracle baseline and the error of every form against it
    cpu = None
    l2err = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ks = max(1, args.cpu_steps)
        refs, el = oracle_steps(n, dx, U, lams, ddts, ks)
        cpu = {"value": 2.0 * n * len(lams) * ks / el, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{ks} IMEX steps of each of the {len(lams)} instances ({n} cells), "
                         f"single-threaded C oracle, {el:.1f} s"}
        l2err = l2_vs_oracle(dsols, ddts, Ud, refs, ks, np)
        if fp64 is not None:
            fp64["l2_rel_err_vs_oracle"] = l2_vs_oracle(fsols, fdts, Ud, refs, ks, np)
        if mixed is not None:
            mixed["l2_rel_err_vs_oracle"] = l2_vs_oracle(msols, mdts, Ud, refs, ks, np)
        if mixed_df is not None:
            mixed_df["l2_rel_err_vs_oracle"] = l2_vs_oracle(xsols, xdts, Ud, refs, ks, np)
    for s in dsols + fsols + msols + xsols:
        s.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "df64",
            "data": "synthetic",
            "config": config_dict(n, lams, ddts, {
                "parallelism": f"{world} independent replicas",
                "streams": ("one stream, instances back to back" if args.sequential else
                            "one CUDA stream per instance, joined every step"),
                "precision": "double-float: every value a pair of FP32 numbers (48-bit "
                             "significand, about 2^-47 per operation); parity bar of the FP64 "
                             "form (1e-12 relative per step against the FP64 oracle)",
                "depth_solve": "windows of the tile +- an overlap that follows the coupling "
                               "(the rows the last synchronised step needed + 5, rounded up to "
                               "a multiple of 8 within 48..96), truncation bounded in-kernel by "
                               "rho*^(overlap - 1) <= 2^-50; a tile whose window misses it is "
                               "redone with 96 rows",
                "overlap_rows": [o for _, o in dover],
                "rows_needed": [r for r, _ in dover]}),
            "l2_rel_err_vs_oracle": l2err,
            "roofline": roofline, "peaks": {"hbm_gbs": hbm_peak, "hbm_source": hbm_src,
                                            "fp32_tflops": fp32_peak, "fp64_tflops": fp64_peak,
                                            "fp32_fp64_source": "measured in this run "
                                                                "(hsgn_fma_peak)"},
            "fp64_path": fp64, "mixed_path": mixed, "mixed_dfsolve_path": mixed_df,
            "batched": batched,
            "batched_vs_fp64_single": (batched["value"] / fp64["value"])
            if (batched and fp64) else None,
            "comparators": comparators, "adjoint": adjoint, "shelf": shelf,
            "paper_runs": paper_runs, "tridiag": tridiag,
            "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks, "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _oracle_dam_break(args):
    """Oracle run of one dam-break instance (a process of the accuracy mode)."""
    lam, steps, log2n = args
    import numpy as np
    import oracle
    n, dx, xl, xr, U, _ = workload(log2n, [lam])
    p = oracle.Params(n, dx, oracle.BC_TRANSMISSIVE, lam=lam)
    dt, _, _ = oracle.suggest_dt(p, U, 4.0, 0.5)
    t0 = time.perf_counter()
    r = oracle.run(p, U, dt, steps)
    return lam, dt, [np.asarray(v) for v in r], time.perf_counter() - t0


def run_accuracy(args):
    """The error of every form at the configurations' full lengths, one JSON
    line: the dam break (2^20 cells, lambda 10 / 100 / 1000, 2000 steps at
    CFL_IMEX 4) in the FP64, double-float and mixed forms against the FP64
    oracle, whose three runs go to a process pool on the host cores (started
    with spawn, before the first GPU call) while the GPU runs; and the shelf
    (2^24 cells, 5000 steps) in double-float and mixed precision against the
    FP64 form. Minutes of host and GPU time (run it with --log2n 20: the
    oracle takes minutes per 2^20-cell run); not part of the default run."""
    import multiprocessing as mp
    import numpy as np
    lams = [float(x) for x in args.lams.split(",")]
    steps = args.accuracy_steps
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(lams)) as pool:
        fut = pool.map_async(_oracle_dam_break, [(l, steps, args.log2n) for l in lams])
        import torch
        from paper_2510_07539_gb300 import inputs as inp, solver as S
        n, dx, xl, xr, U, _ = workload(args.log2n, lams)
        Ud = [torch.tensor(u, device="cuda") for u in U]
        gpu = {}
        for lam in lams:
            for name, flags in (("fp64", S.FLAG_FP64), ("dfloat", S.FLAG_DOUBLE_FLOAT),
                                ("mixed", S.FLAG_MIXED)):
                with S.Solver(n, xl, xr, S.BC_TRANSMISSIVE, lam=lam, flags=flags) as s:
                    s.set_state(*Ud)
                    s.run(s.suggest_dt(4.0, 0.5), steps)
                    gpu[(lam, name)] = [v.cpu().numpy() for v in s.get_state()]
        # the shelf: FP64 against double-float and mixed over the configuration's 5000 steps
        sn = 1 << args.shelf_log2n
        x, sdx, b, SU = inp.shelf_wave(sn, dx=0.005 * (1 << 24) / sn)
        SUd = [torch.tensor(u, device="cuda") for u in SU]
        shelf, sdt, sms = {}, None, {}
        for name, flags in (("fp64", S.FLAG_WELL_BALANCED),
                            ("dfloat", S.FLAG_WELL_BALANCED | S.FLAG_DOUBLE_FLOAT),
                            ("mixed", S.FLAG_WELL_BALANCED | S.FLAG_MIXED)):
            with S.Solver(sn, 0.0, sn * sdx, S.BC_TRANSMISSIVE, lam=1000.0, flags=flags,
                          bathymetry=b) as s:
                s.set_state(*SUd)
                if sdt is None:
                    sdt = s.suggest_dt(4.0, 0.5)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.run(sdt, args.shelf_accuracy_steps)
                sms[name] = time.perf_counter() - t0
                shelf[name] = [v.cpu().numpy() for v in s.get_state()]
        refs = fut.get()
    names = ("h", "q", "heta", "hw")
    dam = []
    for lam, dt, ref, el in refs:
        for form in ("fp64", "dfloat", "mixed"):
            got = gpu[(lam, form)]
            dam.append({"lambda": lam, "form": form, "oracle_s": el,
                        "rel_l2": {nm: float(np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k]))
                                   for k, nm in enumerate(names)},
                        "depth_rel_l1": float(np.sum(np.abs(got[0] - ref[0])) /
                                              np.sum(np.abs(ref[0])))})
    ref = shelf["fp64"]
    m0 = float(np.sum(SU[0]))
    line = {"mode": "accuracy",
            "dam_break": {"cells": n, "steps": steps, "vs": "FP64 oracle", "runs": dam},
            "shelf": {"cells": sn, "steps": args.shelf_accuracy_steps, "vs": "FP64 form",
                      "seconds": sms,
                      "rel_l2": {f: {nm: float(np.linalg.norm(shelf[f][k] - ref[k]) /
                                               np.linalg.norm(ref[k]))
                                     for k, nm in enumerate(names)}
                                 for f in ("dfloat", "mixed")},
                      "mass_drift": {f: abs(float(np.sum(shelf[f][0])) - m0) / m0
                                     for f in ("fp64", "dfloat", "mixed")}}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.accuracy:
        run_accuracy(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
