"""Benchmark: cell-integrations/s of the per-cell stiff thermochemistry integrator.

One step = one integrate call over the whole synthetic batch of the workload (all
cells advanced over the full dt): rates, Jacobian, LU, solve and adaptive sub-steps
for every cell.  Default workload: the combustion-like network (10 species,
2 elements, 30 reversible reactions, temperature equation), 65,536 cells, dt = 1e-6 s.

Printed JSON line (rank 0): value = the chosen form's cells/s (TR-BDF2 sub-steps,
FP32-LU simplified Newton, persistent longest-first queue replayed from a CUDA graph,
the queue ordered by the next interval's Newton counts), with the plain FP64 forms
(backward Euler and TR-BDF2) alongside under "forms"; "e2e" = the same metric through
kt_state upload / integrate / download with pinned host buffers; "roofline" =
algorithmic FLOP/s of the integrate kernel against the FP64 pipe peak measured in the
run; "cpu_baseline" = the FP64 oracle on a bounded sample on the host.
--workload 3 / 5 with --ncells run the ISM and the 64-species networks.

--impl reference times the FP64 CPU oracle itself on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2504_04941_gb300 import inputs as I  # noqa: E402
from paper_2504_04941_gb300 import shard  # noqa: E402

METRIC = ("cell-integrations/s over fixed Δt at 1e-6 rel error vs FP64 oracle; "
          "plain vs chosen form")
UNIT = "cell-integrations/s"
# Nominal pipes of GB300 (context; the roofline uses the peaks measured in the run by
# kt_fma_peak): FP64 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz = 1.26 TFLOP/s,
# FP32 152 x 128 FMA/clk x 2 x 2.07 GHz = 80.5 TFLOP/s.
FP64_NOMINAL_TFLOPS = 1.25
FP32_NOMINAL_TFLOPS = 80.5
# DRAM bytes (read + write) per cell of one launch of the chosen-form lane kernel on the
# combustion network, from an ncu capture of the kernel built from the sources whose
# hash is the key (a different build reports traffic null until it is captured again).
LANE_TRAFFIC_BYTES_PER_CELL = {
    # lean lane kernel, full interval, 8-warp blocks: 8,111,360 B read + 345,856 B written
    # (captured on sources f60b55e70311ee05; this key adds comments in include/kt.h only)
    "b6a2b16ed131dd4b": (8111360 + 345856) / 65536,
}


def kernel_source_hash() -> str:
    """sha256 (16 hex digits) of the CUDA sources and the C header the library is built from."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2504_04941_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(fn.encode() + b"\0" + f.read())
    with open(os.path.join(ROOT, "include", "kt.h"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------ work counts


def _lu_flops(N: int) -> int:
    f = 0
    for j in range(N):
        for i in range(N):
            f += 2 * min(i, j)
        f += N - 1 - j           # scale the L column by the inverse pivot
    return f


def flops_per_newton(net: I.Network, form: int):
    """(fp64 flops, fp32 flops per factorisation, transcendentals) of one Newton
    iteration, counting each multiply and add once (an FMA as 2)."""
    N = net.n
    rates = fp64 = fp32 = 0
    for ins, outs in zip(net.reac_in, net.reac_out):
        nin, nout = len(ins), len(outs)
        r64 = (7 if net.energy else 0) + nin + (nin + nout) + (2 if net.energy else 0)
        jac = nin * (nin + (nin + nout) + (2 if net.energy else 0))
        if net.energy:
            jac += (nin + 2) + (nin + nout) + 2
        fp64 += r64
        if form == 0:
            fp64 += jac
        else:
            fp32 += jac
        rates += 1 if net.energy else 0
    lu, solve = _lu_flops(N), 2 * N * N - N
    if form == 0:
        fp64 += N + lu + solve + 3 * N + 3 * N
    else:
        fp64 += 3 * N + 3 * N
        fp32 += 2 * N * N + lu + solve
    return fp64, fp32, rates


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
                power.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle legs


def oracle_time(wl: I.Workload, ncells: int, seed_offset: int = 0, scheme: int = 1):
    """Time the FP64 oracle (as it stands) on the first ``ncells`` cells of a fresh
    draw of the workload; returns (cells/s, threads, wall seconds)."""
    from oracle import oracle
    sub = I.workload(wl.wid, ncells, seed=I.SEED_BASE + wl.wid + seed_offset).cells
    net = oracle.OracleNetwork(wl.network)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = net.integrate(sub, wl.tol.dt, oracle.options(wl.tol, scheme=scheme), threads)
    wall = time.perf_counter() - t0
    assert np.all(r["status"] <= 1)
    return ncells / wall, threads, wall


def hbm_peak_gbs() -> tuple:
    """(GB/s, source) of the measured copy bandwidth of the GB300s, else the
    earlier single measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback (one earlier GB300 measurement)"


SCHEME_NAMES = {0: "be_step_doubling", 1: "trbdf2"}


def oracle_on(network: I.Network, cells: I.Cells, tol: I.Tolerances, scheme: int = 0,
              threads: int = 0):
    """The FP64 oracle (as it stands) on these cells with all host cores (or `threads`);
    returns (result dict, threads, wall seconds)."""
    from oracle import oracle
    net = oracle.OracleNetwork(network)
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    r = net.integrate(cells, tol.dt, oracle.options(tol, scheme=scheme), threads)
    return r, threads, time.perf_counter() - t0


def accuracy(gpu: dict, ora: dict, network: I.Network, y0: np.ndarray) -> dict:
    """Errors of a GPU result against the oracle's on the same cells: the largest
    relative error per species above 1e-20 (over all cells, and over the cells whose
    accepted sub-step count equals the oracle's: the step-doubling accept test is a
    discontinuous function of rounding), the largest relative error of T, and the
    largest relative change of the element totals."""
    yg, yo = np.asarray(gpu["y"], float), np.asarray(ora["y"], float)
    Tg, To = np.asarray(gpu["T"], float), np.asarray(ora["T"], float)
    big = yo > 1e-20
    rel = np.where(big, np.abs(yg - yo) / np.where(big, yo, 1.0), 0.0)
    same = np.asarray(gpu["nsub"]) == np.asarray(ora["nsub"])
    y0c = np.maximum(y0, 0.0)
    b0 = network.counts.T @ y0c
    scale = np.abs(network.counts.T) @ y0c
    cons = np.abs(network.counts.T @ yg - b0) / np.where(scale > 0, scale, 1.0)
    return {"cells": int(yo.shape[1]),
            "max_rel_err_y": float(rel.max(initial=0.0)),
            "max_rel_err_y_same_substeps": float(rel[:, same].max(initial=0.0)),
            "cells_with_other_substep_count": int((~same).sum()),
            "max_rel_err_T": float((np.abs(Tg - To) / np.abs(To)).max(initial=0.0)),
            "max_conservation_err": float(cons.max(initial=0.0)),
            "status_equal": bool(np.array_equal(np.asarray(gpu["status"]), np.asarray(ora["status"])))}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = I.workload(args.workload, 1)
    n = args.ref_cells
    times = []
    for s in range(args.warmup + args.steps):
        v, threads, wall = oracle_time(wl, n, seed_offset=0)
        if s >= args.warmup:
            times.append(wall)
    value = n * len(times) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            # the GPU arm's workload; each step times a bounded sample of its cells
            "config": dict(config_of(args, wl, args.ncells or I.FULL_CELLS[args.workload]),
                           timed_cells_per_step=n),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "scheme": SCHEME_NAMES[1],
                             "sample": f"{n} cells of the {wl.name} workload per step (same "
                                       f"network, tolerances, dt and scheme), pthreads over cells"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(args, wl: I.Workload, ncells: int) -> dict:
    t = wl.tol
    return {"workload": f"{wl.name}: {wl.network.ns} species / {wl.network.ne} elements / "
                        f"{wl.network.nr} directed reactions"
                        f"{' + temperature' if wl.network.energy else ''}, {ncells} cells, "
                        f"dt={t.dt:g} s, rtol={t.rtol:g}, atol={t.atol:g}",
            "ncells": ncells, "dt": t.dt, "rtol": t.rtol, "atol": t.atol,
            "scheme": "TR-BDF2 sub-steps (the chosen form and the reference arm); "
                      "the plain form is also timed with backward-Euler step doubling",
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"cells sharded over {args.gpus} GPU(s), no collective"}


# ------------------------------------------------------------------ GPU arm


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--ncells", type=int, default=None)
    ap.add_argument("--forms", default="plain,plain_trbdf2,chosen")
    ap.add_argument("--plain-steps", type=int, default=1,
                    help="timed steps of the plain FP64 form (context line, not the headline)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--dt-scale", type=float, default=1.0,
                    help="scale the workload's dt (profiling captures on a short interval)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--lane-variant", type=int, default=None,
                    help="fix the FP32-LU lane kernels' storage variant (kt.h KT_LANE_*) instead of tuning it")
    ap.add_argument("--block-warps", type=int, default=None,
                    help="fix the warps per block of the chosen form instead of tuning it")
    ap.add_argument("--cpu-cells", type=int, default=1024)
    ap.add_argument("--ref-cells", type=int, default=4096)
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2504_04941_gb300 import kt

    ncells = args.ncells or I.FULL_CELLS[args.workload]
    # weak scaling: every rank integrates its own full batch (rank-dependent seed)
    wl = I.workload(args.workload, ncells, seed=shard.rank_seed(args.workload, rank))
    wl.tol.dt *= args.dt_scale
    net = kt.Network(wl.network)
    dev = torch.device("cuda", local)
    y_in = torch.from_numpy(wl.cells.y).to(dev)
    T_in = torch.from_numpy(wl.cells.T).to(dev)
    rho = torch.from_numpy(wl.cells.rho).to(dev)
    out = dict(y=torch.empty_like(y_in), T=torch.empty_like(T_in),
               status=torch.empty(ncells, dtype=torch.int32, device=dev),
               nsub=torch.empty(ncells, dtype=torch.int32, device=dev),
               nnewton=torch.empty(ncells, dtype=torch.int32, device=dev))
    scratch = torch.zeros(kt.scratch_bytes(), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    forms = {"plain": dict(form=kt.KT_FORM_FP64, persistent=0, scheme=kt.KT_SCHEME_BE),
             "plain_trbdf2": dict(form=kt.KT_FORM_FP64, persistent=0, scheme=kt.KT_SCHEME_TRBDF2),
             "chosen": dict(form=kt.KT_FORM_FP32LU, persistent=1, use_graph=1, schedule=1,
                            scheme=kt.KT_SCHEME_TRBDF2)}
    tuned = None
    if not args.no_tune:
        base = kt.options(wl.tol, **forms["chosen"])
        # launch-shape cache (per network size, form and GPU name)
        cache = os.environ.get("KT_TUNE_CACHE", os.path.join(ROOT, ".tuned.json"))
        # tune the launch shape on the whole batch over a tenth of the interval: every
        # candidate runs at full occupancy with each cell past its first sub-steps (much
        # shorter intervals favour the variant that is cheapest to start a cell with)
        topts, tuned = kt.tuned_options(net, y_in, T_in, wl.tol.dt * 0.1, base, cache,
                                        sample=ncells)
        for f in ("cells_per_warp", "persistent", "block_warps", "blocks_per_sm", "lane_variant"):
            forms["chosen"][f] = int(getattr(topts, f))
    if args.lane_variant is not None:
        forms["chosen"]["lane_variant"] = args.lane_variant
    if args.block_warps is not None:
        forms["chosen"]["block_warps"] = args.block_warps
    state = kt.State(net, ncells)
    zero_cost = torch.zeros(ncells, dtype=torch.int32, device=dev)
    results = {}
    clocks = ClockSampler(local)
    clock_started = False
    # measured peaks of the FP64 and FP32 pipes (kt_fma_peak, ~0.5 s each, best of 3)
    peaks = {"fp64_tflops": kt.fma_peak(False), "fp32_tflops": kt.fma_peak(True)}
    cost = {"next": None}

    def run_step(name, opts):
        if forms[name].get("use_graph"):
            # the library-owned state replays a captured graph (queue order + kernel);
            # each step integrates the same input batch, copied in device to device,
            # with the cost estimate the longest-first order reads
            if forms[name].get("schedule") and cost["next"] is not None:
                state.set_cost(cost["next"])
            state.upload(y_in, T_in, rho)
            state.integrate(wl.tol.dt, opts)
        else:
            kt.integrate(net, y_in, T_in, wl.tol.dt, opts, rho=rho, out=out, scratch=scratch)

    for name in [f for f in args.forms.split(",") if f]:
        opts = kt.options(wl.tol, **forms[name])
        nsteps = args.steps if name == "chosen" else args.plain_steps
        # the plain form is a context line timed once without warm-up (one launch of
        # tens of seconds; module load and attribute setup are microseconds of it)
        nwarm = args.warmup if name == "chosen" else 0
        sched = bool(forms[name].get("schedule"))
        if sched:
            state.set_cost(zero_cost)          # the first warm-up runs without a cost history
        warm_ms = []
        for _ in range(nwarm):
            w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            w0.record(stream)
            run_step(name, opts)
            w1.record(stream)
            torch.cuda.synchronize()
            warm_ms.append(w0.elapsed_time(w1))
        if sched:
            # cost estimate of an operator-split simulation: the Newton counts of the next
            # interval (the batch's end state advanced by dt once more), not of the timed
            # interval itself.  The state holds y(dt) after the warm-ups.
            state.integrate(wl.tol.dt, opts)
            nxt = state.download()["nnewton"]
            cost["next"] = torch.from_numpy(nxt.copy()).to(dev)
        kt.check_scratch(scratch)
        state.check()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        if name == "chosen" and not clock_started:
            clocks.start()
            clock_started = True
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(nsteps):
            flush.fill_(s & 0xff)
            ev[s][0].record(stream)
            run_step(name, opts)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        step_ms = [a.elapsed_time(b) for a, b in ev]
        kt.check_scratch(scratch)
        state.check()
        tot_ms = sum(step_ms)
        if forms[name].get("use_graph"):
            st_h = state.download()
            for k in ("status", "nsub", "nnewton"):
                out[k].copy_(torch.from_numpy(st_h[k]))
        tot_ms = shard.max_over_ranks(tot_ms, dev)
        nnew = out["nnewton"].to(torch.int64).sum().item()
        nsub = out["nsub"].to(torch.int64).sum().item()
        st = out["status"].cpu().numpy()
        f64, f32, trans = flops_per_newton(wl.network, forms[name]["form"])
        per_launch_ms = tot_ms / nsteps
        results[name] = {
            "steps": nsteps, "warmup": nwarm,
            "options": {k: int(v) for k, v in forms[name].items()},
            "value": shard.weak_throughput(ncells, world, nsteps, tot_ms / 1e3),
            "ms_per_step": per_launch_ms,
            "step_ms": step_ms,
            "wall_s": wall,
            "newton_iters": int(nnew), "substeps": int(nsub),
            "status_counts": {int(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
            "fp64_flops_per_launch": float(nnew) * f64,
            "fp64_tflops": float(nnew) * f64 / (per_launch_ms / 1e3) / 1e12,
            "exp_per_s": float(nnew) * trans / (per_launch_ms / 1e3),
            "fp32_flops_per_factorisation": f32,
        }
        if forms[name]["form"] == kt.KT_FORM_FP32LU:
            # FP32 work with the counts the kernel keeps: a triangular solve per Newton
            # iteration, and per accepted sub-step at least one Jacobian and two
            # factorisations (h and h/2); rejected attempts and refreshes add more
            N = wl.network.n
            lu, solve = _lu_flops(N), 2 * N * N - N
            jac32 = f32 - (2 * N * N + lu + solve)
            results[name]["fp32_flops_lower_bound"] = float(nnew * solve + nsub * (jac32 + 2 * (2 * N * N + lu)))
        if sched:
            # warm-up 1 has no cost history (index order); later warm-ups order the queue
            # by the exact counts of the same integration (perfect foresight, a bound no
            # caller reaches); the timed steps use the next interval's counts
            results[name].update({
                "cold_ms": warm_ms[0] if warm_ms else None,
                "foresight_ms": min(warm_ms[1:]) if len(warm_ms) > 1 else None,
                "perturbed_ms": per_launch_ms,
                "history": "Newton counts of the following interval (end state advanced by dt)"})
        else:
            results[name]["warmup_ms"] = warm_ms
    clk = clocks.stop() if clock_started else {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}

    head = results.get("chosen") or results.get("plain")
    head_name = "chosen" if "chosen" in results else "plain"

    # ---- end to end through the public C-ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        opts = kt.options(wl.tol, **forms[head_name])
        hy = torch.from_numpy(wl.cells.y).pin_memory().numpy()
        hT = torch.from_numpy(wl.cells.T).pin_memory().numpy()
        hr = torch.from_numpy(wl.cells.rho).pin_memory().numpy()
        ho = dict(y=torch.empty(tuple(hy.shape), dtype=torch.float64).pin_memory().numpy(),
                  T=torch.empty(ncells, dtype=torch.float64).pin_memory().numpy(),
                  status=torch.empty(ncells, dtype=torch.int32).pin_memory().numpy(),
                  nsub=torch.empty(ncells, dtype=torch.int32).pin_memory().numpy(),
                  nnewton=torch.empty(ncells, dtype=torch.int32).pin_memory().numpy())
        # the cost estimate of the longest-first order comes from the host too, like the
        # inputs (an operator-split caller would pass its previous step's counts)
        use_cost = bool(forms[head_name].get("schedule")) and cost["next"] is not None
        hc = cost["next"].cpu().pin_memory().numpy() if use_cost else None
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            if use_cost:
                state.set_cost(hc)
            state.upload(hy, hT, hr)
            state.integrate(wl.tol.dt, opts)
            state.download(out=ho)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_s = shard.max_over_ranks(e2e_s, dev)
        ns = wl.network.ns
        e2e = {"value": shard.weak_throughput(ncells, world, args.e2e_steps, e2e_s), "unit": UNIT, "steps": args.e2e_steps,
               "h2d_bytes_per_step": ncells * (ns + 2) * 8 + (ncells * 4 if use_cost else 0),
               "d2h_bytes_per_step": ncells * (ns + 1) * 8 + 3 * ncells * 4}

    # ---- CPU baseline: the oracle on a bounded sample of the batch (rank 0, one GPU
    # only), and the error of each GPU form against it on the same cells (one more
    # launch per form on the sample, after the timed region)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nsample = min(args.cpu_cells, ncells)
        sample = wl.cells.subset(range(nsample))
        ora = {}
        for scheme in sorted({int(forms[name].get("scheme", 0)) for name in results}):
            ora[scheme] = oracle_on(wl.network, sample, wl.tol, scheme=scheme)
        head_scheme = int(forms[head_name].get("scheme", 0))
        _, threads, wall = ora[head_scheme]
        cpu = {"value": nsample / wall, "unit": UNIT, "cores": threads, "kind": "oracle",
               "scheme": SCHEME_NAMES[head_scheme],
               "sample": f"first {nsample} cells of the benchmark batch ({wl.name}, dt={wl.tol.dt:g} s), "
                         f"{wall:.1f} s wall"}
        for scheme, (_, thr, w) in ora.items():
            cpu[f"value_{SCHEME_NAMES[scheme]}"] = nsample / w
        # one host thread on the first 128 cells of the same sample (the chosen scheme)
        try:
            n1 = min(128, nsample)
            _, _, w1 = oracle_on(wl.network, sample.subset(range(n1)), wl.tol, scheme=head_scheme, threads=1)
            cpu["value_1thread"] = n1 / w1
            cpu["sample_1thread"] = f"first {n1} cells of the sample, 1 thread, {w1:.1f} s wall"
        except Exception as ex:              # a report, never a reason to lose the line
            cpu["value_1thread"] = {"error": repr(ex)[:300]}
        for name in results:
            try:
                so = kt.options(wl.tol, **forms[name])
                r = kt.integrate(net, torch.from_numpy(sample.y).to(dev), torch.from_numpy(sample.T).to(dev),
                                 wl.tol.dt, so, rho=torch.from_numpy(sample.rho).to(dev))
                kt.check_scratch(r["scratch"])
                g = {k: r[k].cpu().numpy() for k in ("y", "T", "status", "nsub")}
                results[name]["accuracy_vs_oracle"] = accuracy(
                    g, ora[int(forms[name].get("scheme", 0))][0], wl.network, sample.y)
            except Exception as ex:          # a report, never a reason to lose the line
                results[name]["accuracy_vs_oracle"] = {"error": repr(ex)[:300]}

    if rank == 0:
        r = head
        per_cell = LANE_TRAFFIC_BYTES_PER_CELL.get(kernel_source_hash())
        traffic = (per_cell * ncells if per_cell and args.workload == 2 and head_name == "chosen"
                   else None)
        hbm_peak, hbm_src = hbm_peak_gbs()
        hbm_gbs = traffic / (r["ms_per_step"] * 1e-3) / 1e9 if traffic else None
        p64, p32 = peaks["fp64_tflops"], peaks["fp32_tflops"]
        roof = {"bound": "alu", "achieved": r["fp64_tflops"], "peak": p64,
                "unit": "TFLOP/s", "frac": r["fp64_tflops"] / p64, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "pipe": "fp64",
                "peak_source": "measured in this run: kt_fma_peak FP64 FMA loop, best of 3 (of measured)",
                "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS,
                "fp32_peak_tflops": p32, "fp32_peak_source": "measured in this run: kt_fma_peak FP32 FMA loop",
                # the same launch against HBM: evidence that the path is not memory bound
                "hbm_gbs": hbm_gbs, "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src,
                "hbm_frac": hbm_gbs / hbm_peak if hbm_gbs else None,
                "kernel_source_hash": kernel_source_hash(),
                "kernel": f"{'lane_kernel' if wl.network.n <= 16 else 'warp_kernel'} ({head_name} form)"}
        if head_name == "chosen" and "fp32_flops_lower_bound" in r:
            roof["fp32_achieved_tflops"] = r["fp32_flops_lower_bound"] / (r["ms_per_step"] * 1e-3) / 1e12
            roof["fp32_frac"] = roof["fp32_achieved_tflops"] / p32
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if head_name == "plain" else "f64+f32",
                "data": "synthetic", "config": config_of(args, wl, ncells),
                "forms": results, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                # per timed step: the integrate kernel, plus the three queue-order kernels
                # (histogram, scan, scatter) when the longest-first schedule is on
                "gpu_launches": args.steps * (1 + (3 if forms[head_name].get("schedule") else 0)),
                "clocks": clk, "autotune": tuned}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
