#!/usr/bin/env python3
"""Benchmark: CPR-FPF Newton-step solves of the 200x200x50 dual-porosity
problem (4M cells, 8M unknowns) on GB300.

One step = the first 5-day backward-Euler timestep by Algorithm 1, from the
same initial state each time: every Newton iteration assembles R and J,
checks convergence, then solves (decoupling, block ILU(0), AMG value
refresh, CPR-FPF preconditioned FGMRES to the forcing term, update).
`value` is Newton-step solves per second over all GPUs (one replica of the
realisation per GPU, no collective on the data path); the median and p90
of the per-solve device time are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) each rank runs its own replica; rank 0 prints one
JSON line.  `--impl reference` times the CPU oracle on a bounded sample of
the same workload (rank 0 only).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CPR-FPF Newton-step solve time & HBM GB/s at 8M unknowns; served p99 latency"
UNIT = "Newton-step solves/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TIMED_KERNEL = "k_bsr_spmv<0>"
# DRAM bytes (read + written) per launch of TIMED_KERNEL on the 200x200x50 field: one
# launch captured with ncu on the 200x200x20 field (316,643,072 + 21,299,968 bytes against
# its 342,181,804 algorithmic bytes; the capture's summary is kept under profiles/), scaled by
# the algorithmic bytes of a 200x200x50 launch (859,771,804): the kernel streams every block
# once, so its traffic grows with them
TIMED_TRAFFIC = {(200, 200, 50, 0): round((316643072 + 21299968) * 859771804 / 342181804)}


def workload(args):
    import dp_inputs as di
    return di.field8m(args.nx, args.ny, args.nz)


def over_ranks(dist, device, elapsed, units):
    """Whole-job numbers over the ranks of a replica run: the slowest rank's
    elapsed time (max) and the units that all ranks processed (sum).  No-op
    on one process (dist None)."""
    if dist is None:
        return float(elapsed), float(units)
    import torch
    mx = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    sm = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx.item()), float(sm.item())


def spmv_bytes(nb, nnzb):
    """Algorithmic bytes of one y = A x launch (FP64 2x2 BSR): values,
    column indices, row pointers, x and y read/written once."""
    return 32 * nnzb + 4 * nnzb + 4 * (nb + 1) + 16 * nb + 16 * nb


# GB300's FP64 rate: 1.20 TFLOP/s, measured on this machine's GB300 with independent FMA
# chains on every SM (the nominal figure is 1.25)
FP64_TFLOPS = 1.20


def spmv_fp64(nnzb, ms_per_launch):
    """The FP64 side of the product's roofline: four FMAs (8 flops) per 2x2
    block, against GB300's FP64 rate; the product is bound by HBM and by the
    FP64 pipe together."""
    flops = 8 * nnzb
    tf = flops / (ms_per_launch / 1000.0) / 1e12
    return {"flops_per_launch": flops, "achieved_tflops": tf, "peak_tflops": FP64_TFLOPS,
            "frac": tf / FP64_TFLOPS,
            "peak_source": "FP64 FMA microbenchmark (independent chains, all SMs)"}


def sweep_bytes(nb, nnzb, c0_rows, c0_nnz, first_fused=True):
    """Algorithmic bytes of one full sweep (all colours) of the FP32 ILU(0)
    forward and backward solves and of one level-0 Gauss-Seidel sweep.  The
    pattern is structurally symmetric, so L and U hold (nnzb - nb)/2 blocks
    each.  Forward: per L block 16 B of values + 4 B column; per row the row
    pointer, pivot position and permutation (12 B), the FP64 right-hand side
    (16 B), the FP32 result written (8 B) and its neighbours' values read
    once (8 B).  Backward: per U block 20 B; per row 12 B of indices, the
    inverted pivot block (16 B), z read, gathered and written (24 B).
    Gauss-Seidel (FP32 pressure values, level 0 in the colour order of the
    ILU(0)): per entry 4 B value + 4 B column; per row the row pointer, 1/a_ii,
    b, x read and written, x gathered (24 B).  The pre-smoothing starts from
    x = 0, so its first colour (c0_rows rows, c0_nnz entries) reads no matrix
    entries and no x (12 B a row); with the FP32 preconditioner that colour
    (and x = 0 elsewhere) is written by the kernel that forms the V-cycle's
    right-hand side (first_fused), so the pre-smoothing sweep starts with the
    second colour.  The figure is the mean of the pre- and the
    post-smoothing sweep."""
    half = (nnzb - nb) // 2
    post = 8 * nnzb + 24 * nb
    pre = post - 8 * c0_nnz - (24 if first_fused else 12) * c0_rows
    return {"k_ilu_fwd": 20 * half + 44 * nb, "k_ilu_bwd": 20 * half + 52 * nb,
            "k_gs_c": (pre + post) // 2}


# Sweeps timed as a region (one event pair around the whole sweep) instead
# of launch by launch: the well rows of the level-0 Gauss-Seidel and of the
# ILU(0) forward sweep are launched as programmatic dependents of the colour
# launch before them, which an event between the two launches would prevent.
SWEEP_REGIONS = {"k_ilu_fwd": "sweep.ilu_fwd", "k_ilu_bwd": "sweep.ilu_bwd", "k_gs_c": "sweep.gs"}

ASSEMBLY_KERNELS = ("k_props", "k_conn_flux", "k_assemble")


def assembly_bytes(nb, nnzb, nc):
    """Algorithmic bytes of one assembly (the three kernels k_props,
    k_conn_flux, k_assemble together): what it must read and write once.
    Per block its column, its transmissibility or well index and the 2x2
    FP64 block written (44 B); per cell p, s_w and the reference porosity
    read, the old phase masses read and the new ones written (56 B); per
    block row its row pointer, diagonal position and the two residual
    entries (24 B).  The cell properties and the connection fluxes that the
    kernels pass to one another are not counted."""
    return 44 * nnzb + 56 * nc + 24 * nb


def coarse_cycle_bytes(levels, precision):
    """Algorithmic bytes of the part of one V-cycle below level 0 (levels
    1 .. L-1, the region "cycle.coarse"): per level above the coarsest, the
    pre-smoothing with its residual (the operator once: 4 B column and the
    value per entry, 4 B row pointer a row, b and 1/a_ii read, x and r
    written: 16 B a row), the restriction (P's entries as R's, R's row
    pointers, r read, the coarse b written), the prolongation (P's entries
    and row pointers, the coarse x read, x read and written) and the
    post-smoothing (the operator once more, b, 1/a_ii and x read, the result
    written: 16 B a row); on the coarsest level the dense FP64 inverse and
    b, x (or, smoothed there, the two sweeps).  Values are FP32, or BF16 on
    levels 1 .. L-2 with precision 2."""
    total = 0
    nl = len(levels)
    for l in range(1, nl):
        L = levels[l]
        n, nnz = L["n"], L["nnz"]
        vb = 2 if precision == 2 and l <= nl - 2 else 4
        if l == nl - 1:
            if L["smoother"] == 2:
                total += 8 * n * n + 8 * n
            else:
                total += 2 * ((4 + vb) * nnz + 4 * (n + 1) + 16 * n)
            continue
        nagg, pn = L["nagg"], L["p_nnz"]
        total += 2 * ((4 + vb) * nnz + 4 * (n + 1) + 16 * n)          # both smoothings
        total += (4 + vb) * pn + 4 * (nagg + 1) + 4 * n + 4 * nagg    # restriction
        total += (4 + vb) * pn + 4 * (n + 1) + 4 * nagg + 8 * n       # prolongation
    return total


def state_error(a, b):
    """Max |dp| / max |p| and max |ds_w| between two states."""
    import numpy as np
    return {"dp_rel": float(np.abs(a[0] - b[0]).max() / np.abs(b[0]).max()),
            "dsw_abs": float(np.abs(a[1] - b[1]).max())}


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for s in self.samples for n, v in zip(names, s[4:]) if v.strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def _oracle_steps(prob, budget_s, max_steps, min_steps=1):
    """Set up the oracle on `prob` (its first Newton step, which builds the
    colouring and the AMG hierarchy, untimed), then time whole Newton steps
    of the first timestep (assembly and solve_step from x^n) until the
    budget or max_steps is reached.  Returns (oracle sim, step times)."""
    import oracle as O
    s = O.OracleSim(prob, O.options("report"))
    s.assemble(prob.dt)
    s.solve_step()
    times = []
    t_start = time.perf_counter()
    while len(times) < max_steps:
        s.set_state(prob.p0, prob.sw0, prob.bhp0)
        t0 = time.perf_counter()
        s.assemble(prob.dt)
        s.solve_step()
        times.append(time.perf_counter() - t0)
        if len(times) >= min_steps and time.perf_counter() - t_start > budget_s:
            break
    return s, times


def oracle_sample(args, budget_s=20.0, keep=None):
    """The CPU oracle, as it stands, on the bench's own workload (the whole
    grid, no scaling): median time of up to three Newton steps after the
    untimed set-up step.  `keep` (a list) receives the oracle realisation
    for the precision-error check."""
    import dp_inputs as di
    prob = di.field8m(args.nx, args.ny, args.nz)
    s, times = _oracle_steps(prob, budget_s, 3)
    if keep is not None:
        keep.append(s)
    t = statistics.median(times)
    return {"value": 1.0 / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one Newton step (assembly, decoupling, ILU(0), AMG refresh, FGMRES to the "
                      f"forcing term) of the whole {args.nx}x{args.ny}x{args.nz} grid "
                      f"({prob.n_unknowns} unknowns), median of {len(times)} after an untimed "
                      f"set-up step; single-threaded C, no scaling"}


def _oracle_worker(nx, ny, nz, nsteps, barrier, out):
    """One process of the all-core oracle sample: set up, wait for the
    others, then time nsteps Newton steps of its own copy of the grid."""
    import dp_inputs as di
    import oracle as O
    prob = di.field8m(nx, ny, nz)
    s = O.OracleSim(prob, O.options("report"))
    s.assemble(prob.dt)
    s.solve_step()
    barrier.wait(timeout=1200)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        s.set_state(prob.p0, prob.sw0, prob.bhp0)
        s.assemble(prob.dt)
        s.solve_step()
    out.put(time.perf_counter() - t0)


def _host_mem_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def oracle_sample_all_cores(args, nsteps=2):
    """The same oracle on every host core at once: one process per core
    (started with spawn), each running nsteps Newton steps of its own copy of
    the whole grid after its set-up; throughput = steps of all processes /
    the slowest process's time.  The number of processes is bounded by the
    host memory available (about 700 bytes per unknown each, half the free
    memory at most) and by 64; `cores` reports how many ran.  The oracle
    itself is single-threaded C, unchanged."""
    import multiprocessing as mp
    unknowns = 4 * args.nx * args.ny * args.nz + 50
    mem = _host_mem_bytes()
    cores = min(os.cpu_count() or 1, 64)
    if mem:
        cores = max(1, min(cores, int(0.5 * mem // (700 * unknowns))))
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker,
                         args=(args.nx, args.ny, args.nz, nsteps, barrier, out))
             for _ in range(cores)]
    for p in procs:
        p.start()
    times = [out.get(timeout=1800) for _ in procs]
    for p in procs:
        p.join()
    return {"value": cores * nsteps / max(times), "unit": UNIT, "cores": cores,
            "kind": "oracle", "steps_per_process": nsteps,
            "sample": f"{cores} processes (of {os.cpu_count()} host cores), each {nsteps} Newton "
                      f"steps of its own copy of the whole {args.nx}x{args.ny}x{args.nz} grid "
                      f"after its set-up step, started together; steps of all processes / the "
                      f"slowest process's time; no scaling"}


def run_reference(args):
    """The reference arm: the oracle on every host core, and on one core,
    on the bench's own workload.  `steps` and `warmup` report what was
    timed: Newton steps per process, after one untimed set-up step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    nsteps = 2
    cb = oracle_sample_all_cores(args, nsteps)
    cb["single_core"] = oracle_sample(args)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": nsteps, "warmup": 1,
            "steps_requested": args.steps, "warmup_requested": args.warmup,
            "ms_per_step": 1000.0 / cb["value"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args), "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ensemble(args):
    """The 64-realisation ensemble (20x20x5 to 80x80x20 locations, own seeds
    and shape factors): one step = one 5-day timestep of every realisation
    from its initial state.  Timed twice on the same resident realisations:
    one after another on one host thread, and concurrently through
    sim_advance_many (each realisation on its own stream).  Wall clock
    around device-synchronised steps, since the work spans many streams."""
    import torch
    import dp_inputs as di
    from paper_1808_04338_gb300 import dpsim
    members = [di.ensemble_member(r) for r in range(64)]
    # the coarse V-cycle in per-level launches (the batch's requirement) for
    # every run here, so that the three ways run the same arithmetic
    opts = dpsim.options("report", precision=args.precision, schur=args.schur, cluster_rows=-1)
    sims, x0, streams = [], [], []
    for prob in members:
        streams.append(dpsim.OwnedStream())
        sims.append(dpsim.Sim(prob, opts, stream=streams[-1].torch))
        x0.append([torch.from_numpy(a).cuda() for a in (prob.p0, prob.sw0, prob.bhp0)])
    torch.cuda.synchronize()
    dts = [p.dt for p in members]

    tuned = 0
    if args.autotune:
        for s, (p, sw, b) in zip(sims, x0):
            s.set_state_device(p, sw, b)
        dpsim.advance_many(sims, dts, threads=args.threads)
        for s in sims:
            tuned += sum(1 for l in s.autotune(10).splitlines() if "->" in l)

    def step(threads, ss=None):
        ss = ss or sims
        for s, (p, sw, b) in zip(ss, x0):
            s.set_state_device(p, sw, b)
        rc, stats, _ = dpsim.advance_many(ss, dts, threads=threads)
        if rc != 0:
            raise RuntimeError(f"sim_advance_many failed ({rc})")
        return sum(st.newton_iters for st in stats), sum(st.linear_iters for st in stats)

    def timed(threads, ss=None):
        ss = ss or sims
        for _ in range(args.warmup):
            step(threads, ss)
        torch.cuda.synchronize()
        l0 = sum(s.launch_count() for s in ss)
        t0 = time.perf_counter()
        solves = its = 0
        for _ in range(args.steps):
            a, b = step(threads, ss)
            solves += a
            its += b
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        return {"sec": sec, "solves": solves, "its": its,
                "launches": sum(s.launch_count() for s in ss) - l0}

    # the lockstep batched engine: one launch per phase over all members of a
    # batch; `groups` batches (members dealt round-robin by size) advance
    # concurrently from their own host threads and streams, so that one
    # batch's per-member set-up overlaps another's batched FGMRES
    import concurrent.futures as cf

    def make_batches(groups):
        bss = [dpsim.OwnedStream() for _ in range(groups)]
        idx = [list(range(g, 64, groups)) for g in range(groups)]
        bts = [dpsim.Batch([sims[k] for k in ix], stream=st.torch) for ix, st in zip(idx, bss)]
        return bss, idx, bts

    def bstep(idx, bts, pool):
        for s, (p, sw, b) in zip(sims, x0):
            s.set_state_device(p, sw, b)
        torch.cuda.synchronize()
        res = list(pool.map(lambda q: bts[q].advance([dts[k] for k in idx[q]]), range(len(bts))))
        for rc, _, _ in res:
            if rc != 0:
                raise RuntimeError(f"batch_advance failed ({rc})")
        return (sum(st.newton_iters for _, stats, _ in res for st in stats),
                sum(st.linear_iters for _, stats, _ in res for st in stats))

    def btimed(groups):
        bss, idx, bts = make_batches(groups)
        with cf.ThreadPoolExecutor(max_workers=groups) as pool:
            for _ in range(args.warmup):
                bstep(idx, bts, pool)
            torch.cuda.synchronize()
            l0 = sum(bt.launch_count() for bt in bts)
            p0 = [bt.profile() for bt in bts]
            t0 = time.perf_counter()
            solves = its = 0
            for _ in range(args.steps):
                a, b = bstep(idx, bts, pool)
                solves += a
                its += b
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
        p1 = [bt.profile() for bt in bts]
        prof = {"ms_setup": sum(b[0][0] - a[0][0] for a, b in zip(p0, p1)),
                "ms_fgmres": sum(b[0][1] - a[0][1] for a, b in zip(p0, p1)),
                "ms_update": sum(b[0][2] - a[0][2] for a, b in zip(p0, p1)),
                "newton_rounds": sum(b[1][0] - a[1][0] for a, b in zip(p0, p1)),
                "arnoldi_steps": sum(b[1][2] - a[1][2] for a, b in zip(p0, p1)), "groups": groups}
        launches = sum(bt.launch_count() for bt in bts) - l0
        for bt in bts:
            bt.close()
        for st in bss:
            st.close()
        return {"sec": sec, "solves": solves, "its": its, "launches": launches, "profile": prof}

    clk = Clocks(torch.cuda.current_device())
    one = timed(1)
    many = timed(args.threads)
    by_groups = {g: btimed(g) for g in (1, 2, 4)}
    best = max(by_groups, key=lambda g: 64 * args.steps / by_groups[g]["sec"])
    clk.__enter__()
    bat = btimed(best)
    clk.__exit__()
    # the plain FP64 path on the same members, run the fastest plain way
    # (host threads, a stream each), for the comparison at equal tolerance
    fp64 = None
    if args.precision >= 1:
        o64 = dpsim.options("report", precision=0, schur=args.schur, cluster_rows=-1)
        s64 = [dpsim.Sim(prob, o64, stream=st.torch) for prob, st in zip(members, streams)]
        if args.autotune:
            step(args.threads, s64)
            for s in s64:
                s.autotune(10)
        r64 = timed(args.threads, s64)
        fp64 = {"value": 64 * args.steps / r64["sec"], "unit": "realisation timesteps/s",
                "threads": args.threads, "ms_per_step": 1000.0 * r64["sec"] / args.steps,
                "newton_solves_per_s": r64["solves"] / r64["sec"],
                "fgmres_iters_per_solve": r64["its"] / max(r64["solves"], 1),
                "note": "plain FP64 path (FP64 ILU(0) and AMG), sim_advance_many"}
        for s in s64:
            s.close()
    cells = sum(p.n_cells for p in members)
    line = {"metric": "batched ensemble timesteps", "value": 64 * args.steps / bat["sec"],
            "unit": "realisation timesteps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * bat["sec"] / args.steps,
            "higher_is_better": True, "dtype": "f64" if args.precision == 0 else "f64 (f32 preconditioner)",
            "data": "synthetic",
            "config": {"workload": f"64 realisations, 20x20x5 to 80x80x20 locations, {cells} cells",
                       "engine": "lockstep batches (one launch per phase over the members' "
                                 "tiles), concurrent batches from host threads",
                       "precision": args.precision, "schur": args.schur},
            "newton_solves_per_s": bat["solves"] / bat["sec"],
            "fgmres_iters_per_solve": bat["its"] / max(bat["solves"], 1),
            "threads": {"value": 64 * args.steps / many["sec"], "unit": "realisation timesteps/s",
                        "threads": args.threads, "ms_per_step": 1000 * many["sec"] / args.steps,
                        "newton_solves_per_s": many["solves"] / many["sec"],
                        "gpu_launches": many["launches"],
                        "note": "sim_advance_many: host threads, one stream per realisation"},
            "one_at_a_time": {"value": 64 * args.steps / one["sec"], "unit": "realisation timesteps/s",
                              "ms_per_step": 1000 * one["sec"] / args.steps,
                              "newton_solves_per_s": one["solves"] / one["sec"]},
            "autotune_decisions": tuned if args.autotune else None,
            "batch_profile": bat["profile"],
            "batch_groups": {g: 64 * args.steps / v["sec"] for g, v in by_groups.items()},
            "fp64_path": fp64,
            "gpu_launches": bat["launches"], "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    for s in sims:
        s.close()
    for st in streams:
        st.close()


def serve_stream(workers, precision, schur, budget_gb=160, warm=False):
    """One served stream: 512 timestep requests with Poisson arrivals (mean
    200/s) over 128 realisations of about 10k to 1M cells, served by the
    library's request server under a device budget of budget_gb.  Cold (the
    default): nothing is resident when the stream starts, so a realisation's
    first request includes building it (pattern, AMG set-up), and requests
    wait for admission and evictions as the budget dictates.  warm: every
    requested realisation is first made resident by one untimed 1-day
    request.  The stream arrives in real time; latency = result ready -
    arrival on the server's clock."""
    import numpy as np
    import torch
    import dp_inputs as di
    from paper_1808_04338_gb300 import dpsim
    members = [di.served_member(r) for r in range(128)]
    arrivals, real, dts = di.request_stream()
    budget = int(budget_gb) << 30
    srv = dpsim.Server(workers, budget, dpsim.options("report", precision=precision,
                                                      schur=schur))
    ids = [srv.add(p) for p in members]
    if warm:
        for t in [srv.submit(ids[r], di.DAY) for r in sorted(set(real.tolist()))]:
            if srv.wait(t).status != 0:
                raise RuntimeError("warm-up request failed")
    torch.cuda.synchronize()
    e0 = srv.info().evictions
    l0 = srv.info().launches
    t0 = time.perf_counter()
    tickets = []
    for a, r, d in zip(arrivals, real, dts):
        lag = a - (time.perf_counter() - t0)
        if lag > 0:
            time.sleep(lag)
        tickets.append(srv.submit(ids[int(r)], float(d) * di.DAY))
    res = [srv.wait(t) for t in tickets]
    info = srv.info()
    srv.close()
    lat = np.array([x.t_done_ms - x.t_submit_ms for x in res])
    span = (max(x.t_done_ms for x in res) - min(x.t_submit_ms for x in res)) / 1000.0
    newton = sum(x.stats.newton_iters for x in res)
    loads = sum(x.loaded for x in res)
    return {"solves_per_s": len(res) / span, "newton_solves_per_s": newton / span,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "makespan_s": span, "failed": int(sum(x.status != 0 for x in res)),
            "newton_per_request": newton / len(res), "workers": workers,
            "precision": precision, "budget_gb": budget_gb, "warm": warm,
            "requests_with_build": int(loads),
            "resident_gb": info.peak_resident_bytes / 1e9,
            "evictions": int(info.evictions - e0), "launches": info.launches - l0}


def serve_variants(workers, precision, schur):
    """The served stream cold at 160 GB (the headline), warm at 160 GB, cold
    under a 40 GB budget that forces evictions, and the plain FP64 path cold
    at 160 GB with the same number of workers."""
    return {"cold": serve_stream(workers, precision, schur),
            "warm": serve_stream(workers, precision, schur, warm=True),
            "evicting_40gb": serve_stream(workers, precision, schur, budget_gb=40),
            "fp64_same_workers": serve_stream(workers, 0, schur)}


def run_serve(args):
    """The served stream (serve_variants) with `--threads` workers."""
    import torch
    import dp_inputs as di
    members = [di.served_member(r) for r in range(128)]
    clk = Clocks(torch.cuda.current_device())
    clk.__enter__()
    v = serve_variants(args.threads, args.precision, args.schur)
    clk.__exit__()
    served = v["cold"]
    cells = sum(p.n_cells for p in members)
    line = {"metric": "served timestep-solve stream: p50/p99 latency and throughput",
            "value": served["solves_per_s"], "unit": "timestep solves/s", "n_gpus": 1,
            "higher_is_better": True, "p50_ms": served["p50_ms"], "p99_ms": served["p99_ms"],
            "dtype": "f64" if args.precision == 0 else "f64 (f32 preconditioner)",
            "data": "synthetic",
            "config": {"workload": f"512 requests, Poisson 200/s, 128 realisations "
                                   f"({cells} cells), dt 1-10 days, budget 160 GB, cold start",
                       "workers": args.threads, "precision": args.precision,
                       "schur": args.schur},
            "variants": v,
            "gpu_launches": served["launches"], "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_period(args):
    """A whole simulation period: Example 1's physics (Section 4) on the
    --nx x --ny x --nz grid (500x500x50 is Example 3's size), 800 days by
    sim_run (steps from 1 day doubling up to 20, halved when Newton fails),
    reported in the units of the paper's Table for Example 3: time steps,
    Newton and linear iterations, running time.  The time is the wall clock
    of the whole run on the device (set-up of the realisation excluded)."""
    import torch
    import dp_inputs as di
    from paper_1808_04338_gb300 import dpsim
    prob = di.paper_example(1, grid=(args.nx, args.ny, args.nz))
    opts = dpsim.options("report", precision=args.precision, schur=args.schur)
    sim = dpsim.Sim(prob, opts)
    torch.cuda.synchronize()
    clk = Clocks(torch.cuda.current_device())
    clk.__enter__()
    t0 = time.perf_counter()
    rc, st = sim.run(800 * di.DAY, 1 * di.DAY, 20 * di.DAY, 0.001 * di.DAY)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk.__exit__()
    kinds, _ = sim.well_controls()
    q_oil, q_wat = sim.well_rates()
    line = {"metric": "whole-period run (800 days) of Example 1's physics", "value": wall,
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "rc": rc,
            "time_steps": st.steps, "cuts": st.cuts, "newton_iters": st.newton_iters,
            "linear_iters": st.linear_iters, "days": st.t / di.DAY,
            "newton_solves_per_s": st.newton_iters / wall,
            "s_per_newton_iter": wall / max(st.newton_iters, 1),
            "dtype": "f64" if args.precision == 0 else "f64 (f32 preconditioner)",
            "data": "synthetic",
            "config": {"workload": f"Example 1's physics on {args.nx}x{args.ny}x{args.nz} "
                                   f"({prob.n_cells} cells, {prob.n_unknowns} unknowns), "
                                   f"wells at the same relative cells, 800 days",
                       "precision": args.precision, "schur": args.schur},
            "final_well_controls": [int(k) for k in kinds],
            "final_oil_rates_stb_day": [float(-q / (58.0 * di.LBM_FT3) / di.BBL_DAY)
                                        for q in q_oil],
            "paper_example3_64_ranks": {"time_steps": 68, "newton_iters": 267,
                                        "linear_iters": 623, "running_time_s": 2531.91},
            "gpu_launches": sim.launch_count(), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    sim.close()


def config_dict(args, nnzb=None):
    return {"workload": f"dual-porosity oil-water, {args.nx}x{args.ny}x{args.nz} grid, "
                        f"{2 * args.nx * args.ny * args.nz} cells, "
                        f"{4 * args.nx * args.ny * args.nz + 50} unknowns, 25 wells, "
                        f"lognormal perm (sd 2), first 5-day Newton step",
            "grid": [args.nx, args.ny, args.nz], "precision": args.precision,
            "decouple": args.decouple, "eta_mode": args.eta_mode, "schur": args.schur,
            "precond": "CPR-FPF",
            "l2": f"inputs larger than L2 (Jacobian {32 * nnzb / 1e6:.0f} MB)" if nnzb else
                  "inputs larger than L2",
            "parallelism": f"replicas x{args.gpus}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--nx", type=int, default=200)
    ap.add_argument("--ny", type=int, default=200)
    ap.add_argument("--nz", type=int, default=50)
    ap.add_argument("--precision", type=int, default=1,
                    help="0: FP64 everywhere; 1: FP32 ILU(0)/AMG inside FP64 FGMRES; 2: as 1 "
                         "with the AMG levels >= 1 stored in BF16")
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--no-schur-path", action="store_true")
    ap.add_argument("--no-bf16-path", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the served stream's p50/p99 in the default bench line")
    ap.add_argument("--cluster-rows", type=int, default=0,
                    help="AMG levels up to this many rows run in one cluster launch (0: default)")
    ap.add_argument("--decouple", type=int, default=0,
                    help="0: the paper's modified Gauss-Jordan step; 1: ABF; 2: True-IMPES")
    ap.add_argument("--eta-mode", type=int, default=2,
                    help="forcing term of Algorithm 1: 1, 2 or 3 (Section 3.1), 0: fixed")
    ap.add_argument("--schur", type=int, default=0,
                    help="1: eliminate the matrix cells exactly and solve the fracture-and-well "
                         "system")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the autotuner (sim_autotune: launch shapes of the AMG level "
                         "kernels and of level 0's colour sweeps, the V-cycle schedule), which "
                         "otherwise runs after one untimed timestep")
    ap.add_argument("--l0-kernel", type=int, default=None,
                    help="level 0's colour-sweep kernel (sim_set_l0_kernel), set after the "
                         "autotuner: for profiling a given kernel")
    ap.add_argument("--threads", type=int, default=16,
                    help="ensemble mode: host threads driving realisations concurrently")
    ap.add_argument("--mode", default="bench",
                    choices=["bench", "newton2", "ensemble", "serve", "period"],
                    help="newton2: create the realisation, run the first Newton solve of the "
                         "first step (AMG set-up), autotune (unless --no-autotune) and run the "
                         "second one, print their timings (a short run for profilers)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    from paper_1808_04338_gb300 import dpsim

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    if args.mode == "ensemble":
        return run_ensemble(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "period":
        return run_period(args)
    prob = workload(args)
    opts = dpsim.options("report", precision=args.precision, cluster_rows=args.cluster_rows,
                         decouple=args.decouple, eta_mode=args.eta_mode, schur=args.schur)
    if args.mode == "newton2":
        sim = dpsim.Sim(prob, opts)
        out = {}
        for k in ("first", "second"):
            sim.assemble(prob.dt)
            rc, st = sim.solve_step()
            out[k] = {"fgmres_iters": st.linear_iters, "ms_setup": st.ms_setup,
                      "ms_solve": st.ms_solve}
            if k == "first" and args.autotune:   # the bench's launch shapes for the second
                rep = sim.autotune(10)
                out["autotune"] = [l for l in rep.splitlines() if "->" in l]
            if k == "first" and args.l0_kernel is not None:
                sim.set_l0_kernel(args.l0_kernel)
        torch.cuda.synchronize()
        out["launches"] = sim.launch_count()
        print(json.dumps(out), flush=True)
        sim.close()
        return
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = dpsim.Sim(prob, opts, stream=stream)
    dev = torch.device("cuda", local)
    p0 = torch.from_numpy(prob.p0).to(dev)
    sw0 = torch.from_numpy(prob.sw0).to(dev)
    b0 = torch.from_numpy(prob.bhp0).to(dev)
    torch.cuda.synchronize()

    def timestep(sim, opts, solve_ms=None):
        """Algorithm 1 for one step through the C ABI; returns (solves, FGMRES iterations)."""
        sim.set_state_device(p0, sw0, b0)
        res0 = None
        solves = its = 0
        for l in range(opts.newton_max + 1):
            sim.assemble(prob.dt)
            nr = sim.norms()
            if res0 is None:
                res0 = nr[0]
            if nr[0] <= opts.newton_tol * res0 or nr[1] <= opts.newton_atol or l == opts.newton_max:
                break
            rc, st = sim.solve_step()
            solves += 1
            its += st.linear_iters
            if solve_ms is not None:
                solve_ms.append(st.ms_setup + st.ms_solve)
        return solves, its

    def measure(sim, opts, steps, warmup, clocks=None):
        for _ in range(warmup):
            timestep(sim, opts)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = sim.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        solve_ms, n_solves, n_its = [], 0, 0
        if clocks:
            clocks.__enter__()
        e0.record(stream)
        for _ in range(steps):
            a_, b_ = timestep(sim, opts, solve_ms)
            n_solves += a_
            n_its += b_
        e1.record(stream)
        torch.cuda.synchronize()
        if clocks:
            clocks.__exit__()
        ms, all_solves = over_ranks(dist, dev, e0.elapsed_time(e1), n_solves)
        if dist:
            dist.barrier()
        solve_ms.sort()
        return {"ms": ms, "solves": n_solves, "all_solves": all_solves, "its": n_its,
                "launches": sim.launch_count() - l0,
                "median": solve_ms[len(solve_ms) // 2] if solve_ms else None,
                "p90": solve_ms[min(len(solve_ms) - 1, int(0.9 * len(solve_ms)))] if solve_ms else None}

    def tune(sim, opts):
        """Launch shapes and the V-cycle schedule chosen by the library's
        autotuner after one untimed timestep (sim_autotune); returns its
        decisions."""
        timestep(sim, opts)
        rep = sim.autotune(20)
        lines = [l for l in rep.splitlines() if "->" in l]

        def changed(l):
            a, b = l.split(" -> ")
            return a.split()[-1] != b.split()[0]
        return {"decisions": len(lines), "changed": sum(1 for l in lines if changed(l)),
                "report": [l for l in lines if changed(l)]}

    tuned = tune(sim, opts) if args.autotune else None
    if args.l0_kernel is not None:
        sim.set_l0_kernel(args.l0_kernel)
    clk = Clocks(local)
    main = measure(sim, opts, args.steps, args.warmup, clk)
    timestep(sim, opts)
    states = {"headline": sim.get_state()}   # the converged first timestep of each variant
    ms, n_solves, n_its, launches = main["ms"], main["solves"], main["its"], main["launches"]
    all_solves = main["all_solves"]
    med, p90 = main["median"], main["p90"]

    # the dominant kernel timed with CUDA events on the simulation stream over
    # its own timed region (kernels are then launched one by one, not from graphs)
    sim.time_kernel(TIMED_KERNEL)
    sim.kernel_timing(reset=True)
    for _ in range(max(1, args.steps // 5)):
        timestep(sim, opts)
    k_ms, k_n = sim.kernel_timing(reset=True)
    sim.time_kernel(None)
    # the ILU(0) and Gauss-Seidel sweeps the same way, one kernel per timestep;
    # every FGMRES iteration applies the ILU(0) twice (both CPR-FPF stages) and
    # one V-cycle (one forward and one backward level-0 sweep)
    sweeps = {}
    colour, _ = sim.colours()
    rowptr = sim.jacobian()[0] if not args.schur else None
    if rowptr is not None and len(rowptr) == sim.snb + 1:
        lens = np.diff(rowptr)
        c0 = colour == 0
        c0_rows, c0_nnz = int(c0.sum()), int(lens[c0].sum())
    else:
        c0_rows, c0_nnz = 0, 0
    # the assembly kernels the same way (one launch each per Newton iteration)
    assembly = {"kernels": {}}
    asm_ms, asm_n = 0.0, 0
    for name in ASSEMBLY_KERNELS:
        sim.time_kernel(name)
        sim.kernel_timing(reset=True)
        timestep(sim, opts)
        t_ms, t_n = sim.kernel_timing(reset=True)
        sim.time_kernel(None)
        if t_n:
            assembly["kernels"][name] = {"ms_per_launch": t_ms / t_n, "launches": t_n}
            asm_ms += t_ms / t_n
            asm_n = max(asm_n, t_n)
    if asm_ms > 0.0:
        nbytes = assembly_bytes(sim.nb, sim.nnzb, sim.nc)
        assembly.update(bytes_per_assembly=nbytes, ms_per_assembly=asm_ms,
                        achieved_gbs=nbytes / (asm_ms / 1000.0) / 1e9)
    for name, nbytes in sweep_bytes(sim.snb, sim.snnzb, c0_rows, c0_nnz,
                                    first_fused=args.precision >= 1).items():
        region = SWEEP_REGIONS.get(name)
        sim.time_kernel(region or name)
        sim.kernel_timing(reset=True)
        _, its = timestep(sim, opts)
        t_ms, t_n = sim.kernel_timing(reset=True)
        sim.time_kernel(None)
        if t_n and its:
            n_sweeps = 2 * its
            sweeps[name] = {"achieved_gbs": nbytes * n_sweeps / (t_ms / 1000.0) / 1e9,
                            "bytes_per_sweep": nbytes, "ms_per_sweep": t_ms / n_sweeps,
                            "regions" if region else "launches": t_n}
            if region:
                sweeps[name]["timed_as"] = ("one event pair around each whole sweep ("
                                            + region + "), its launches back to back")

    # the V-cycle below level 0 as one region per V-cycle (its kernels are
    # small and latency-bound: the figure is their share of the copy rate)
    coarse = None
    levels = sim.amg_level_sizes()
    if len(levels) > 1:
        sim.time_kernel("cycle.coarse")
        sim.kernel_timing(reset=True)
        timestep(sim, opts)
        t_ms, t_n = sim.kernel_timing(reset=True)
        sim.time_kernel(None)
        if t_n:
            nbytes = coarse_cycle_bytes(levels, args.precision)
            coarse = {"ms_per_cycle": t_ms / t_n, "cycles": t_n, "bytes_per_cycle": nbytes,
                      "achieved_gbs": nbytes * t_n / (t_ms / 1000.0) / 1e9,
                      "levels": [[L["n"], L["nnz"], L["p_nnz"]] for L in levels[1:]]}

    # end to end through the C ABI with host buffers (pinned), copies timed
    hp = torch.from_numpy(prob.p0).pin_memory()
    hs = torch.from_numpy(prob.sw0).pin_memory()
    hb = torch.from_numpy(prob.bhp0).pin_memory()
    op = torch.empty_like(hp).pin_memory()
    osw = torch.empty_like(hs).pin_memory()
    ob = torch.empty_like(hb).pin_memory()
    e2e_steps = 0 if args.no_e2e else max(2, args.steps // 2)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_solves = 0
    for _ in range(e2e_steps):
        sim.set_state_ptr(hp.data_ptr(), hs.data_ptr(), hb.data_ptr())
        rc, st = sim.advance(prob.dt)
        e2e_solves += st.newton_iters
        sim.get_state_ptr(op.data_ptr(), osw.data_ptr(), ob.data_ptr())
    torch.cuda.synchronize()
    e2e_s, e2e_all = over_ranks(dist, dev, time.perf_counter() - t0, e2e_solves)
    nbytes_state = 8 * (2 * prob.n_cells + prob.n_wells)  # per timestep of e2e

    schur = None
    if args.schur == 0 and not args.no_schur_path:
        osch = dpsim.options("report", precision=args.precision, cluster_rows=args.cluster_rows,
                             decouple=args.decouple, eta_mode=args.eta_mode, schur=1)
        with torch.cuda.stream(stream):
            simsch = dpsim.Sim(prob, osch, stream=stream)
        if args.autotune:
            tune(simsch, osch)
        r = measure(simsch, osch, max(2, args.steps // 2), args.warmup)
        timestep(simsch, osch)
        states["schur_path"] = simsch.get_state()
        simsch.close()
        schur = {"value": r["all_solves"] / (r["ms"] / 1000.0), "unit": UNIT,
                 "solve_ms_median": r["median"], "solve_ms_p90": r["p90"],
                 "fgmres_iters_per_solve": r["its"] / max(r["solves"], 1),
                 "ms_per_step": r["ms"] / max(2, args.steps // 2),
                 "note": "the same timestep with the matrix cells eliminated exactly before "
                         "the solve (CPR-FPF on the fracture-and-well system, 4M unknowns)"}

    bf16 = None
    if args.precision == 1 and not args.no_bf16_path:
        obf = dpsim.options("report", precision=2, cluster_rows=args.cluster_rows,
                            decouple=args.decouple, eta_mode=args.eta_mode, schur=args.schur)
        with torch.cuda.stream(stream):
            simbf = dpsim.Sim(prob, obf, stream=stream)
        if args.autotune:
            tune(simbf, obf)
        r = measure(simbf, obf, max(2, args.steps // 2), args.warmup)
        timestep(simbf, obf)
        states["bf16_coarse_path"] = simbf.get_state()
        simbf.close()
        bf16 = {"value": r["all_solves"] / (r["ms"] / 1000.0), "unit": UNIT,
                "solve_ms_median": r["median"], "solve_ms_p90": r["p90"],
                "fgmres_iters_per_solve": r["its"] / max(r["solves"], 1),
                "ms_per_step": r["ms"] / max(2, args.steps // 2),
                "note": "the same timestep with the AMG levels >= 1 stored in BF16 "
                        "(precision 2; FP32 arithmetic, FP64 FGMRES)"}

    fp64 = None
    if args.precision != 0 and not args.no_fp64_path:
        o64 = dpsim.options("report", precision=0, cluster_rows=args.cluster_rows,
                            decouple=args.decouple, eta_mode=args.eta_mode, schur=args.schur)
        with torch.cuda.stream(stream):
            sim64 = dpsim.Sim(prob, o64, stream=stream)
        if args.autotune:
            tune(sim64, o64)
        r = measure(sim64, o64, max(2, args.steps // 2), args.warmup)
        timestep(sim64, o64)
        states["fp64_path"] = sim64.get_state()
        sim64.close()
        fp64 = {"value": r["all_solves"] / (r["ms"] / 1000.0), "unit": UNIT,
                "solve_ms_median": r["median"], "solve_ms_p90": r["p90"],
                "fgmres_iters_per_solve": r["its"] / max(r["solves"], 1),
                "note": "the same timestep with FP64 ILU(0) and AMG"}

    if rank == 0:
        value = all_solves / (ms / 1000.0)
        peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
        peak = peaks.get("hbm_gbs", 6800.0)
        ach = spmv_bytes(sim.snb, sim.snnzb) / (k_ms / max(k_n, 1) / 1000.0) / 1e9 if k_n else None
        cpu = None
        errors = None
        if not args.no_cpu_baseline:
            keep = []
            try:
                cpu = oracle_sample(args, keep=keep)
            except Exception as e:  # report, do not fail the bench
                cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                       "sample": f"failed: {e}"}
            # each variant's converged first timestep against the FP64 oracle: the
            # oracle's scaled residual there relative to its residual at x^n (the
            # Newton tolerance is 1e-6), its mass balance, and the state's
            # distance from the plain FP64 GPU path's
            if keep:
                o = keep[0]
                o.set_state(prob.p0, prob.sw0, prob.bhp0)
                o.assemble(prob.dt)
                r0 = o.norms()[0]
                errors = {"newton_tol": opts.newton_tol}
                for k, x in states.items():
                    o.set_iterate(*x)
                    o.assemble(prob.dt)
                    nr = o.norms()
                    e = {"oracle_residual_ratio": float(nr[0] / r0),
                         "oracle_mass_balance_rel": float(max(
                             abs(nr[4 + a] - nr[6 + a] * prob.dt) /
                             max(abs(nr[4 + a]), abs(nr[6 + a] * prob.dt)) for a in range(2)))}
                    if k != "fp64_path" and "fp64_path" in states:
                        e["vs_fp64_path"] = state_error(x, states["fp64_path"])
                    errors[k] = e
                keep.clear()
                del o
            try:
                cpu["all_cores"] = oracle_sample_all_cores(args)
            except Exception as e:
                cpu["all_cores"] = {"value": None, "sample": f"failed: {e}"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == 0 else "f64 (f32 preconditioner)",
            "data": "synthetic", "config": config_dict(args, sim.nnzb),
            "newton_solves_per_step": n_solves / args.steps,
            "fgmres_iters_per_solve": n_its / max(n_solves, 1),
            "solve_ms_median": med, "solve_ms_p90": p90,
            "roofline": {"bound": "hbm", "kernel": "bsr_spmv (FP64 2x2 BSR, y = A x)",
                         "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": (ach / peak) if ach else None,
                         "traffic": TIMED_TRAFFIC.get((args.nx, args.ny, args.nz, args.schur)),
                         "launches_timed": k_n,
                         "avg_launch_ms": (k_ms / k_n) if k_n else None,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback",
                         "fp64": spmv_fp64(sim.snnzb, k_ms / k_n) if k_n else None},
            "sweeps": {k: dict(v, frac=v["achieved_gbs"] / peak) for k, v in sweeps.items()},
            "assembly": dict(assembly, frac=assembly["achieved_gbs"] / peak)
                        if "achieved_gbs" in assembly else assembly,
            "coarse_cycle": dict(coarse, frac=coarse["achieved_gbs"] / peak) if coarse else None,
            "errors_vs_oracle": errors,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_all / e2e_s if e2e_steps else None, "unit": UNIT,
                    "h2d_bytes_per_step": nbytes_state, "d2h_bytes_per_step": nbytes_state},
            "fp64_path": fp64,
            "bf16_coarse_path": bf16,
            "schur_path": schur,
            "gpu_launches": launches,
            "autotune": tuned,
            "clocks": clk.summary(),
        }
    sim.close()
    if rank == 0:
        # the served stream's p50/p99 (one GPU; the realisations of the 8M-unknown
        # bench are released first)
        if not args.no_serve and world == 1:
            torch.cuda.synchronize()
            try:
                v = serve_variants(args.threads, args.precision, args.schur)
                sv = v["cold"]
                keys = ("p50_ms", "p99_ms", "solves_per_s", "evictions", "requests_with_build",
                        "failed", "workers", "precision", "budget_gb")
                line["served"] = dict(
                    {k: sv[k] for k in keys},
                    workload=f"512 timestep requests, Poisson 200/s, 128 realisations of "
                             f"10k-1M cells, {args.threads} workers, cold start (first "
                             f"request of a realisation builds it)",
                    gpu_launches=sv["launches"],
                    warm={k: v["warm"][k] for k in keys},
                    evicting_40gb={k: v["evicting_40gb"][k] for k in keys},
                    fp64_same_workers={k: v["fp64_same_workers"][k] for k in keys})
            except Exception as e:  # report, do not fail the bench
                line["served"] = {"p50_ms": None, "p99_ms": None, "error": str(e)}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
