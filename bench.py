"""Benchmark: cell-updates per second per SSP-RK3 stage (FP64) of the TENO-M Euler solver,
the face kernel's roofline fraction, and the adjoint/forward cost ratio.

Default workload: 3D Euler, 256^3 periodic on [0, 2 pi]^3, seeded solenoidal velocity
(E(k) ~ k^4 exp(-2 (k/4)^2), rms Mach 0.6), TENO8A-M-MP, CFL 0.4 -- the largest of the
paper-shaped workloads that fits one GPU ("throughput at scale").  One step = one SSP-RK3
step (3 stages: CFL reduction, face sweeps on the three axes, flux difference + stage
combine), all on the GPU through the C ABI.  The same line carries the adjoint workload's
figures (2D 512^2, 200 steps, checkpoints every 20: backward over forward time per step,
central-difference check on 16 seeded directions at two step sizes).

Prints one JSON line.  --impl reference times the CPU oracle (the deliberately slow,
plain FP64 restatement of the method) on a bounded sample of the same workload.
Multi-GPU (torchrun): independent replicas, one problem per rank (the method has no
exchange between problems); value = all ranks' cell updates / max rank time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator, shape x-first, K, limiter)
    "broadband_2d_2048_teno6_mp": ("broadband_2d", (2048, 2048), 6, 0),
    "broadband_2d_2048_teno8_tvd5": ("broadband_2d", (2048, 2048), 8, 1),
    "solenoidal_3d_256_teno8_mp": ("solenoidal_3d", (256, 256, 256), 8, 0),
    # a smaller case of the same 3D field recipe, for ncu captures (0.5 GB on the device)
    "solenoidal_3d_128_teno8_mp": ("solenoidal_3d", (128, 128, 128), 8, 0),
    # slabs of the 256^3 field for ncu captures of its face kernels: 32 planes thin in z
    # (the x and y sweeps see exactly the full field's stencils) or thin in y (the z sweep)
    "solenoidal_3d_256_slab_z32_teno8_mp": ("solenoidal_3d_slab_z", (256, 256, 32), 8, 0),
    "solenoidal_3d_256_slab_y32_teno8_mp": ("solenoidal_3d_slab_y", (256, 32, 256), 8, 0),
}
BATCH_WORKLOADS = {
    # name: (problems, seed, nmin, nmax, K, limiter)
    "batched_riemann_512_teno6_mp": (512, 4, 128, 8192, 6, 0),
}
ADJOINT_WORKLOADS = {
    # name: (n, seed, steps, window, checkpoint_every, K, limiter)
    "adjoint_broadband_2d_512_teno6_mp": (512, 5, 200, 64, 20, 6, 0),
}
DEFAULT = "solenoidal_3d_256_teno8_mp"
ADJOINT_DEFAULT = "adjoint_broadband_2d_512_teno6_mp"
FP64_LANES_PER_CLK = 304  # FP64 pipe: 2 lanes per clock per SM x 152 SMs


FACE_SOURCES = ("tenom_face.cuh", "tenom_face_fwd.cuh", "tenom_recon.cuh", "tenom_linear.cuh",
                "tenom_stats.cuh", "teno_coeffs.cuh", "tenom_fastmath.cuh", "tenom_launch.cuh", "tenom_internal.h")


BATCH_SOURCES = FACE_SOURCES + ("tenom_batch.cu", "tenom_batch_kernel.cuh", "tenom_positivity.cuh")


def face_source_hash(sources=FACE_SOURCES):
    """Hash of the sources a kernel is compiled from (tags the ncu figures)."""
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2010_13289_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_figures(name, kernel="face_kernel", sources=FACE_SOURCES):
    """ncu figures of a kernel committed for this workload (profiles/<kernel>_<name>.md), or
    None when there are none or they were taken from other kernel sources than the ones
    built now."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, name))
    if not os.path.exists(path):
        return None
    fig, inside = {}, False
    for line in open(path):
        if line.strip() == "```figures":
            inside = True
        elif inside and line.strip() == "```":
            break
        elif inside and ":" in line:
            k, v = line.split(":", 1)
            fig[k.strip()] = v.strip()
    if fig.get("source_sha256") != face_source_hash(sources):
        return None
    fig["file"] = os.path.relpath(path, ROOT)
    return fig


def flops_per_face(name):
    """Stored algorithmic FP64 operation counts per face (oracle op counter)."""
    key = {"broadband_2d_2048_teno6_mp": ("broadband_2d_2048", "K=6", "lim=MP"),
           "broadband_2d_2048_teno8_tvd5": ("broadband_2d_2048", "K=8", "lim=TVD5"),
           "solenoidal_3d_256_teno8_mp": ("solenoidal_3d_256", "K=8", "lim=MP"),
           "batched_riemann_512_teno6_mp": ("riemann_1d_batch", "K=6", "lim=MP")}.get(name)
    if key is None:
        return None
    with open(os.path.join(ROOT, "tests", "golden", "flops_per_face.txt")) as fh:
        for line in fh:
            parts = line.split()
            if parts and not line.startswith("#") and tuple(parts[:3]) == key:
                vals = [float(x) for x in parts[3:]]
                return sum(vals) / len(vals)
    raise KeyError(name)


def make_prim(name, seed):
    import numpy as np
    from paper_2010_13289_gb300 import problems as PB
    gen, shape, K, lim = WORKLOADS[name]
    if gen == "broadband_2d":
        prim, dx = PB.broadband_2d(shape[0], seed)
        return prim, (dx, dx)
    if gen == "solenoidal_3d_slab_z":
        prim, dx = PB.solenoidal_3d(256, seed)
        return np.ascontiguousarray(prim[:, :shape[2]]), (dx, dx, dx)
    if gen == "solenoidal_3d_slab_y":
        prim, dx = PB.solenoidal_3d(256, seed)
        return np.ascontiguousarray(prim[:, :, :shape[1]]), (dx, dx, dx)
    prim, dx = PB.solenoidal_3d(shape[0], seed)
    return prim, (dx, dx, dx)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, ws, device="cuda"):
    """The largest x over the ranks of the job (x itself for one rank): every timing of the
    replicas path is the slowest rank's."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_rate(units_per_rank, ws, seconds):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest time."""
    return float(units_per_rank) * ws / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


_PRIM_CACHE = {}


def cached_prim(name, seed):
    if (name, seed) not in _PRIM_CACHE:
        _PRIM_CACHE[(name, seed)] = make_prim(name, seed)
    return _PRIM_CACHE[(name, seed)]


def oracle_rate(name, seconds=12.0, seed=2):
    """CPU oracle (single thread): one operator evaluation (all axes) on a row block of the
    workload's initial state, sized for about `seconds` of work.
    Returns (cell-updates/s per stage, sample description, elapsed s); the block's row count
    is left in oracle_rate.rows."""
    import numpy as np
    import oracle as orc
    gen, shape, K, lim = WORKLOADS[name]
    prim, dx = cached_prim(name, seed)
    S = orc.make_scheme(K, limiter=lim)

    def block(rows):
        if len(shape) == 2:
            p = np.ascontiguousarray(prim[:, :rows, :])
            sh = (shape[0], rows)
        else:
            p = np.ascontiguousarray(prim[:, :rows, :, :])
            sh = (shape[0], shape[1], rows)
        g = orc.make_grid(sh, dx, (orc.BC_PERIODIC,) * len(shape))
        return g, orc.init_state(g, p), int(np.prod(sh))
    g, U, nc = block(4)
    t0 = time.perf_counter()
    orc.rhs(g, S, U)
    t_cell = (time.perf_counter() - t0) / nc
    rows = max(4, min(shape[-1], int(seconds / (t_cell * nc / 4))))
    g, U, nc = block(rows)
    t0 = time.perf_counter()
    orc.rhs(g, S, U)
    el = time.perf_counter() - t0
    sample = ("one operator evaluation (all %d axes, periodic wrap of the block) on a %s block of the "
              "%s initial state, 1 thread" % (len(shape), "x".join(str(n) for n in (shape[:-1] + (rows,))), name))
    oracle_rate.rows = rows
    return nc / el, sample, el


def _oracle_block_worker(job):
    """One process of the all-cores oracle figure: one operator evaluation on its own block."""
    import numpy as np
    import oracle as orc
    sh, dx, bc, K, lim, p = job
    g = orc.make_grid(sh, dx, bc)
    S = orc.make_scheme(K, limiter=lim)
    U = orc.init_state(g, p)
    t0 = time.perf_counter()
    orc.rhs(g, S, U)
    return int(np.prod(sh)), time.perf_counter() - t0


def oracle_rate_all_cores(name, rows_single, seed=2):
    """CPU oracle on every core the process may use: the same single-thread code, one process
    per core (spawned), each evaluating the operator on its own block of rows_single rows of
    the workload's initial state (wrapping around the grid).  Returns (cell-updates/s per
    stage = all cells / the slowest process's time, cores, sample)."""
    import multiprocessing as mp
    import numpy as np
    import oracle as orc
    orc.build()
    gen, shape, K, lim = WORKLOADS[name]
    prim, dx = cached_prim(name, seed)
    ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    jobs = []
    for w in range(ncores):
        idx = (np.arange(rows_single) + w * rows_single) % prim.shape[1]
        p = np.ascontiguousarray(np.take(prim, idx, axis=1))
        sh = tuple(shape[:-1]) + (rows_single,)
        jobs.append((sh, dx, (orc.BC_PERIODIC,) * len(shape), K, lim, p))
    with mp.get_context("spawn").Pool(ncores) as pool:
        res = pool.map(_oracle_block_worker, jobs, chunksize=1)
    cells = sum(c for c, _ in res)
    el = max(t for _, t in res)
    sample = ("%d processes, each one operator evaluation on its own %s block of the %s initial state"
              % (ncores, "x".join(str(n) for n in (shape[:-1] + (rows_single,))), name))
    return cells / el, ncores, sample


def oracle_rate_batch(name, seconds):
    """CPU oracle (single thread): operator evaluations of the batch's problems, in order,
    until about `seconds` of work; returns (cell-updates/s per stage, sample, elapsed s)."""
    import oracle as orc
    from paper_2010_13289_gb300 import problems as PB
    nprob, seed, nmin, nmax, K, lim = BATCH_WORKLOADS[name]
    if name not in _PRIM_CACHE:
        _PRIM_CACHE[name] = PB.batch_riemann(nprob, seed, nmin, nmax)
    sizes, prims, dxs = _PRIM_CACHE[name]
    S = orc.make_scheme(K, limiter=lim)
    cells, el, used = 0, 0.0, 0
    for n, p, dx in zip(sizes, prims, dxs):
        g = orc.make_grid((int(n),), (dx,), (orc.BC_TRANSMISSIVE,))
        U = orc.init_state(g, p)
        t0 = time.perf_counter()
        orc.rhs(g, S, U)
        el += time.perf_counter() - t0
        cells += int(n)
        used += 1
        if el >= seconds:
            break
    return cells / el, "operator evaluations of the first %d of the %d batch problems (%d cells), 1 thread" % (
        used, nprob, cells), el


def launches_per_step(dim, positivity):
    """Kernel launches of one SSP-RK3 step of a grid workload: the signal-speed reduction, dt
    and the time update, and per stage the primitives, one face sweep per axis (plus one
    limiter pass per axis when the positivity limiter is on) and the cell update."""
    return 3 + 3 * (dim * (2 if positivity else 1) + 2)


def grid_config(name, ws, positivity):
    """The config object of a grid workload, identical in both arms."""
    gen, shape, K, lim = WORKLOADS[name]
    nv = len(shape) + 2
    ncell = 1
    for m in shape:
        ncell *= m
    nface = sum(ncell // shape[a] * (shape[a] + 1) for a in range(len(shape)))
    return {"workload": name, "shape": list(shape), "K": K, "limiter": "MP" if lim == 0 else "TVD5",
            "parallelism": "replicas" if ws > 1 else "single", "cfl": 0.4,
            "positivity_limiter": bool(positivity),
            "l2": "working set per stage (state, stage buffer, face buffers: %.0f MB) > L2"
                  % ((2 * nv * ncell + nv * nface) * 8 / 1e6)}


def batch_config(name, ws):
    """The config object of a batched workload, identical in both arms."""
    from paper_2010_13289_gb300 import problems as PB
    nprob, seed, nmin, nmax, K, lim = BATCH_WORKLOADS[name]
    cells = int(PB.batch_sizes(nprob, seed, nmin, nmax).sum())
    return {"workload": name, "problems": nprob, "cells": cells, "K": K, "limiter": "MP" if lim == 0 else "TVD5",
            "parallelism": "replicas" if ws > 1 else "single",
            "l2": "state + 2 stage buffers: %.0f MB < L2: L2 flushed (256 MB write) before every timed step"
                  % (3 * 8 * 3 * cells / 1e6)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    name = args.workload
    if name in BATCH_WORKLOADS:
        per_step = args.ref_seconds if args.ref_seconds else max(1.0, min(12.0, 150.0 / (args.steps + args.warmup)))
        for _ in range(args.warmup):
            oracle_rate_batch(name, min(1.0, per_step))
        rates, times = [], []
        for _ in range(args.steps):
            r, sample, el = oracle_rate_batch(name, per_step)
            rates.append(r)
            times.append(el)
        v = statistics.median(rates)
        nprob, seed, nmin, nmax, K, lim = BATCH_WORKLOADS[name]
        out = {"impl": "reference", "metric": "cell-updates/s per RK stage (FP64)", "value": v,
               "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded, shaped like the paper's workloads)",
               "config": batch_config(name, ws),
               "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle", "sample": sample},
               "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return
    per_step = args.ref_seconds if args.ref_seconds else max(1.0, min(12.0, 150.0 / (args.steps + args.warmup)))
    rates, samples, times = [], None, []
    for _ in range(args.warmup):
        oracle_rate(name, seconds=min(1.0, per_step))
    for _ in range(args.steps):
        r, samples, el = oracle_rate(name, seconds=per_step)
        rates.append(r)
        times.append(el)
    v = statistics.median(rates)
    gen, shape, K, lim = WORKLOADS[name]
    out = {"impl": "reference", "metric": "cell-updates/s per RK stage (FP64)", "value": v,
           "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded, shaped like the paper's workloads)",
           "config": grid_config(name, ws, args.positivity),
           "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle", "sample": samples},
           "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_13289_gb300 import tenom as T

    name = args.workload
    gen, shape, K, lim = WORKLOADS[name]
    prim, dx = make_prim(name, args.seed + rank)
    pp = T.PP_ON if args.positivity else T.PP_OFF
    S = T.Solver(shape, dx, (T.BC_PERIODIC,) * len(shape), T.make_scheme(K, limiter=lim, positivity=pp))
    U0 = S.init_state(torch.from_numpy(prim).cuda())
    U = U0.clone()
    ncell = int(np.prod(shape))
    nface = sum(ncell // shape[a] * (shape[a] + 1) for a in range(len(shape)))
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up
    S.advance(U, args.warmup)
    barrier()
    # timed region: K SSP-RK3 steps, device-side dt; face kernels timed with events
    clocks = ClockSampler(local)
    clocks.start()
    S.kernel_timing(True)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    S.advance(U, args.steps)
    ev1.record(stream)
    barrier()
    face_ms, face_launches = S.kernel_timing(False)
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws)
    assert S.status() == 0, "non-physical state in the benchmark run"
    value = job_rate(float(ncell) * 3 * args.steps, ws, ms * 1e-3)

    # end to end through the C ABI with host buffers: H2D of the state, one RK3 step, D2H
    host_in = torch.empty(S.state_shape, dtype=torch.float64, pin_memory=True)
    host_out = torch.empty(S.state_shape, dtype=torch.float64, pin_memory=True)
    host_in.copy_(U.cpu())
    e2e_steps = max(1, min(args.steps, 5))
    S.advance_host(host_in, host_out, nsteps=1)  # warm
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        S.advance_host(host_in, host_out, nsteps=1)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    e2e = job_rate(float(ncell) * 3 * e2e_steps, ws, e2e_s)
    state_bytes = 8 * S.nv * ncell

    # roofline of the dominant kernel (face flux): bound by FP64 instruction issue
    probe = T.fp64_peak()
    roof = face_roofline(name, shape, S.nv, face_ms, face_launches, clk, probe)
    lps = launches_per_step(len(shape), args.positivity)

    out = {"metric": "cell-updates/s per RK stage (FP64)", "value": value, "unit": "cell-updates/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded, shaped like the paper's workloads)",
           "config": grid_config(name, ws, args.positivity),
           "e2e": {"value": e2e, "unit": "cell-updates/s", "h2d_bytes_per_step": state_bytes,
                   "d2h_bytes_per_step": state_bytes},
           "gpu_launches": lps * args.steps,
           "roofline": roof, "clocks": clk}
    # decision statistics of the method at the end state (a logging pass after the timed
    # region): nonsmooth share per candidate, limiter activity, near-cutoff decisions
    cnt = None
    for a in range(len(shape)):
        cnt = S.decision_stats(U, a, counters=cnt)
    out["decision_stats"] = decision_summary(T.stats_dict(cnt.cpu().numpy(), K), K)
    if args.decision_log:
        with open(args.decision_log, "a") as fh:
            fh.write(json.dumps({"workload": name, "steps": args.warmup + args.steps + e2e_steps + 1,
                                 "state": "end of the run", **out["decision_stats"]}) + "\n")
    S.close()
    del U, U0, host_in, host_out
    torch.cuda.empty_cache()
    if ws == 1 and name == DEFAULT and not args.no_adjoint:
        # the metric's second figure: the adjoint workload's cost ratio, in the same process
        out["adjoint"] = measure_adjoint(ADJOINT_DEFAULT, fd_dirs=args.fd_dirs)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, sample, el = oracle_rate(name, seconds=args.ref_seconds or 12.0, seed=args.seed)
        ra, cores, sample_all = oracle_rate_all_cores(name, oracle_rate.rows, seed=args.seed)
        out["cpu_baseline"] = {"value": ra, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                               "sample": sample_all,
                               "single_thread": {"value": r, "cores": 1, "sample": sample}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def decision_summary(c, K):
    """Shares of the counters of tenom_decision_stats (per split side: face x characteristic
    field x f+/f-)."""
    n = max(c["sides"], 1)
    out = {"sides": c["sides"], "counts": c,
           "nonsmooth_share_per_k": [c["nonsmooth_k%d" % k] / n for k in range(K - 2)],
           "all_smooth_share": c["all_smooth"] / n, "limited_share": c["limited_sides"] / n,
           "limiter_changed_per_side": c["limiter_changed"] / n,
           "certified_share": c["certified"] / n, "certified_disagree": c["certified_disagree"],
           "near_cutoff_decisions": c["near_cutoff"], "near_cutoff_sides": c["near_cutoff_sides"],
           "near_integer_beta": c["near_integer_beta"]}
    ct = [c["ct_exp_%d" % e] for e in (7, 8, 9, 10)]
    if sum(ct):
        out["adaptive_ct_share"] = {"1e-%d" % e: v / n for e, v in zip((7, 8, 9, 10), ct)}
    return out


def face_roofline(name, shape, nv, face_ms, face_launches, clk, probe_flops):
    """Roofline of the face kernel.  The kernel is bound by FP64 instruction issue (about 36
    algorithmic flops per byte against a ridge point of 0.2), so the bound is the FP64
    pipe: achieved = FP64 thread instructions per face (ncu count of DFMA + DADD + DMUL,
    committed under profiles/ for these kernel sources) x faces per launch / the CUDA-event
    launch time of the timed region; peak = the DFMA probe's measured instruction rate
    (the pool's peaks file has no FP64 figure).  HBM use and the oracle's op count per
    face (the textbook formulation's work rate) are reported beside it, not as the
    fraction."""
    ncell = 1
    for m in shape:
        ncell *= m
    faces_per_launch = sum(ncell // shape[a] * (shape[a] + 1) for a in range(len(shape))) / len(shape)
    probe_inst = probe_flops / 2.0  # the probe counts an FMA as 2 flops
    smax = clk.get("sm_max_mhz") or 2070.0
    fig = profile_figures(name)
    ipf = float(fig["fp64_thread_instr_per_face"]) if fig else None
    achieved = ipf * faces_per_launch / (face_ms * 1e-3) if ipf and face_ms > 0 else None
    alg_bytes = (nv + (nv + 2) + nv) * 8 * faces_per_launch  # read U and the primitives, write the fluxes
    hbm_peak = measured_hbm_gbs()
    roof = {"bound": "alu", "achieved": achieved, "peak": probe_inst, "unit": "FP64 inst/s",
            "frac": achieved / probe_inst if achieved else None,
            "traffic": float(fig["dram_bytes_per_launch"]) if fig else None,
            "kernel": "face_kernel (fused characteristic TENO-M face flux)",
            "fp64_inst_per_face": ipf, "faces_per_launch": faces_per_launch, "ms_per_launch": face_ms,
            "launches_timed": face_launches,
            "peak_note": "measured: DFMA probe (8 independent FMA chains per thread) in FP64 instructions/s; "
                         "nominal %d lanes/clock x %.0f MHz = %.3g inst/s" % (FP64_LANES_PER_CLK, smax,
                                                                              FP64_LANES_PER_CLK * smax * 1e6),
            "achieved_note": ("ncu FP64 thread instructions per face from %s (same kernel sources) x faces per "
                              "launch / CUDA-event launch time" % fig["file"]) if fig else
                             "no ncu count for these kernel sources: achieved and traffic unmeasured",
            "hbm": {"algorithmic_bytes_per_launch": alg_bytes,
                    "achieved_gbs": alg_bytes / (face_ms * 1e-3) / 1e9 if face_ms > 0 else None,
                    "peak_gbs": hbm_peak, "frac": (alg_bytes / (face_ms * 1e-3) / 1e9 / hbm_peak)
                    if face_ms > 0 and hbm_peak else None}}
    if fig:
        roof["fp64_pipe_busy_ncu"] = float(fig["fp64_pipe_busy"])
        if "warp_inst_per_face" in fig and face_ms > 0:
            # the SM schedulers' issue slots: 4 warp instructions per clock per SM
            wi = float(fig["warp_inst_per_face"]) * faces_per_launch / (face_ms * 1e-3)
            ipeak = 4 * 152 * smax * 1e6
            roof["issue"] = {"warp_inst_per_face": float(fig["warp_inst_per_face"]), "achieved": wi,
                             "peak": ipeak, "unit": "warp inst/s", "frac": wi / ipeak,
                             "note": "all instructions issued (FP32 screen, integer, loads, FP64) against "
                                     "4 per clock per SM x 152 SMs at the maximum SM clock"}
    fpf = flops_per_face(name)
    if fpf and face_ms > 0:
        roof["oracle_equivalent_rate"] = {
            "flops_per_face": fpf, "flop_per_s": fpf * faces_per_launch / (face_ms * 1e-3),
            "note": "the oracle's op count of the textbook formulation (indicators, comparisons and "
                    "min/max in FP64, no central shortcut) per face over the launch time; the kernel "
                    "retires far fewer FP64 operations, so this rate is not bounded by the FP64 peak"}
    return roof


def batch_roofline(name, faces, stage_ms, probe_flops):
    """Roofline of the batched stage kernel (faces, flux difference and stage combine of
    every problem in one persistent launch), on the same unit as the face kernel's: FP64
    thread instructions per face (ncu, committed under profiles/ for these kernel sources)
    x faces per launch / the CUDA-event launch time, against the DFMA probe's measured
    instruction rate."""
    probe_inst = probe_flops / 2.0
    fig = profile_figures(name, kernel="batch_stage_kernel", sources=BATCH_SOURCES)
    ipf = float(fig["fp64_thread_instr_per_face"]) if fig else None
    achieved = ipf * faces / (stage_ms * 1e-3) if ipf and stage_ms > 0 else None
    roof = {"bound": "alu", "achieved": achieved, "peak": probe_inst, "unit": "FP64 inst/s",
            "frac": achieved / probe_inst if achieved else None,
            "traffic": float(fig["dram_bytes_per_launch"]) if fig else None,
            "kernel": "batch_stage_kernel (persistent faces + flux difference + stage combine)",
            "fp64_inst_per_face": ipf, "faces_per_launch": faces, "ms_per_launch": stage_ms,
            "peak_note": "measured: DFMA probe (8 independent FMA chains per thread) in FP64 instructions/s",
            "achieved_note": ("ncu FP64 thread instructions per face from %s (same kernel sources) x faces per "
                              "launch / CUDA-event launch time" % fig["file"]) if fig else
                             "no ncu count for these kernel sources: achieved and traffic unmeasured"}
    if fig:
        roof["fp64_pipe_busy_ncu"] = float(fig["fp64_pipe_busy"])
    fpf = flops_per_face(name)
    if fpf and stage_ms > 0:
        roof["oracle_equivalent_rate"] = {
            "flops_per_face": fpf, "flop_per_s": fpf * faces / (stage_ms * 1e-3),
            "note": "the oracle's op count of the textbook formulation per face over the launch time; not "
                    "bounded by the FP64 peak"}
    return roof


def measured_hbm_gbs():
    """HBM copy bandwidth of this machine's GPUs (GB/s) from the generated peaks file."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


def run_batch(args):
    """Batched workload: 512 independent seeded 1D Riemann problems, sizes log-uniform
    128..8192, one persistent launch per RK stage, a CUDA graph per RK step, autotuned tiles;
    compared with advancing the same problems by separate plain launches (one context each)."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_13289_gb300 import problems as PB
    from paper_2010_13289_gb300 import tenom as T
    name = args.workload
    nprob, seed, nmin, nmax, K, lim = BATCH_WORKLOADS[name]
    sizes, prims, dxs = PB.batch_riemann(nprob, seed + rank, nmin, nmax)
    B = T.Batch(sizes, dxs, T.make_scheme(K, limiter=lim))
    prim = np.zeros((3, B.total))
    for j in range(nprob):
        prim[:, B.off[j]:B.off[j + 1]] = prims[j]
    U = B.init_state(torch.from_numpy(prim).cuda())
    U0 = U.clone()
    tile, ctas = B.autotune(U)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    B.step(U, nsteps=args.warmup)
    barrier()
    # the batch's working set fits in L2: flush it (a 256 MB write) before every timed step
    # and time the steps alone
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        B.step(U, nsteps=1)
        ev1.record(stream)
        evs.append((ev0, ev1))
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), ws)
    assert B.status() == 0
    value = job_rate(float(B.total) * 3 * args.steps, ws, ms * 1e-3)

    # the same problems advanced by separate plain launches (one context per problem)
    sep_steps = max(1, min(args.steps, 3))
    solvers, Us = [], []
    for n, p, dx in zip(sizes, prims, dxs):
        S = T.Solver((int(n),), (dx,), (T.BC_TRANSMISSIVE,), T.make_scheme(K, limiter=lim))
        solvers.append(S)
        Us.append(S.init_state(torch.from_numpy(p).cuda()))
    for S, u in zip(solvers, Us):
        S.advance(u, 1)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(sep_steps):
        for S, u in zip(solvers, Us):
            S.advance(u, 1)
    e1.record(stream)
    barrier()
    sep_ms = e0.elapsed_time(e1)
    sep_value = float(B.total) * 3 * sep_steps / (sep_ms * 1e-3)
    for S in solvers:
        S.close()

    # stage-kernel time: persistent stage-1 launches with CUDA events (dt from the last step)
    lib = T.lib()
    import ctypes
    reps = 10
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(reps):
        lib.tenom_batch_stage(B._b, 1, ctypes.c_void_p(U.data_ptr()))
    k1.record(stream)
    barrier()
    stage_ms = k0.elapsed_time(k1) / reps

    # end to end: host state in pinned memory -> device, one graph step, device -> host
    host_in = torch.empty((3, B.total), dtype=torch.float64, pin_memory=True)
    host_out = torch.empty_like(host_in)
    host_in.copy_(U0.cpu())
    Ue = torch.empty_like(U)
    e2e_steps = max(1, min(args.steps, 5))
    B.step(Ue.copy_(host_in, non_blocking=True), nsteps=1)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Ue.copy_(host_in, non_blocking=True)
        B.step(Ue, nsteps=1)
        host_out.copy_(Ue, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = float(B.total) * 3 * e2e_steps * ws / e2e_s
    state_bytes = 8 * 3 * B.total

    faces = float(np.sum(sizes + 1))
    roof = batch_roofline(name, faces, stage_ms, T.fp64_peak())
    out = {"metric": "cell-updates/s per RK stage (FP64)", "value": value, "unit": "cell-updates/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded, shaped like the paper's workloads)",
           "config": batch_config(name, ws),
           "launch_config": {"tile": tile, "ctas_per_sm": ctas,
                             "launch": "persistent stage kernel per RK stage, CUDA graph per step"},
           "separate_launches": {"value": sep_value, "unit": "cell-updates/s", "steps": sep_steps,
                                 "speedup_of_batched": value / sep_value},
           "e2e": {"value": e2e, "unit": "cell-updates/s", "h2d_bytes_per_step": state_bytes,
                   "d2h_bytes_per_step": state_bytes},
           "gpu_launches": 6 * args.steps, "roofline": roof, "clocks": clk}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, sample, el = oracle_rate_batch(name, args.ref_seconds or 10.0)
        out["cpu_baseline"] = {"value": r, "unit": "cell-updates/s", "cores": 1, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(out), flush=True)
    B.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def _linear_tape(S, steps, tape):
    from paper_2010_13289_gb300.autograd import _use_linear
    return _use_linear(S, steps, tape)


COST_VARIANTS = [
    # (label, K, limiter, weights): the paper's cost comparison (Section 4) is TENO-M with
    # each limiter against the classical TENO with renormalised weights on the same stencil
    ("TENO6", 6, 0, 1), ("TENO6-M-MP", 6, 0, 0), ("TENO6-M-TVD5", 6, 1, 0), ("TENO6-M-VA", 6, 2, 0),
    ("TENO8A", 8, 0, 1), ("TENO8A-M-MP", 8, 0, 0), ("TENO8A-M-TVD5", 8, 1, 0), ("TENO8A-M-VA", 8, 2, 0),
]


def run_cost_ratios(args):
    """Time per SSP-RK3 step of TENO-M with MP / TVD5 / VA relative to the classical TENO
    (renormalised weights, no limiter) on the 2D 2048^2 broadband field, K = 6 and K = 8.
    The paper quotes MP at about 1.09-1.12x and TVD-type limiters at about 0.99x TENO8A
    (CPU, its own hardware); these are the GPU kernels' ratios."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_13289_gb300 import tenom as T
    shape = (2048, 2048)
    prim, dx = make_prim("broadband_2d_2048_teno6_mp", args.seed)
    primd = torch.from_numpy(prim).cuda()
    stream = torch.cuda.current_stream()
    times = {}
    clocks = ClockSampler(0)
    clocks.start()
    for label, K, lim, w in COST_VARIANTS:
        S = T.Solver(shape, dx, (T.BC_PERIODIC,) * 2, T.make_scheme(K, limiter=lim, weights=w))
        U = S.init_state(primd)
        S.advance(U, args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.advance(U, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        times[label] = e0.elapsed_time(e1) / args.steps
        S.close()
    clk = clocks.stop()
    ncell = float(np.prod(shape))
    out = {"metric": "time per SSP-RK3 step relative to TENO (renormalised weights)", "unit": "ratio",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
           "dtype": "f64", "data": "synthetic (seeded, shaped like the paper's workloads)",
           "config": {"workload": "cost_ratios_2d_2048", "shape": list(shape),
                      "l2": "working set per stage (537 MB) > L2"},
           "ms_per_step": times,
           "cell_updates_per_s": {k: ncell * 3 / (v * 1e-3) for k, v in times.items()},
           "ratios": {k: times[k] / times[k.split("-")[0]] for k in times},
           "paper": {"MP": "1.09-1.12 x TENO8A", "TVD": "0.99 x TENO8A"},
           "clocks": clk}
    print(json.dumps(out), flush=True)


def run_tgv(args):
    """Inviscid Taylor-Green vortex (Section 4.3.1): 64^3 periodic on [0, 2 pi]^3, TENO8A-M-MP,
    CFL 0.4, to t = 10.  Reports the normalised kinetic energy at t = 1..10, its decay
    exponent over t = 5..10 (the paper's reference behaviour is t^-1.2), the relative drift
    of mass, momentum and total energy (conserved to rounding by the flux form), and the
    run's cell-updates/s per RK stage."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_13289_gb300 import problems as PB
    from paper_2010_13289_gb300 import tenom as T
    n, t_final = 64, 10.0
    prim, dx = PB.taylor_green_3d(n)
    S = T.Solver((n, n, n), (dx, dx, dx), (T.BC_PERIODIC,) * 3, T.make_scheme(8, limiter=T.LIM_MP))
    U = S.init_state(torch.from_numpy(prim).cuda())

    def ke(U):
        return float((0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]).sum())

    def totals(U):
        return U.sum(dim=(1, 2, 3)).cpu().numpy()

    ke0, tot0 = ke(U), totals(U)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hist, steps, chunk, dt_est = {}, 0, 25, 0.0
    clocks = ClockSampler(0)
    clocks.start()
    e0.record(stream)
    for target in range(1, int(t_final) + 1):
        while t.item() < target * (1.0 - 1e-14):
            t_before = t.item()
            # whole chunks while they stay short of the target, then single steps (a step
            # past t_end does no update and is not counted)
            m = chunk if dt_est == 0.0 or t_before + 1.5 * chunk * dt_est < target else 1
            S.advance(U, m, t_end=float(target), cfl=0.4, t_dev=t)
            steps += m
            if m == chunk:
                dt_est = (t.item() - t_before) / chunk
        hist[target] = ke(U) / ke0
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    tot = totals(U)
    scale = U.abs().sum(dim=(1, 2, 3)).cpu().numpy()  # momentum sums are zero: measure against sum |m|
    drift = [float(abs(a - b) / s) for a, b, s in zip(tot, tot0, scale)]
    def slope(a, b):
        ts = np.arange(a, b + 1, dtype=float)
        return float(np.polyfit(np.log(ts), np.log([hist[int(x)] for x in ts]), 1)[0])
    out = {"metric": "cell-updates/s per RK stage (FP64)", "value": float(n ** 3) * 3 * steps / (ms * 1e-3),
           "unit": "cell-updates/s", "n_gpus": 1, "steps": steps, "warmup": 0, "ms_per_step": ms / steps,
           "higher_is_better": True, "dtype": "f64", "data": "analytic initial condition (Eq. TGV)",
           "config": {"workload": "tgv_3d_64_teno8_mp", "shape": [n, n, n], "K": 8, "limiter": "MP",
                      "l2": "state 10 MB fits in L2: a whole validation run timed warm, not a kernel figure",
                      "t_final": t_final, "cfl": 0.4},
           "kinetic_energy": {str(k): v for k, v in hist.items()},
           "decay_exponent": {"t5_t10": slope(5, 10), "t7_t10": slope(7, 10)},
           "paper_decay_exponent": "-1.2 (fitting range not stated)",
           "conservation_drift": {"mass": drift[0], "momentum": max(drift[1:4]), "energy": drift[4],
                                  "note": "|change of the sum| / sum of |values|"},
           "clocks": clk}
    print(json.dumps(out), flush=True)
    assert S.status() == 0
    S.close()


def run_le_blanc(args):
    """Le Blanc problem (Section 4.4.2, Eq. Leblanc): 900 cells on [0, 9], gamma = 5/3,
    TENO8-MP with the minmod curvature and beta = 1 and the positivity-preserving flux
    limiter (Section 4.4), CFL 0.4, to t = 6, timed end to end on the device (a 900-cell
    grid is launch-bound: about 16 launches per step).  Also times the limiter's cost on the
    2D 2048^2 broadband workload (step time with the limiter over step time without) and
    512 Le Blanc problems of log-uniform size 128..8192 through the batched launch, with and
    without the limiter."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_13289_gb300 import problems as PB
    from paper_2010_13289_gb300 import tenom as T
    n, t_final = 900, 6.0
    prim, dx = PB.le_blanc_1d(n)
    gam = PB.LE_BLANC_GAMMA
    sch = T.make_scheme(8, limiter=T.LIM_MP, mp_curv=T.CURV_MM, mp_beta=1.0, positivity=T.PP_ON)
    S = T.Solver((n,), (dx,), (T.BC_TRANSMISSIVE,), sch, gamma=gam)
    primd = torch.from_numpy(prim).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    # untimed pass: count the steps to t_final
    U = S.init_state(primd)
    steps = 0
    while t.item() < t_final:
        S.advance(U, 1, t_end=t_final, cfl=0.4, t_dev=t)
        steps += 1
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    clocks.start()
    runs = []
    for _ in range(max(1, args.steps // 5)):
        U = S.init_state(primd)
        t.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.advance(U, steps, t_end=t_final, cfl=0.4, t_dev=t)
        e1.record(stream)
        torch.cuda.synchronize()
        runs.append(e0.elapsed_time(e1))
    assert t.item() == t_final
    Un = U.cpu().numpy()
    p = (gam - 1.0) * (Un[2] - 0.5 * Un[1] ** 2 / Un[0])
    st = S.status()
    S.close()
    # the limiter's cost on a large grid
    prim2, dx2 = make_prim("broadband_2d_2048_teno6_mp", args.seed)
    prim2d = torch.from_numpy(prim2).cuda()
    ms2 = {}
    for label, pp in (("off", T.PP_OFF), ("on", T.PP_ON)):
        S2 = T.Solver((2048, 2048), dx2, (T.BC_PERIODIC,) * 2, T.make_scheme(6, positivity=pp))
        U2 = S2.init_state(prim2d)
        S2.advance(U2, args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S2.advance(U2, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms2[label] = e0.elapsed_time(e1) / args.steps
        S2.close()
    # batched: 512 Le Blanc problems of log-uniform size 128..8192 (each on its own [0, 9]
    # grid), one persistent launch per RK stage, with and without the limiter
    sizes = PB.batch_sizes(512, 4, 128, 8192)
    bprims = [PB.le_blanc_1d(int(m)) for m in sizes]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    bat = {}
    for label, pp in (("off", T.PP_OFF), ("on", T.PP_ON)):
        B = T.Batch(sizes, np.array([d for _, d in bprims]), gamma=gam,
                    scheme=T.make_scheme(8, limiter=T.LIM_MP, mp_curv=T.CURV_MM, mp_beta=1.0, positivity=pp))
        bp = np.zeros((3, B.total))
        for j in range(B.P):
            bp[:, B.off[j]:B.off[j + 1]] = bprims[j][0]
        UB = B.init_state(torch.from_numpy(bp).cuda())
        tile, ctas = B.autotune(UB)
        B.step(UB, nsteps=args.warmup)
        torch.cuda.synchronize()
        evs = []
        for _ in range(args.steps):
            flush.zero_()  # the batch (79 MB) fits in L2
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.step(UB, nsteps=1)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        bms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
        bat[label] = {"ms_per_step": bms, "cell_updates_per_s": float(B.total) * 3 / (bms * 1e-3),
                      "tile": tile, "ctas_per_sm": ctas}
        B.close()
    clk = clocks.stop()
    ms = statistics.median(runs)
    out = {"metric": "cell-updates/s per RK stage (FP64)", "value": float(n) * 3 * steps / (ms * 1e-3),
           "unit": "cell-updates/s", "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": ms / steps,
           "higher_is_better": True, "dtype": "f64", "data": "analytic initial condition (Eq. Leblanc)",
           "config": {"workload": "le_blanc_1d_900_teno8_mp_pp", "shape": [n], "K": 8, "limiter": "MP",
                      "l2": "state 22 KB fits in L2: a whole latency-bound run timed warm; the 2D 2048^2 "
                            "limiter-cost steps (537 MB) exceed L2; before every batched Le Blanc step "
                            "(79 MB) L2 is flushed by a 256 MB write",
                      "mp_curv": "minmod", "mp_beta": 1.0, "positivity": True, "gamma": gam,
                      "t_final": t_final, "cfl": 0.4},
           "time_to_t_final_ms": ms, "timed_runs": len(runs),
           "final_state": {"min_rho": float(Un[0].min()), "min_p": float(p.min()),
                           "finite": bool(np.isfinite(Un).all()), "status_word": int(st)},
           "limiter_cost_2d_2048_teno6_mp": {"ms_per_step_off": ms2["off"], "ms_per_step_on": ms2["on"],
                                             "ratio": ms2["on"] / ms2["off"]},
           "batched_512_le_blanc": {"cells": int(np.sum(sizes)), "steps": args.steps, "limiter_on": bat["on"],
                                    "limiter_off": bat["off"],
                                    "limiter_cost": bat["on"]["ms_per_step"] / bat["off"]["ms_per_step"]},
           "clocks": clk}
    print(json.dumps(out), flush=True)


def measure_adjoint(name, tape="auto", rollout_steps=0, fd_dirs=16, fd_steps=(1e-8, 1e-7)):
    """Adjoint workload: 2D 512^2 broadband field with circular jumps, TENO6-MP, 200 SSP-RK3
    steps at a fixed dt, loss = integral of p over a seeded 64 x 64 window at the end;
    gradient with respect to the initial density through the frozen-branch adjoint with
    checkpoints every 20 steps (torch.autograd); central differences on fd_dirs seeded
    unit directions at each step size in fd_steps.  Returns the figures as a dict: forward
    and backward device time per step (CUDA events on the stream), their ratio, the
    backward pass's cell-updates/s per RK stage, and the central-difference errors."""
    import numpy as np
    import torch
    from paper_2010_13289_gb300 import problems as PB
    from paper_2010_13289_gb300 import tenom as T
    from paper_2010_13289_gb300.autograd import rollout
    n, seed, steps, win_n, every, K, lim = ADJOINT_WORKLOADS[name]
    if rollout_steps:  # shorter rollouts for profiling runs (not the workload's number)
        steps = rollout_steps
    prim, dx = PB.broadband_2d(n, seed)
    rng = np.random.default_rng(seed)
    wy, wx = rng.integers(0, n - win_n, 2)
    win = (slice(int(wy), int(wy) + win_n), slice(int(wx), int(wx) + win_n))
    S = T.Solver((n, n), (dx, dx), (T.BC_PERIODIC,) * 2, T.make_scheme(K, limiter=lim))
    primd = torch.from_numpy(prim).cuda()
    dt = S.max_dt(S.init_state(primd), 0.4).item()
    gam = 1.4
    stream = torch.cuda.current_stream()
    tape = "linear" if _linear_tape(S, min(every, steps), tape) else "flags"

    def loss_of(rho0, grad=False):
        pr = primd.clone()
        pr[0] = rho0
        U0 = S.init_state(pr)
        if grad:
            U0.requires_grad_(True)
        UN = rollout(U0, S, dt, steps, checkpoint_every=every, tape=tape)
        rho, mx, my, E = UN[0], UN[1], UN[2], UN[3]
        p = (gam - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho)
        return (p[win] * dx * dx).sum(), U0

    # warm-up
    L, U0 = loss_of(primd[0], grad=True)
    L.backward()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    L, U0 = loss_of(primd[0], grad=True)
    e1.record(stream)
    L.backward()
    e2.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    fwd_ms = e0.elapsed_time(e1)
    bwd_ms = e1.elapsed_time(e2)
    Ub = U0.grad
    u, v = primd[1], primd[2]
    grad_rho = Ub[0] + u * Ub[1] + v * Ub[2] + 0.5 * (u * u + v * v) * Ub[3]
    gnorm = float(torch.linalg.norm(grad_rho))
    # central differences on seeded unit directions, at each step size
    rng = np.random.default_rng(seed + 16)
    dirs = [rng.normal(size=(n, n)) for _ in range(fd_dirs)]
    fd = {}
    with torch.no_grad():
        for h in fd_steps:
            errs, rel = [], []
            for dv in dirs:
                d = torch.from_numpy(dv).cuda()
                d /= torch.linalg.norm(d)
                Lp, _ = loss_of(primd[0] + h * d)
                Lm, _ = loss_of(primd[0] - h * d)
                fdv = (Lp - Lm).item() / (2 * h)
                ad = float((grad_rho * d).sum())
                errs.append(abs(fdv - ad) / gnorm)
                rel.append(abs(fdv - ad) / max(abs(ad), 1e-300))
            fd["%g" % h] = {"max_err_over_grad_norm": max(errs) if errs else None,
                            "median_err_over_grad_norm": float(np.median(errs)) if errs else None,
                            "median_err_over_directional_derivative": float(np.median(rel)) if rel else None}
    best = min(fd, key=lambda k: fd[k]["max_err_over_grad_norm"]) if fd_dirs > 0 and fd else None
    if fd_dirs == 0:
        fd = {}
    S.close()
    return {"workload": name, "shape": [n, n], "K": K, "limiter": "MP" if lim == 0 else "TVD5", "steps": steps,
            "window": win_n, "checkpoint_every": every, "dt": dt, "tape": tape,
            "adjoint_forward_ratio": bwd_ms / fwd_ms,
            "forward_ms_per_step": fwd_ms / steps, "backward_ms_per_step": bwd_ms / steps,
            "backward_cell_updates_per_s": float(n * n) * 3 * steps / (bwd_ms * 1e-3),
            "loss": L.item(), "grad_norm": gnorm,
            "fd_check": {"directions": fd_dirs, "by_step": fd, "best_step": best,
                         "max_err_over_grad_norm": fd[best]["max_err_over_grad_norm"] if best else None,
                         "note": "central differences of the full forward (cutoff, limiter and LLF switches "
                                 "included) against the frozen-branch adjoint; error / |gradient|"},
            "clocks": clk}


def run_adjoint(args):
    """The adjoint workload on its own line: the backward pass's cell-updates/s per RK stage
    as the value, with the adjoint/forward cost ratio and the central-difference check."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    r = measure_adjoint(args.workload, tape=args.tape, rollout_steps=args.rollout_steps, fd_dirs=args.fd_dirs)
    n = r["shape"][0]
    out = {"metric": "cell-updates/s per RK stage (FP64)", "value": r["backward_cell_updates_per_s"],
           "unit": "cell-updates/s", "n_gpus": 1, "steps": r["steps"], "warmup": 1,
           "ms_per_step": r["backward_ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded, shaped like the paper's workloads)",
           "config": {"workload": args.workload, "shape": [n, n], "K": r["K"], "limiter": r["limiter"],
                      "window": r["window"], "checkpoint_every": r["checkpoint_every"], "dt": r["dt"],
                      "l2": "the forward state (8 MB) fits in L2; the backward streams the recorded "
                            "linearisation (GBs per segment) from HBM",
                      "tape": r["tape"],
                      "pass": "backward (frozen-branch adjoint, segment recomputation included)"},
           "adjoint_forward_ratio": r["adjoint_forward_ratio"],
           "forward_ms_per_step": r["forward_ms_per_step"], "backward_ms_per_step": r["backward_ms_per_step"],
           "loss": r["loss"], "grad_norm": r["grad_norm"], "fd_check": r["fd_check"], "clocks": r["clocks"]}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT,
                    choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS) + sorted(ADJOINT_WORKLOADS) + ["cost_ratios_2d_2048", "tgv_3d_64_teno8_mp", "le_blanc_1d_900_teno8_mp_pp"])
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--ref-seconds", type=float, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--positivity", action="store_true",
                    help="grid workloads: add the positivity-preserving flux limiter to every RK stage")
    ap.add_argument("--tape", default="auto", choices=["auto", "linear", "flags"],
                    help="adjoint workloads: tape of the recomputed segments")
    ap.add_argument("--rollout-steps", type=int, default=0,
                    help="adjoint workloads: rollout length (default: the workload's 200); for profiling runs")
    ap.add_argument("--fd-dirs", type=int, default=16,
                    help="adjoint workloads: finite-difference directions (default 16)")
    ap.add_argument("--decision-log", default=None,
                    help="grid workloads: append the decision statistics as a JSON line to this file")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="default workload: leave out the adjoint workload's figures")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in BATCH_WORKLOADS:
        run_batch(args)
    elif args.workload in ADJOINT_WORKLOADS:
        run_adjoint(args)
    elif args.workload == "cost_ratios_2d_2048":
        run_cost_ratios(args)
    elif args.workload == "tgv_3d_64_teno8_mp":
        run_tgv(args)
    elif args.workload == "le_blanc_1d_900_teno8_mp_pp":
        run_le_blanc(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
