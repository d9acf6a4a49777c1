#!/usr/bin/env python
"""Benchmark of the recycling solvers on the synthetic stand-ins of the
paper's workloads. Default: the porous medium at 192^3 (19-point skewed
stencil, low-conductivity spheres, Dirichlet inlet/outlet), the hybrid of
Sec. 2.4 — rGCROT(40,20) for the first 5 time steps, then rBiCGStab reusing
that k = 20 recycle space — right point Jacobi, relative tolerance 1e-8 on
the true residual, FP64.

One "step" is one solve of one time step (every phase of the solver: stencil
products with the preconditioner, projections onto the recycle space,
Arnoldi orthogonalisation or the BiCGStab recurrences, cycle updates and the
harmonic Ritz recycle update). A hybrid sequence is timed from its first
step: after W warm-up solves the problem starts a new sequence
(rk_problem_reset) and the K timed solves are steps 0 .. K-1. The timed
region runs the production path (captured Arnoldi cycles replayed); the
per-kernel breakdown comes from a separate untimed replay of the same steps
with CUDA events around every launch. Inputs (all right-hand sides) are
resident in HBM before the timed region; every step's working set exceeds
the 129 MB L2. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload porous192|channel128|...] [--precision fp64|df|mixed]
  --impl reference times the CPU oracle (FP64, host cores) on a bounded
  sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading

import numpy as np
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/sec and solver HBM GB/s (% of peak) at rel-res 1e-8; p50/p99 solve latency"
WORKLOADS = {
    # name: (config id, grid edge, mode, m, k)
    "channel128": (2, 128, "rGCROT", 40, 20),
    "porous192": (3, 192, "hybrid", 40, 20),
    "convdiff32": (1, 32, "rGCROT", 30, 10),
    # the channel at 96^3: a smaller case of the same kernels (profiling)
    "channel96": (2, 96, "rGCROT", 40, 20),
    # batched uneven set: 64 porous problems, edges log-uniform in [24, 96]
    "batch64": (4, 0, "hybrid", 40, 10),
    # serving: resident problems, Poisson requests, memory budget with eviction
    "serve": (5, 0, "hybrid", 40, 20),
}
# Matrix-vector products per solve of the channel128 sequence in steady state
# (steps 3-12 of the sequence), measured on the GB300 arm; used only to turn
# the reference arm's per-cycle time into solves/s.
# arithmetic of the path per precision: FP64 operator and true residual with
# double-float basis and projections; the same with the recurrences' products
# in double-float; or with those products in FP32
DTYPES = {"fp64": "f64", "df": "f64+df64", "mixed": "f64+f32-operator"}
MV_PER_SOLVE = {"channel128": {1: 1500.0}, "channel96": {1: 1100.0}, "convdiff32": {1: 60.0},
                "porous192": {1: 1311.0, 2: 911.0}}
# the same with the sub-domain preconditioner (left rGCROT), measured likewise
MV_PER_SOLVE_SD = {"channel128": {1: 513.0}, "porous192": {1: 360.0, 2: 309.0}}
# the preconditioner each workload is defined with: the channel names the
# paper's "Jacobi preconditioner" (the sub-domain one of Sec. 2.1), the
# convection-diffusion case point Jacobi
PRECOND_DEFAULT = {"channel128": "subdomain", "channel96": "subdomain"}
FP64_TOPS = 0.625                    # nominal 1.25 TFLOP/s FP64, one DFMA = 2 flops (fallback)
# where the basis, the recycle space and the projection arithmetic live
BASIS = {"fp64": "f64", "df": "double-float", "mixed": "f64"}
FP32_TOPS = 152 * 128 * 2.07e9 / 1e12  # FP32 lanes x SMs x max SM clock


def fp64_peak_tops():
    """The FP64 fma issue rate of this GPU in T lane operations per second,
    measured by librk's probe (rk_fp64_fma_rate); the nominal rate if the
    probe cannot run."""
    try:
        import ctypes
        import torch
        from paper_1501_03358_gb300 import native
        lib = native.load()
        v = ctypes.c_double()
        native.check(lib.rk_fp64_fma_rate(ctypes.byref(v), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
        return v.value / 1e12, "measured (rk_fp64_fma_rate: FP64 fma chains, CUDA events)"
    except Exception as e:  # pragma: no cover - reported, not hidden
        return FP64_TOPS, f"nominal 1.25 TFLOP/s / 2 (probe failed: {e})"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def rd():
            for line in self.proc.stdout:
                self.lines.append(line.strip())

        self.th = threading.Thread(target=rd, daemon=True)
        self.th.start()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("RK_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _oracle_prec(precond):
    """The oracle's solver arguments for a --precond choice: the sub-domain
    preconditioner is applied from the left in rGCROT (Sec. 2.1)."""
    return dict(left=True, prec="schwarz") if precond == "subdomain" else {}


def subdomain_ops(grid, S, df):
    """Arithmetic of one launch of the sub-domain local-sweep kernel, per
    grown-box cell inside the grid: the first sweep from zero is
    omega (dinv r), each later sweep s = a_0 z + sum_t a_t z_t,
    u = dinv (r - s), z += omega u, and the last sweep runs on owned cells
    only. FP64 variant: FP64 pipe instructions (S + 3 per cell-sweep, 2 in the
    first sweep). Double-float variant: FP32 pipe instructions of its
    error-free transformations (TwoProduct 4, lazy multiply-add 12,
    renormalisation 3, add 11, multiply 7, fused multiply-add 15: 112 per
    cell-sweep for 7 bands, 262 for 19; 14 in the first sweep). Grown-box
    cells inside the grid factor per axis, so the sums over boxes are
    products of per-axis sums."""
    box, ov, sweeps = (16, 8, 8), 1, 5
    dims = (grid.nx, grid.ny, grid.nz)
    g = []
    for n, bsz, per in zip(dims, box, grid.periodic):
        tot = 0
        for c0 in range(0, n, bsz):
            w = min(bsz, n - c0)
            lo = ov if (per or c0 > 0) else 0
            hi = ov if (per or c0 + w < n) else 0
            tot += w + lo + hi
        g.append(tot)
    grown = g[0] * g[1] * g[2]
    if df:
        first, per_cell = 14, (4 + 12 * (S - 1) + 3 * (1 if S == 7 else 3) + 11 + 7 + 15)
    else:
        first, per_cell = 2, S + 3
    return float(first * grown + (sweeps - 2) * per_cell * grown + per_cell * grid.n)


def _standin_space(n, k):
    """k orthonormal columns (normalised indicators of k equal slabs of
    cells) used as both U and C: a recycle space of dimension k for timing
    the oracle's arithmetic only. A U = C does not hold for it, which the
    operation count of a sample does not depend on."""
    C = np.zeros((n, k))
    sl = n // k
    for c in range(k):
        C[c * sl:(c + 1) * sl, c] = 1.0 / np.sqrt(sl)
    return C.copy(), C


def oracle_per_matvec(cfg, precond, m, k, modes, nmv):
    """Seconds per matrix-vector product of the CPU oracle, per solver, on a
    bounded sample of step 0 of the workload at recycle dimension k:
    rGCROT (mode 1) one cycle of nmv Arnoldi steps (recycle update off),
    rBiCGStab (mode 2) nmv products. Returns ({mode: s}, threads, note)."""
    import oracle
    op = oracle.Stencil(cfg.grid, cfg.coef)
    b = cfg.rhs(0)
    U, C = _standin_space(cfg.n, k) if k > 0 else (None, None)
    pk = _oracle_prec(precond)
    out = {}
    for mode in sorted(modes):
        t0 = time.perf_counter()
        if mode == 2:
            _, info = oracle.rbicgstab(op, b, tol=1e-14, U=U, C=C, max_matvec=nmv, max_restarts=0,
                                       prec=pk.get("prec", "jacobi"))
        else:
            _, _, _, info = oracle.rgcrot(op, b, tol=1e-14, m=m, k=k if mode == 1 else 0,
                                          U=U if mode == 1 else None, C=C if mode == 1 else None, update=False,
                                          max_matvec=nmv, **pk)
        out[mode] = (time.perf_counter() - t0) / max(info["matvecs"], 1)
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    note = (f"the oracle on step 0 at recycle dimension {k} (stand-in orthonormal space): "
            + ", ".join(f"{['GMRES', 'rGCROT', 'rBiCGStab'][md]} {nmv} products "
                        f"({1e3 * t:.0f} ms per product)" for md, t in sorted(out.items()))
            + "; the recycle update of each rGCROT cycle is not included")
    return out, threads, note


def cpu_baseline(cfg, args, m, k, tinfo):
    """The oracle as it stands, timed on the host cores on a bounded sample
    (oracle_per_matvec), scaled to solves/s with the products per solve and
    the solver of each timed step measured on the GPU."""
    modes = {i["mode_used"] for i in tinfo}
    per, threads, note = oracle_per_matvec(cfg, args.precond, m, k, modes, args.cpu_sample_matvecs)
    secs = sum(per[i["mode_used"]] * i["matvecs"] for i in tinfo)
    return {"value": len(tinfo) / secs, "unit": "solves/s", "cores": threads, "kind": "oracle",
            "sample": note + f"; solves/s = {len(tinfo)} / sum over the timed steps of (products of the step x "
                             f"seconds per product of its solver)"}


def run_reference(args, ws, rank):
    """The reference arm: the CPU oracle (FP64, host cores) on the same
    workload. Each step is a bounded sample of the solve of that time step
    (the solver the hybrid uses at that step, args.cpu_sample_matvecs
    products at recycle dimension k), converted to solves/s with the
    products per solve that the GPU arm measured for that solver."""
    if rank != 0:
        return
    table = MV_PER_SOLVE_SD if args.precond == "subdomain" else MV_PER_SOLVE
    mvs = table.get(args.workload)
    if mvs is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no measured products per solve for "
                          f"{args.workload} with the {args.precond} preconditioner"}), flush=True)
        return
    from problems import make_config
    cid, edge, mode, m, k = WORKLOADS[args.workload]
    cfg = make_config(cid, size=edge)
    hybrid = mode == "hybrid"
    step_mode = [(1 if (not hybrid or t < args.hybrid_switch) else 2) for t in range(args.steps)]
    t_all = time.perf_counter()
    # warm-up: one sample of each solver (loads the C loops, touches the operator)
    per, threads, note = oracle_per_matvec(cfg, args.precond, m, k, set(step_mode), args.cpu_sample_matvecs)
    times = []
    for t in range(args.steps):
        md = step_mode[t]
        p1, _, _ = oracle_per_matvec(cfg, args.precond, m, k, {md}, args.cpu_sample_matvecs)
        times.append(p1[md] * mvs[md])
    total = time.perf_counter() - t_all
    value = args.steps / sum(times)
    sample = (note + "; each step: the same sample of its solver, solves/s = steps / sum of (seconds per product "
              "x products per solve of that solver measured on the GPU arm: "
              + ", ".join(f"{['GMRES', 'rGCROT', 'rBiCGStab'][md]} {v:.0f}" for md, v in sorted(mvs.items())) + ")")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "grid": [edge] * 3, "stencil": cfg.S,
                       "solver": (f"hybrid rGCROT({m},{k}) for {args.hybrid_switch} steps -> rBiCGStab(k={k})"
                                  if hybrid else f"{mode}({m},{k})"), "tol": 1e-8,
                       "precond": args.precond, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed_solves(prob, rhs, kw, stream, x, keep=None):
    """Solve the right-hand sides in order on `stream` with CUDA events around
    each solve and around the whole run. Returns (ms, [(ms, info)])."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ev, infos = [], []
    e0.record(stream)
    for i, b in enumerate(rhs):
        ts = torch.cuda.Event(enable_timing=True)
        te = torch.cuda.Event(enable_timing=True)
        ts.record(stream)
        x.zero_()
        _, info = prob.solve(b, out=x, **kw)
        te.record(stream)
        if keep is not None:
            keep.append(x.clone())
        ev.append((ts, te))
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), [(a.elapsed_time(b), inf) for (a, b), inf in zip(ev, infos)]


def _phase_summary(per, hbm_peak):
    """Per phase of a hybrid sequence (mode_used 1 = rGCROT, 2 = rBiCGStab):
    solves, time, products, modelled bytes and their HBM fraction."""
    out = {}
    for mode, name in ((0, "GMRES"), (1, "rGCROT"), (2, "rBiCGStab")):
        sel = [(ms, i) for ms, i in per if i["mode_used"] == mode]
        if not sel:
            continue
        ms = sum(s[0] for s in sel)
        by = sum(s[1]["model_bytes"] for s in sel)
        gbs = by / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        out[name] = {"solves": len(sel), "ms": ms, "ms_per_solve": ms / len(sel),
                     "matvecs_per_solve": statistics.mean(s[1]["matvecs"] for s in sel),
                     "model_GBps": gbs, "frac_of_hbm": gbs / hbm_peak}
    return out


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    from problems import make_config
    from paper_1501_03358_gb300 import Context, Problem

    cid, edge, mode, m, k = WORKLOADS[args.workload]
    cfg = make_config(cid, size=edge, seed=None if rank == 0 else 20150113 + cid + 1000 * rank)
    W, K = args.warmup, args.steps
    stream = torch.cuda.current_stream()
    ctx = Context()
    prob = Problem(ctx, cfg.grid, torch.from_numpy(cfg.coef))
    x = torch.zeros(cfg.n, dtype=torch.float64, device="cuda")
    side = "left" if (args.precond == "subdomain" and mode != "rBiCGStab") else "right"
    kw = dict(tol=1e-8, m=m, k=k, mode=mode, max_matvec=args.max_matvec, hybrid_switch=args.hybrid_switch,
              precision=args.precision, precond=args.precond, precond_side=side)
    hybrid = mode == "hybrid"
    P = 0
    if hybrid:
        # a hybrid sequence is timed from its first step: steps 0 .. K-1 (the
        # rGCROT phase builds the recycle space, the rBiCGStab phase reuses it);
        # the warm-up runs W steps of the same sequence with the switch moved
        # so that both phases run, then the problem starts a new sequence
        t0s = 0
        seq = list(range(K))
        warm = list(range(W))
    else:
        # sequence pre-roll (untimed, before warm-up): the first solves of an
        # rGCROT sequence build the recycle space and may stall until it holds
        # the slowest modes; run them with a matvec cap, stopping at the first
        # one that converges, so that the timed steps are steady-state solves
        for t in range(args.preroll):
            x.zero_()
            _, info = prob.solve(torch.from_numpy(cfg.rhs(t)).cuda(), out=x,
                                 **dict(kw, max_matvec=args.preroll_matvec))
            P += 1
            if info["status"] == 0:
                break
        t0s = P
        warm = list(range(t0s, t0s + W))
        seq = list(range(t0s + W, t0s + W + K))
    steps_needed = sorted(set(warm) | set(seq) | set(range(seq[-1] + 1, seq[-1] + 1 + K)) if not hybrid
                          else set(warm) | set(seq))
    # all right-hand sides resident in HBM before timing; pinned host copies for e2e
    rhs_host = {t: torch.from_numpy(cfg.rhs(t)).pin_memory() for t in steps_needed}
    rhs_dev = {t: h.to("cuda", non_blocking=True) for t, h in rhs_host.items()}
    wkw = dict(kw, hybrid_switch=max(1, min(args.hybrid_switch, W - 1))) if hybrid else kw
    for t in warm:
        x.zero_()
        prob.solve(rhs_dev[t], out=x, **wkw)
    if hybrid:
        prob.reset()
    torch.cuda.synchronize()
    # ---- timed region: the production path (captured cycles replayed, no
    # per-kernel events), device events on the solve stream
    sampler = ClockSampler(local)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    xs_keep = [] if (args.vs_fp64 and args.precision != "fp64") else None
    ms, per = _timed_solves(prob, [rhs_dev[t] for t in seq], kw, stream, x, keep=xs_keep)
    barrier(ws)
    clocks = sampler.stop()
    tinfo = [p[1] for p in per]
    lat_ms = [p[0] for p in per]
    ms_max = max_over_ranks(ws, ms)
    # ---- end to end through the public API: pinned host b -> device, solve,
    # device -> pinned host x, every step
    if hybrid:
        prob.reset()
        e2e_steps = seq
    else:
        e2e_steps = list(range(seq[-1] + 1, seq[-1] + 1 + K))
    # one pinned host buffer per step (the same bytes as reusing one): with
    # variants they hold the headline precision's solutions for comparison
    keep_host = bool(args.variants) and hybrid
    xhs = [torch.empty(cfg.n, dtype=torch.float64).pin_memory() for _ in (e2e_steps if keep_host else [0])]
    bdev = torch.empty(cfg.n, dtype=torch.float64, device="cuda")
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for si, t in enumerate(e2e_steps):
        bdev.copy_(rhs_host[t], non_blocking=True)
        x.zero_()
        prob.solve(bdev, out=x, **kw)
        xhs[si if keep_host else 0].copy_(x, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier(ws)
    e2e_s = max_over_ranks(ws, e2e_s)
    # ---- kernel classes: a separate, untimed replay of the same steps with
    # CUDA events around every launch (captured cycles are not used then)
    if hybrid:
        prob.reset()
    prob.profile(True)
    prof_ms, prof_per = _timed_solves(prob, [rhs_dev[t] for t in (seq if hybrid else e2e_steps)], kw, stream, x)
    prof = prob.profile_read()
    prob.profile(False)

    peaks, peak_src = load_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fp64_peak, fp64_src = fp64_peak_tops()
    # DRAM traffic of one launch over its algorithmic bytes, from one ncu
    # capture (dram__bytes_read.sum + dram__bytes_write.sum) of the same
    # kernels on the 96^3 channel: dots at nq = 40 (335.2 MB for 297.3 MB),
    # update at nq = 58 (437.9 MB for 438.8 MB). Every operand is far larger
    # than L2 at both sizes, so the ratio carries over.
    traffic_ratio = {"dots": 335.2 / 297.3, "update": 437.9 / 438.8}
    # dominant kernel class by time (profiled replay)
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, d = dom
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
    roof = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak,
            "traffic": (traffic_ratio[dname] * d["bytes"] / max(d["launches"], 1)
                        if dname in traffic_ratio else None),
            "traffic_source": "ncu DRAM bytes / algorithmic bytes on the 96^3 channel x this run's "
                              "algorithmic bytes per launch" if dname in traffic_ratio else None,
            "peak_source": peak_src, "timing": "CUDA events around each launch in an untimed replay of the "
                                               "timed steps",
            "launches": d["launches"], "avg_launch_us": 1000.0 * d["ms"] / max(d["launches"], 1),
            "bytes_per_launch": d["bytes"] / max(d["launches"], 1)}
    if d.get("fma", 0.0) > 0 and d["ms"] > 0 and dname not in ("subdomain_local", "subdomain_df"):
        # the FP64 kernels of the class issue their fused multiply-adds on the
        # FP64 pipe: report that bound beside the HBM one, and the tighter as
        # the class's roofline
        alu = d["fma"] / (d["ms"] * 1e-3) / 1e12
        hbm = dict(roof)
        if alu / fp64_peak > roof["frac"]:
            roof.update({"bound": "alu", "achieved": alu, "peak": fp64_peak, "unit": "T FP64 fma/s",
                         "frac": alu / fp64_peak, "peak_source": fp64_src, "fma_per_launch": d["fma"] / d["launches"]})
            roof["hbm"] = {k: hbm[k] for k in ("achieved", "peak", "unit", "frac", "traffic")}
        else:
            roof["alu"] = {"achieved": alu, "peak": fp64_peak, "unit": "T FP64 fma/s", "frac": alu / fp64_peak}
    if dname in ("subdomain_local", "subdomain_df"):
        # bound by the arithmetic pipe: FP64 instructions against the measured
        # FP64 rate, or, for the double-float variant, FP32 instructions
        # against 128 FP32 lanes per SM per clock (152 SMs at 2.07 GHz)
        dfk = dname == "subdomain_df"
        ops = subdomain_ops(cfg.grid, cfg.S, dfk)
        peak = FP32_TOPS if dfk else fp64_peak
        ach = ops * d["launches"] / (d["ms"] * 1e-3) / 1e12 if d["ms"] > 0 else 0.0
        traffic = (63.8 + 2.8) * 1e6 / 96 ** 3 * cfg.grid.n
        roof.update({"bound": "alu", "achieved": ach, "peak": peak,
                     "unit": "T FP32 instr/s" if dfk else "T FP64 instr/s", "frac": ach / peak,
                     "traffic": traffic,
                     "traffic_source": "ncu DRAM bytes of one launch on the 96^3 channel x cells of this grid",
                     "peak_source": "FP32 lanes x SMs x max SM clock" if dfk else fp64_src,
                     "instr_per_launch": ops})
    total_model = sum(i["model_bytes"] for i in tinfo)
    solver_gbs = total_model / (ms * 1e-3) / 1e9
    launches = int(sum(v["launches"] for v in prof.values()))
    value = ws * K / (ms_max * 1e-3)
    mv = [i["matvecs"] for i in tinfo]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": args.workload, "grid": [edge] * 3, "stencil": cfg.S,
                   "solver": (f"hybrid rGCROT({m},{k}) for {args.hybrid_switch} steps -> rBiCGStab(k={k})"
                              if hybrid else f"{mode}({m},{k})"),
                   "precision": args.precision, "basis": BASIS[args.precision], "precond": args.precond,
                   "precond_side": side, "tol": 1e-8, "preroll_steps": P,
                   "preroll_matvec_cap": args.preroll_matvec if not hybrid else None,
                   "sequence_steps_timed": [seq[0], seq[-1]], "l2": "inputs larger than L2",
                   "solid_fraction": cfg.solid_fraction if hybrid else None,
                   "parallelism": "replicas" if ws > 1 else "single"},
        "solver_hbm_gbs": solver_gbs, "solver_hbm_frac": solver_gbs / hbm_peak,
        "phases": _phase_summary(per, hbm_peak),
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99))},
        "per_step": [{"step": t, "mode": ["GMRES", "rGCROT", "rBiCGStab"][i["mode_used"]], "ms": round(l, 3),
                      "matvecs": i["matvecs"], "relres": i["relres_true"]} for t, l, i in zip(seq, lat_ms, tinfo)],
        "matvecs_per_solve": statistics.mean(mv), "relres_max": max(i["relres_true"] for i in tinfo),
        "all_converged": all(i["status"] == 0 for i in tinfo),
        "roofline": roof,
        "kernel_classes": {kname: {"ms": round(v["ms"], 3), "launches": v["launches"],
                                   "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None,
                                   "hbm_frac": (v["bytes"] / (v["ms"] * 1e-3) / 1e9 / hbm_peak) if v["ms"] > 0 else None,
                                   "fp64_frac": (v.get("fma", 0.0) / (v["ms"] * 1e-3) / 1e12 / fp64_peak)
                                   if v["ms"] > 0 and v.get("fma", 0.0) > 0 else None}
                           for kname, v in prof.items() if v["launches"]},
        "fp64_fma_peak_tops": fp64_peak, "fp64_fma_peak_source": fp64_src,
        "kernel_classes_pass": {"ms": prof_ms, "note": "untimed replay with per-launch events"},
        "gpu_launches": launches,
        "gpu_launches_source": "library launches counted in the profiled replay of the same steps",
        "e2e": {"value": ws * len(e2e_steps) / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 8 * cfg.n,
                "d2h_bytes_per_step": 8 * cfg.n},
        "clocks": clocks,
    }
    if args.variants and hybrid:
        # the same timed steps with the other precisions (side by side with the
        # headline; timed pass only, fresh problem each)
        var = {}
        for vp in [v for v in args.variants.split(",") if v in DTYPES and v != args.precision]:
            vprob = Problem(ctx, cfg.grid, torch.from_numpy(cfg.coef))
            vkw = dict(kw, precision=vp)
            for t in warm:
                x.zero_()
                vprob.solve(rhs_dev[t], out=x, **dict(vkw, hybrid_switch=wkw["hybrid_switch"]))
            vprob.reset()
            torch.cuda.synchronize()
            vkeep = []
            vms, vper = _timed_solves(vprob, [rhs_dev[t] for t in seq], vkw, stream, x, keep=vkeep)
            # per step ||x_variant - x|| / ||x|| against the headline
            # precision's solution of the same step (the end-to-end pass's
            # host copies; with the fp64 headline that is the FP64 path the
            # parity tests hold to the oracle)
            diffs = []
            for si, xv in enumerate(vkeep):
                xr = xhs[si]
                diffs.append(float(torch.linalg.norm(xv.cpu() - xr) / torch.linalg.norm(xr)))
            del vkeep
            var[vp] = {"value": len(seq) / (vms * 1e-3), "ms_per_step": vms / len(seq), "dtype": DTYPES[vp],
                       "basis": BASIS[vp], "phases": _phase_summary(vper, hbm_peak),
                       "relres_max": max(i["relres_true"] for _, i in vper),
                       "all_converged": all(i["status"] == 0 for _, i in vper),
                       "x_rel_diff_vs_" + args.precision: {"per_step": diffs, "max": max(diffs)}}
            vprob.close()
        line["variants"] = var
    if xs_keep is not None:
        # the same sequence in FP64 (a second problem): per-step difference of
        # the solutions, relative to the FP64 one
        ref = Problem(ctx, cfg.grid, torch.from_numpy(cfg.coef))
        errs = []
        fkw = dict(kw, precision="fp64")
        for i, t in enumerate(seq):
            x.zero_()
            ref.solve(rhs_dev[t], out=x, **fkw)
            errs.append(float(torch.linalg.norm(xs_keep[i] - x) / torch.linalg.norm(x)))
        ref.close()
        line["error_vs_fp64"] = {"per_step": errs, "max": max(errs),
                                 "reference": "the same sequence solved by the fp64 path of this library"}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, args, m, k, tinfo)
    if rank == 0:
        print(json.dumps(line), flush=True)
    prob.close()
    ctx.close()


def _percentiles(v):
    return {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99))}


def run_batch(args, ws, rank, local):
    """Config 4: 64 independent porous problems (edges log-uniform in
    [24, 96] per axis, solid fraction U[0.1, 0.4], skew U[0, 15] deg), one
    right-hand side each per time step, hybrid rGCROT(40,10) -> rBiCGStab
    (switch after 5 steps), solved together by rk_solve_batch. One bench step
    is one time step of all 64 sequences; value = solves/s."""
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    from problems.configs import config4_problem, CONFIG_SEED_BASE
    from paper_1501_03358_gb300 import Context, Problem, solve_batch
    _, _, mode, m, k = WORKLOADS["batch64"]
    seed = None if rank == 0 else CONFIG_SEED_BASE + 4 + 1000 * rank
    cfgs = [config4_problem(p, seed=seed) for p in range(args.nprob)]
    W, K = args.warmup, args.steps
    prec = args.precision or "mixed"
    ctx = Context()
    kw = dict(tol=1e-8, m=m, k=k, mode=mode, hybrid_switch=5, max_matvec=args.max_matvec, precision=prec)
    rhs_host = [[torch.from_numpy(c.rhs(t)).pin_memory() for c in cfgs] for t in range(W + K)]
    rhs_dev = [[h.to("cuda", non_blocking=True) for h in row] for row in rhs_host]
    xs = [torch.zeros(c.n, dtype=torch.float64, device="cuda") for c in cfgs]
    xh = [torch.empty(c.n, dtype=torch.float64).pin_memory() for c in cfgs]
    bdev = [torch.empty(c.n, dtype=torch.float64, device="cuda") for c in cfgs]
    stream = torch.cuda.current_stream()

    def arm(host_copies=False):
        """Fresh problems, W untimed steps of their sequences, then the K
        timed steps (CUDA events on the caller's stream; with host_copies the
        right-hand sides come from pinned host memory and the solutions go
        back to it inside the timed region)."""
        probs = [Problem(ctx, c.grid, torch.from_numpy(c.coef)) for c in cfgs]
        for t in range(W):
            for x in xs:
                x.zero_()
            solve_batch(probs, rhs_dev[t], outs=xs, nthreads=args.threads, **kw)
        torch.cuda.synchronize()
        barrier(ws)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        lat, infos = [], []
        t_host = time.perf_counter()
        a0.record(stream)
        for t in range(W, W + K):
            ts = torch.cuda.Event(enable_timing=True)
            te = torch.cuda.Event(enable_timing=True)
            ts.record(stream)
            if host_copies:
                for i in range(len(cfgs)):
                    bdev[i].copy_(rhs_host[t][i], non_blocking=True)
            for x in xs:
                x.zero_()
            _, inf = solve_batch(probs, bdev if host_copies else rhs_dev[t], outs=xs, nthreads=args.threads, **kw)
            if host_copies:
                for i in range(len(cfgs)):
                    xh[i].copy_(xs[i], non_blocking=True)
            te.record(stream)
            lat.append((ts, te))
            infos.extend(inf)
        a1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_host
        barrier(ws)
        for pp in probs:
            pp.close()
        return a0.elapsed_time(a1), [a.elapsed_time(b) for a, b in lat], infos, wall

    # the batched phase's launch shapes are tuned once per workload shape (the
    # first replays time each candidate); tune them here, untimed, on a
    # throwaway set of the same problems running rBiCGStab
    tprobs = [Problem(ctx, c.grid, torch.from_numpy(c.coef)) for c in cfgs]
    for x in xs:
        x.zero_()
    os.environ["RK_BATCHED_BICG"] = "1"
    try:
        solve_batch(tprobs, rhs_dev[0], outs=xs, nthreads=args.threads, **dict(kw, mode="rBiCGStab", k=0))
    finally:
        os.environ.pop("RK_BATCHED_BICG", None)
    torch.cuda.synchronize()
    for pp in tprobs:
        pp.close()
    sampler = ClockSampler(local)
    sampler.start()
    ms, lat_ms, infos, _ = arm()
    clocks = sampler.stop()
    ms = max_over_ranks(ws, ms)
    _, e2e_lat, e2e_inf, e2e_s = arm(host_copies=True)
    e2e_s = max_over_ranks(ws, e2e_s)
    # the same steps with the rBiCGStab iterations in the batched phase (one
    # launch per iteration phase over all problems): the comparison
    os.environ["RK_BATCHED_BICG"] = "1"
    try:
        pms, plat, pinf, _ = arm()
    finally:
        os.environ.pop("RK_BATCHED_BICG", None)
    ntot = sum(c.n for c in cfgs)
    model = sum(i["model_bytes"] for i in infos)
    peaks, peak_src = load_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = model / (ms * 1e-3) / 1e9
    nsol = len(cfgs) * K
    line = {
        "metric": METRIC, "value": ws * nsol / (ms * 1e-3), "unit": "solves/s", "n_gpus": ws, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[prec], "data": "synthetic",
        "config": {"workload": "batch64", "problems": len(cfgs), "cells_total": ntot,
                   "edges": "log-uniform [24, 96] per axis", "stencil": 19, "solver": f"{mode}({m},{k})",
                   "hybrid_switch": 5, "precision": prec, "tol": 1e-8, "threads": args.threads or min(len(cfgs), 16),
                   "sequence_steps_timed": [W, W + K - 1], "l2": "inputs larger than L2",
                   "parallelism": "replicas" if ws > 1 else "single",
                   "executor": "rk_solve_batch: host worker threads, one CUDA stream each (the default; "
                               "batched_phase_executor: the rBiCGStab iterations of all problems in one launch "
                               "per phase over a (problem, block) work list, RK_BATCHED_BICG=1)"},
        "solver_hbm_gbs": achieved, "solver_hbm_frac": achieved / hbm_peak,
        "latency_ms": dict(_percentiles(lat_ms), unit="one time step of all problems"),
        "matvecs_per_solve": statistics.mean(i["matvecs"] for i in infos),
        "relres_max": max(i["relres_true"] for i in infos),
        "all_converged": all(i["status"] == 0 for i in infos),
        "roofline": {"bound": "hbm", "kernel": "whole solver (modelled bytes, concurrent streams)",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "traffic": None, "peak_source": peak_src},
        "gpu_launches": None,
        "e2e": {"value": ws * nsol / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 8 * ntot,
                "d2h_bytes_per_step": 8 * ntot},
        "clocks": clocks,
    }
    modes = ["GMRES", "rGCROT", "rBiCGStab"]
    step_mode = [modes[infos[t * len(cfgs)]["mode_used"]] for t in range(K)]
    line["per_step"] = [{"step": W + t, "mode": step_mode[t], "ms": round(lat_ms[t], 2),
                         "ms_batched_phase": round(plat[t], 2)} for t in range(K)]
    line["batched_phase_executor"] = {
        "solves_per_s": ws * nsol / (max_over_ranks(ws, pms) * 1e-3), "ms_per_step": pms / K,
        "same_products": [i["matvecs"] for i in pinf] == [i["matvecs"] for i in infos]}
    line["e2e"]["same_products"] = [i["matvecs"] for i in e2e_inf] == [i["matvecs"] for i in infos]
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        c0 = cfgs[0]
        op = oracle.Stencil(c0.grid, c0.coef)
        tt = time.perf_counter()
        _, _, _, inf = oracle.rgcrot(op, c0.rhs(0), tol=1e-14, m=m, k=k, max_matvec=2 * m)
        per_cell_mv = (time.perf_counter() - tt) / max(inf["matvecs"], 1) / c0.n
        step_mv_cells = sum(i["matvecs"] * cfgs[j % len(cfgs)].n for j, i in enumerate(infos)) / K
        threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        line["cpu_baseline"] = {"value": len(cfgs) / (per_cell_mv * step_mv_cells), "unit": "solves/s",
                                "cores": threads, "kind": "oracle",
                                "sample": f"two rGCROT({m},{k}) cycles of problem 0 ({c0.n} cells): "
                                          f"{per_cell_mv * 1e9:.1f} ns per matvec per cell; solves/s = problems / "
                                          f"(that x sum over problems of cells x matvecs per step measured above)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_switch_sweep(args, ws, rank, local):
    """The hybrid's switch-step experiment (Sec. 4.3, Table 8) replayed on the
    porous configuration: for each switch step n, a fresh problem solves the
    first T steps of the time-step sequence with the hybrid (rGCROT(40,20)
    for solves 1..n, then rBiCGStab with the recycle space frozen); reports
    per n the summed solve time (CUDA events), products, and whether every
    solve converged. Right-hand sides are generated once, resident in HBM."""
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    from problems import make_config
    from paper_1501_03358_gb300 import Context, Problem
    cfg = make_config(3, size=args.sweep_edge)
    T = args.sweep_steps
    rhs = [torch.from_numpy(cfg.rhs(t)).cuda() for t in range(T)]
    ctx = Context()
    stream = torch.cuda.current_stream()
    kw = dict(tol=1e-8, m=40, k=20, mode="hybrid", max_matvec=args.max_matvec, precision=args.precision or "fp64",
              precond=args.precond, precond_side="left" if args.precond == "subdomain" else "right")
    x = torch.zeros(cfg.n, dtype=torch.float64, device="cuda")
    results = []
    for n in range(1, args.sweep_max + 1):
        prob = Problem(ctx, cfg.grid, torch.from_numpy(cfg.coef))
        per = []
        for t in range(T):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            x.zero_()
            e0.record(stream)
            _, info = prob.solve(rhs[t], out=x, hybrid_switch=n, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            per.append((e0.elapsed_time(e1), info))
        results.append({"switch": n, "ms_total": sum(p[0] for p in per),
                        "ms_rgcrot": sum(p[0] for p in per if p[1]["mode_used"] == 1),
                        "ms_rbicgstab": sum(p[0] for p in per if p[1]["mode_used"] == 2),
                        "matvecs": [p[1]["matvecs"] for p in per],
                        "all_converged": all(p[1]["status"] == 0 for p in per),
                        "relres_max": max(p[1]["relres_true"] for p in per)})
        prob.close()
    best = min((r for r in results if r["all_converged"]), key=lambda r: r["ms_total"], default=None)
    line = {"metric": "hybrid switch-step sweep: summed solve time of the first T steps per switch step n",
            "unit": "ms", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "porous", "grid": [args.sweep_edge] * 3, "stencil": cfg.S, "steps": T,
                       "solver": "hybrid rGCROT(40,20) -> rBiCGStab", "tol": 1e-8, "precond": args.precond,
                       "precision": kw["precision"], "solid_fraction": getattr(cfg, "solid_fraction", None)},
            "results": results, "best_switch": best["switch"] if best else None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_kernel_probe(args, local):
    """One kernel of the path alone, for profilers: `dots2` = the fused
    Arnoldi inner products [Q^T p, Q^T w, p^T p, p^T w, w^T w] of one step
    (rk_arnoldi_dots, FP64, the tensor-core engine) on a row-contiguous N(0, 1) basis of probe-nq
    columns and probe-n rows; prints the largest normwise difference from
    the FP64-pipe kernel on the same operands (the tensor-core engine is
    selected by RK_TC_DOTS=1)."""
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    from paper_1501_03358_gb300 import Context
    ctx = Context()
    gen = torch.Generator(device="cuda").manual_seed(1501)
    n, nq = args.probe_n, args.probe_nq
    Q = torch.randn(nq, n, dtype=torch.float64, device="cuda", generator=gen)
    p = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
    w = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
    out = None
    os.environ["RK_TC_DOTS"] = "1"
    for _ in range(args.probe_reps):
        out = ctx.arnoldi_dots(Q, p, w)
    torch.cuda.synchronize()
    os.environ["RK_TC_DOTS"] = "0"
    ref = ctx.arnoldi_dots(Q, p, w)
    os.environ.pop("RK_TC_DOTS", None)
    qn = torch.linalg.norm(Q, dim=1)
    pn, wn = torch.linalg.norm(p), torch.linalg.norm(w)
    scale = torch.cat([qn * pn, qn * wn, torch.stack([pn * pn, pn * wn, wn * wn])])
    diff = float(torch.max(torch.abs(out - ref) / scale))
    print(json.dumps({"kernel_probe": "dots2", "n": n, "nq": nq, "reps": args.probe_reps,
                      "max_normwise_diff_vs_fp64_pipe": diff}), flush=True)
    ctx.close()


def run_serve(args, ws, rank, local):
    """Serving loop (config 5): resident problems of mixed sizes (channel and
    porous generators alternating over --serve-edges), each request the next
    right-hand side of one problem, arriving as a Poisson process at
    --rate-frac times the measured single-stream capacity; continuous
    admission (serving.Server: --slots worker streams, requests start as
    slots and memory free up) under a device-memory budget with LRU eviction
    of recycle spaces (exact spill to pinned host memory). Reports solves/s
    and p50/p99 latency (completion - arrival) for the hybrid recycling
    solver (mixed precision) and for plain FP64 GMRES(40) without recycling
    on the same arrivals. Problems of one edge and generator share their
    coefficients (generated once); right-hand sides are b_t = F_a + 0.05 t F_b
    from a pool of smoothed divergence fields per edge."""
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    from problems import make_config
    from problems.configs import porous_problem
    from problems.fields import rng_for, face_velocity, divergence, normalise_div
    from paper_1501_03358_gb300 import Context
    from paper_1501_03358_gb300.serving import Server
    edges = [int(e) for e in args.serve_edges.split(",")]
    ops = {}
    for i in range(args.nprob):
        e = edges[i % len(edges)]
        kind = "channel" if (i // len(edges)) % 2 == 0 else "porous"
        if (e, kind) in ops:
            continue
        if kind == "channel":
            c = make_config(2, size=e)
            ops[(e, kind)] = (c.grid, c.coef, c)
        else:
            gr, coef, _ = porous_problem((e, e, e), 0.25, 10.0, 20150113 + 5 + e, max_attempts=200_000)
            ops[(e, kind)] = (gr, coef, None)
    fields = {}
    for (e, kind), (gr, coef, c) in ops.items():
        if e in fields:
            continue
        ones = np.ones(e)
        vol = np.ones((e, e, e))
        fl = []
        for j in range(3):
            u = face_velocity(gr, 4.0, rng_for(20150113 + 5, 7, 1000 * e + j), walls=(False, True, True))
            fl.append(np.ascontiguousarray(normalise_div(divergence(gr, ones, ones, ones, *u), vol).reshape(-1)))
        fields[e] = fl
    probs = []
    for i in range(args.nprob):
        e = edges[i % len(edges)]
        kind = "channel" if (i // len(edges)) % 2 == 0 else "porous"
        probs.append((e, kind))
    nreq = args.requests
    rng = np.random.default_rng(20150113 + 55 + rank)
    order = [int(i) for i in rng.integers(0, len(probs), nreq)]
    ctx = Context()

    def rhs(i, t):
        fl = fields[probs[i][0]]
        b = fl[i % 3] + 0.05 * t * fl[(i + 1) % 3]
        if probs[i][1] == "channel":
            b = b.copy()
            b[0] = 0.0  # the pinned cell of the channel operator
        return torch.from_numpy(b)

    budget = int(args.budget_gb * 1e9)

    def serve(kw, rate, nwarm=1):
        srv = Server(ctx, budget, kw, slots=args.slots)
        for i, (e, kind) in enumerate(probs):
            gr, coef, _ = ops[(e, kind)]
            srv.add(i, gr, torch.from_numpy(coef))
        # warm-up (untimed): the first steps of every problem's sequence
        for t in range(nwarm):
            for i in range(len(probs)):
                srv.submit(i, rhs(i, t).cuda())
        srv.drain()
        srv.done.clear()
        seen = [nwarm] * len(probs)
        reqs = []
        for i in order:
            reqs.append((i, rhs(i, seen[i]).pin_memory()))
            seen[i] += 1
        arr = np.cumsum(rng.exponential(1.0 / rate, nreq)) if rate else np.zeros(nreq)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nxt = 0
        while nxt < nreq or srv.queue or srv.in_flight():
            now = time.perf_counter() - t0
            while nxt < nreq and arr[nxt] <= now:
                srv.submit(reqs[nxt][0], reqs[nxt][1].to("cuda", non_blocking=True), arrival=t0 + arr[nxt])
                nxt += 1
            srv.poll()
            wait = (arr[nxt] - (time.perf_counter() - t0)) if nxt < nreq else 1.0
            if wait > 0:
                srv.wait_any(timeout=min(max(wait, 0.0005), 1.0))
        wall = time.perf_counter() - t0
        lat = [1e3 * (r.finish - r.arrival) for r in srv.done]
        res = {"solves_per_s": len(srv.done) / wall, "latency_ms": _percentiles(lat),
               "converged": sum(1 for r in srv.done if r.info["status"] == 0), "requests": len(srv.done),
               "evictions": srv.evictions, "restores": srv.restores, "max_in_flight": srv.max_in_flight,
               "matvecs_per_solve": statistics.mean(r.info["matvecs"] for r in srv.done),
               "relres_max": max(r.info["relres_true"] for r in srv.done)}
        srv.close()
        return res

    cap_mv = args.max_matvec
    rkw = dict(tol=1e-8, m=40, k=20, mode="hybrid", hybrid_switch=5, max_matvec=cap_mv,
               precision=args.precision or "mixed")
    gkw = dict(tol=1e-8, m=40, k=0, mode="GMRES", max_matvec=cap_mv, precision="fp64")
    cap = serve(rkw, None)                      # burst: every request at t = 0
    rates = [float(r) for r in args.rate_fracs.split(",")]
    sweep = {}
    for rf in rates:
        sweep[str(rf)] = {"hybrid_recycling": serve(rkw, rf * cap["solves_per_s"])}
        if not args.no_gmres:
            sweep[str(rf)]["gmres40_fp64"] = serve(gkw, rf * cap["solves_per_s"])
    head = sweep[str(rates[0])]["hybrid_recycling"]
    line = {
        "metric": METRIC, "value": head["solves_per_s"], "unit": "solves/s", "n_gpus": ws, "steps": nreq,
        "warmup": len(probs), "ms_per_step": 1e3 / max(head["solves_per_s"], 1e-9), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32-operator", "data": "synthetic",
        "config": {"workload": "serve", "problems": len(probs), "edges": edges, "requests": nreq,
                   "budget_bytes": budget, "slots": args.slots, "rate_fracs_of_capacity": rates,
                   "solver": "hybrid rGCROT(40,20)->rBiCGStab, mixed", "tol": 1e-8, "max_matvec": cap_mv,
                   "admission": "continuous (slots x streams), footprint reservation, LRU eviction"},
        "latency_ms": head["latency_ms"], "burst_capacity": cap, "sweep": sweep,
        "roofline": None, "gpu_launches": None,
        "e2e": {"value": head["solves_per_s"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="porous192", choices=sorted(WORKLOADS))
    ap.add_argument("--kernel-probe", choices=["dots2"], default=None,
                    help="run one kernel of the path alone on synthetic operands (a small case for profilers)")
    ap.add_argument("--probe-n", type=int, default=1 << 22, help="kernel probe: rows")
    ap.add_argument("--probe-nq", type=int, default=40, help="kernel probe: basis columns")
    ap.add_argument("--probe-reps", type=int, default=4, help="kernel probe: calls")
    ap.add_argument("--hybrid-switch", type=int, default=5, help="hybrid: rGCROT solves before the switch")
    ap.add_argument("--variants", default="df,mixed",
                    help="hybrid workloads: other precisions timed on the same steps, reported beside the headline "
                         "with their per-step solution difference from it")
    ap.add_argument("--vs-fp64", type=int, default=1,
                    help="precision df/mixed: also solve the timed steps with the fp64 path and report the "
                         "per-step difference of the solutions (1 = on)")
    ap.add_argument("--cpu-sample-matvecs", type=int, default=6,
                    help="CPU oracle sample: products per solver")
    ap.add_argument("--max-matvec", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--preroll", type=int, default=12,
                    help="untimed sequence steps before warm-up (stops at the first converged one)")
    ap.add_argument("--preroll-matvec", type=int, default=4000, help="matvec cap of each pre-roll solve")
    ap.add_argument("--precision", default=None, choices=["fp64", "df", "mixed"],
                    help="fp64: FP64 operator, double-float projections; df: double-float operator in the "
                         "recurrences; mixed: FP32 inner operator (A11). "
                         "Default fp64 for the single-sequence workloads, mixed for batch64 and serve")
    ap.add_argument("--precond", default=None, choices=["jacobi", "subdomain"],
                    help="jacobi: right point Jacobi; subdomain: Sec. 2.1's sub-domain Jacobi preconditioner "
                         "(5 damped local sweeps on overlapping 16x8x8 boxes, one global sweep), left in rGCROT. "
                         "Default: subdomain for the channel workloads, jacobi otherwise")
    ap.add_argument("--switch-sweep", action="store_true",
                    help="replay the hybrid switch-step sweep (Table 8) on the porous configuration")
    ap.add_argument("--sweep-edge", type=int, default=192, help="switch sweep: grid edge")
    ap.add_argument("--sweep-steps", type=int, default=10, help="switch sweep: time steps per switch step")
    ap.add_argument("--sweep-max", type=int, default=9, help="switch sweep: largest switch step")
    ap.add_argument("--nprob", type=int, default=None, help="problems (batch64: 64; serve: 12)")
    ap.add_argument("--threads", type=int, default=0, help="rk_solve_batch worker threads (0: min(n, 16))")
    ap.add_argument("--requests", type=int, default=64, help="serve: number of timed requests")
    ap.add_argument("--serve-edges", default="64,96,128,192,256", help="serve: grid edges, cycled over problems")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serve: device memory budget (GB)")
    ap.add_argument("--rate-fracs", default="0.25,0.5,1,2", help="serve: arrival rates / burst capacity")
    ap.add_argument("--slots", type=int, default=4, help="serve: concurrent solve slots (streams)")
    ap.add_argument("--no-gmres", action="store_true", help="serve: skip the GMRES(40) arm")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_init()
    if args.nprob is None:
        args.nprob = 64 if args.workload == "batch64" else 32
    if args.precond is None:
        args.precond = "subdomain" if args.switch_sweep else PRECOND_DEFAULT.get(args.workload, "jacobi")
    if args.impl == "reference":
        if args.workload in ("batch64", "serve"):
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single sequences; "
                                  "batch64 reports its oracle baseline in cpu_baseline"}), flush=True)
        else:
            run_reference(args, ws, rank)
    elif args.workload == "batch64":
        run_batch(args, ws, rank, local)
    elif args.workload == "serve":
        run_serve(args, ws, rank, local)
    elif args.switch_sweep:
        run_switch_sweep(args, ws, rank, local)
    elif args.kernel_probe:
        run_kernel_probe(args, local)
    else:
        if args.precision is None:
            args.precision = "fp64"
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
