#!/usr/bin/env python
"""Benchmark: ms per zero-beta MHD step at 256x256x512 (FP64, with the FP32-inner / FP64
refinement form beside it) and PCG bandwidth against the HBM roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one full predictor-corrector step (coefficients, two momentum-force passes, two
semi-implicit PCG solves, the constrained-transport induction and the viscous PCG solve) on the
synthetic flux-rope workload (seeded dipole + 5-mode perturbation + twisted flux rope, seeded
5-mode velocity). Every input vector is 268-805 MB, larger than the 129 MB L2, so no L2 flush is
needed between steps. Kernel durations come from CUDA events recorded on the grid's stream
around each launch inside the timed region.

With N > 1 (torchrun) every rank runs an independent replica of the workload on its own GPU;
the step has no data-path exchange between replicas. --impl reference times the CPU oracle (its
OpenMP timing build on every host core, and one thread beside it) on a bounded sample of the same
workload, scaled by the oracle's own PCG iteration count, with whole oracle steps measured at
32x32x64 and 128x128x256 as anchors, and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "fluxrope_256x256x512"
METRIC = "ms/zero-beta step, PCG HBM GB/s (% peak) at 256x256x512: FP64 vs mixed"
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070  # 2 DFMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz = 1.259 TFLOP/s
# algorithmic work of one scaled CG iteration per cell (3 components):
#   bytes: x, r, p read + written once each = 6 passes x 3 x 8 B (FP64), x 4 B (FP32)
#   FP64 flops of the SpMV kernel: the 6 neighbour multiply-adds of the unit-diagonal 7-point
#   stencil plus the dot product's multiply-add = 14 flops per component (the two phi neighbours
#   share one coefficient, so the kernel issues 7 FP64 instructions for these 14 flops)
SPMV_FLOPS_PER_CELL = 3 * (2 * 6 + 2)
PCG_BYTES_PER_CELL = {"fp64": 6 * 3 * 8, "fp32": 6 * 3 * 4}
# DRAM bytes (read + write) per cell of one k_spmv_dot<double,2,3> launch, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum = 369.8 MB + 172.4 MB) on the flux-rope physics at
# 160x160x320 (8.19M cells, vectors larger than L2); scaled by the cell count for the roofline's
# traffic field. 48 B per cell is algorithmic: the extra reads are i+-1 planes re-read from DRAM,
# which costs nothing while the FP64 pipe binds.
SPMV64_DRAM_BYTES_PER_CELL = (369.818624e6 + 172.424192e6) / (160 * 160 * 320)
SPMV_BYTES_PER_CELL = {"fp64": 2 * 3 * 8, "fp32": 2 * 3 * 4}
# FP64 instructions per cell of one FP64 CG iteration (3 components): the p update 2 per component
# (x += ax p, p = r + beta p), the stencil 7 per component, the update 7.5 per cell (r -= alpha q
# and r~^2 per component, the cell sum, <r~, r~> and sum dg r~^2); against 2 DFMA per clock per SM
FP64_INSTR_PER_CELL_ITER = 6 + 21 + 7.5
FP64_INSTR_PEAK = 2 * 152 * 2.070e9
# one RKL2 stage per cell (3 components, difference form): the 7-point K stencil of D_{j-1} folded
# with the mu term (1 multiply, 1 add, 5 FMAs), the nv D_{j-2} and ly0 terms (2 FMAs) = 16 flops
# per component, plus the per-cell share of the 6 stage coefficients (3 flops); bytes: D_{j-1},
# D_{j-2} and ly0 read, D_j written = 4 x 3 x 8 B
STS_FLOPS_PER_CELL = 3 * 16 + 3
STS_BYTES_PER_CELL = 4 * 3 * 8
# FP64 PC2 line kernel per cell: x, p, r, q read, x, r, z written (7 x 3 x 8 B) plus 1/dt (8 B,
# shared by the three components)
PC2_LINE_BYTES_PER_CELL = 7 * 3 * 8 + 8
# resistivity of the explicit-against-implicit comparison (the workload itself has eta = 0)
RES_ETA = 1e-3


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def gen_state(name, grid=None):
    """Workload inputs; `grid` ("NRxNTxNP") keeps the workload's physics on another grid size."""
    from paper_1811_02605_gb300 import inputs as I
    if grid is None:
        return I.workload(name)
    nr, nt, np_ = (int(x) for x in grid.lower().split("x"))
    w = dict(I.WORKLOADS[name])
    d0 = w["desc"]
    w["desc"] = I.GridDesc(nr, nt, np_, d0.r0, d0.r1, d0.stretch)
    return w, I.initial_state(w["desc"], w["index"], w["rope"])


# ----------------------------------------------------------------------------------------------
# reference arm and CPU baseline: the C oracle (its OpenMP timing build) on the host's cores
# ----------------------------------------------------------------------------------------------
def host_cores():
    return os.cpu_count() or 1


def oracle_sample(w, st, iters_per_step, pcg_iters=3, threads=0):
    """Time the oracle's explicit passes once and `pcg_iters` PCG iterations on the step's SI
    system with `threads` threads of its OpenMP timing build (0: every host core), and scale to one
    step with `iters_per_step` PCG iterations. Returns (ms, sample text, threads used, parts)."""
    import numpy as np
    import oracle as O
    used = O.set_threads(threads if threads > 0 else host_cores())
    d = w["desc"]
    g = O.Grid.from_desc(d, omp=True)
    v = np.stack([st["vr"], st["vt"], st["vp"]])
    t0 = time.perf_counter()
    c = g.coeffs(v, st["br"], st["bt"], st["bp"], nu=w["nu"], cfl=w["cfl"])
    t1 = time.perf_counter()
    b = g.force(v, st["br"], st["bt"], st["bp"], c["dt"])
    t2 = time.perf_counter()
    er, et, ep = g.efield_edges(v, st["br"], st["bt"], st["bp"], w["eta"])
    g.ct(er, et, ep, c["dt"], st["br"], st["bt"], st["bp"])
    t3 = time.perf_counter()
    g.pcg(c["alpha_si"], b, fixed_iters=1)
    t4 = time.perf_counter()
    g.pcg(c["alpha_si"], b, fixed_iters=1 + pcg_iters)
    t5 = time.perf_counter()
    per_iter = (t5 - t4) / pcg_iters
    setup = (t4 - t3) - per_iter  # residual, diagonal and one iteration
    parts = dict(coeffs_ms=1e3 * (t1 - t0), force_ms=1e3 * (t2 - t1), induction_ms=1e3 * (t3 - t2),
                 solve_setup_ms=1e3 * setup, pcg_iteration_ms=1e3 * per_iter)
    ms = 1e3 * ((t1 - t0) + 2 * (t2 - t1) + (t3 - t2) + 3 * setup + iters_per_step * per_iter)
    sample = (f"oracle (OpenMP timing build, {used} threads) at {d.nr}x{d.nt}x{d.np}: one coefficient, force "
              f"and induction pass and {pcg_iters + 2} PCG iterations timed ({t5 - t0:.1f} s), scaled to one "
              f"step of {iters_per_step} PCG iterations (2 force passes, 3 solve set-ups)")
    return ms, sample, used, parts


def oracle_full_step(name, grid, threads=0):
    """One whole oracle step (OpenMP timing build): (ms, PCG iterations, threads, its sampled model)."""
    import oracle as O
    w, st = gen_state(name, grid)
    used = O.set_threads(threads if threads > 0 else host_cores())
    g = O.Grid.from_desc(w["desc"], omp=True)
    t0 = time.perf_counter()
    _, info = g.step(st, nu=w["nu"], eta=w["eta"], cfl=w["cfl"], tol=w["tol"])
    ms = 1e3 * (time.perf_counter() - t0)
    iters = int(sum(info["iters"]))
    model, _, _, _ = oracle_sample(w, st, iters, pcg_iters=3, threads=threads)
    return dict(ms=round(ms, 1), pcg_iters=iters, threads=used, sampled_model_ms=round(model, 1),
                model_over_measured=round(model / ms, 3))


def oracle_iteration_counts(name):
    """The oracle's own PCG iteration count for the first step of the workload (recorded by
    tests/golden/make_golden.py), or None."""
    p = os.path.join(ROOT, "tests", "golden", f"{name}_oracle_step1.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    return int(sum(rec["info"]["iters"]))


def cpu_baseline_iters(args, fallback):
    """PCG iterations per step by which both oracle figures are scaled, and where the number
    comes from."""
    rec = oracle_iteration_counts(args.workload) if args.grid is None else None
    if rec is not None:
        return rec, f"the oracle's own first step at this size (tests/golden/{args.workload}_oracle_step1.json)"
    return int(fallback), "no oracle record for this grid: the count given"


def run_reference(args):
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            dist.destroy_process_group()
            return
    w, st = gen_state(args.workload, args.grid)
    d = w["desc"]
    iters, iters_src = cpu_baseline_iters(args, args.ref_iters)
    vals = []
    sample = ""
    parts = {}
    used = 1
    for s in range(args.warmup + args.steps):
        ms, sample, used, parts = oracle_sample(w, st, iters, pcg_iters=3)
        if s >= args.warmup:
            vals.append(ms)
    value = sum(vals) / len(vals)
    one, _, _, _ = oracle_sample(w, st, iters, pcg_iters=2, threads=1)
    anchors = {}
    if not args.no_anchors:
        anchors["32x32x64"] = oracle_full_step("parity_32x32x64", None)
        anchors["128x128x256"] = oracle_full_step(args.workload, "128x128x256")
    cpu = dict(value=round(value, 3), unit="ms/step", cores=used, kind="oracle", sample=sample,
               single_thread_value=round(one, 1), iters_per_step=iters, iters_source=iters_src,
               parts_ms={k: round(v, 2) for k, v in parts.items()},
               measured_full_steps=anchors,
               note="extrapolated from the timed sample by the iteration count; measured_full_steps are whole "
                    "oracle steps on smaller grids with the same sampled model beside them")
    line = dict(impl="reference", metric=METRIC, value=round(value, 3), unit="ms/step", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=round(value, 3), higher_is_better=False,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload, grid=f"{d.nr}x{d.nt}x{d.np}", precision="fp64",
                            l2="inputs larger than L2"),
                cpu_baseline=cpu,
                e2e=dict(value=round(value, 3), unit="ms/step", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if not args.all_entries:
            # N replicas of the same workload: the headline and the end-to-end leg are the scaling
            # measurement; the per-configuration entries are the single-GPU line's (N GPUs stay held
            # for about a minute of timed work instead of several)
            args.no_mixed = args.no_cg = args.no_pc2 = args.no_res = args.no_sts = True
    from paper_1811_02605_gb300 import build as B
    B.build()
    import paper_1811_02605_gb300 as P

    w, st0 = gen_state(args.workload, args.grid)
    d = w["desc"]
    N = d.nr * d.nt * d.np
    stream = torch.cuda.Stream()
    g = P.mhd_grid_create(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch, stream)

    def dev_state():
        with torch.cuda.stream(stream):
            return {k: torch.from_numpy(v).to("cuda", non_blocking=False) for k, v in st0.items()}

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def run(precision, steps, warmup, profile, inner_tol=1e-5, restart=1, snapshot=None, sts=0, variant=0, pc=0,
            eta=None, res=0):
        ds = dev_state()
        torch.cuda.synchronize()
        f = P.make_fields(ds["br"], ds["bt"], ds["bp"], ds["vr"], ds["vt"], ds["vp"])
        prm = P.make_params(nu=w["nu"], eta=w["eta"] if eta is None else eta, cfl=w["cfl"], tol=w["tol"],
                            precision=precision, inner_tol=inner_tol, max_outer=200, max_iter=20000,
                            mixed_restart=restart, viscosity_sts=sts, pcg_variant=variant, preconditioner=pc,
                            resistivity_implicit=res)
        for _ in range(warmup):
            st, info = P.mhd_step(g, prm, f)
            if st != P.MHD_OK:
                raise RuntimeError(f"warm-up step failed: {P.STATUS_NAMES[st]} {P.mhd_last_error(g)}")
        barrier()
        if snapshot is not None:  # state at the start of the timed region, for the end-to-end leg
            for k in ds:
                snapshot[k] = ds[k].cpu().pin_memory()
        P.mhd_profile_enable(g, profile)
        infos = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            barrier()
            e0.record(stream)
            for _ in range(steps):
                st, info = P.mhd_step(g, prm, f)
                if st != P.MHD_OK:
                    raise RuntimeError(f"step failed: {P.STATUS_NAMES[st]} {P.mhd_last_error(g)}")
                infos.append(info)
            e1.record(stream)
            barrier()
        ms = e0.elapsed_time(e1) / steps
        prof = P.mhd_profile_read(g)
        P.mhd_profile_enable(g, False)
        return ms, infos, prof, clk.summary(), ds

    def maxr(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    hbm, peak_src = peaks()
    # ---- FP64 (headline): K steps as a user runs them (CUDA graphs of PCG iterations, no per-launch
    # events), then a short profiled run of the same workload for the per-kernel times
    snap = {}
    ms64, infos64u, _, clk64, ds64 = run(P.PREC_FP64, args.steps, args.warmup, False, snapshot=snap)
    ms64 = maxr(ms64)
    it64 = sum(sum(i["iters"]) for i in infos64u) / len(infos64u)
    psteps = max(1, min(args.steps, args.profile_steps))
    ms64p, infos64, prof64, clk64p, ds64p = run(P.PREC_FP64, psteps, 1, True)
    ms64p = maxr(ms64p)
    spmv_ms, spmv_n = prof64["spmv64"]
    pcg64_ms = sum(prof64[k][0] for k in ("pupdate64", "spmv64", "update64"))
    pcg64_n = prof64["spmv64"][1]
    it64_total = max(sum(sum(i["iters"]) for i in infos64), 1)   # CG iterations actually run
    # share of the FP64 PCG time spent in the viscous solves (by iteration count)
    visc_it = sum(i["iters"][2] for i in infos64)
    visc64_ms = pcg64_ms * visc_it / it64_total / len(infos64)
    form64, _ = P.mhd_grid_kernel_forms(g)
    overlap64 = form64 == -2
    # ms per FP64 CG iteration, unprofiled: a fixed-count solve of the first step's SI system (the
    # kernels of the overlapped form run concurrently, so their per-launch times do not add up)
    ds_i = dev_state()
    f_i = P.make_fields(ds_i["br"], ds_i["bt"], ds_i["bp"], ds_i["vr"], ds_i["vt"], ds_i["vp"])
    c_i = P.mhd_step_coeffs(g, P.make_params(nu=w["nu"], cfl=w["cfl"]), f_i)
    b_i = torch.empty((3, d.nr, d.nt, d.np), dtype=torch.float64, device="cuda")
    P.mhd_force(g, f_i, c_i["dt"], b_i)
    x_i = torch.zeros_like(b_i)
    iter_n = 200
    P.pcg_solve(g, c_i["alpha_si"], b_i, x_i, P.make_params(tol=1e-30, max_iter=iter_n))
    x_i.zero_()
    barrier()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    P.pcg_solve(g, c_i["alpha_si"], b_i, x_i, P.make_params(tol=1e-30, max_iter=iter_n))
    eb.record(stream)
    barrier()
    iter64_ms = maxr(ea.elapsed_time(eb)) / iter_n
    del ds_i, f_i, b_i, x_i
    if overlap64:
        # one stencil launch per component, each overlapping the next component's p update
        spmv_avg = spmv_ms / max(spmv_n, 1)
        spmv_tflops = SPMV_FLOPS_PER_CELL / 3 * N / (spmv_avg * 1e-3) / 1e12
    else:
        spmv_avg = spmv_ms / max(min(spmv_n, sum(sum(i["iters"]) for i in infos64)), 1)
        spmv_tflops = SPMV_FLOPS_PER_CELL * N / (spmv_avg * 1e-3) / 1e12
    pcg64_gbs = PCG_BYTES_PER_CELL["fp64"] * N * it64_total / (pcg64_ms * 1e-3) / 1e9
    if overlap64:   # concurrent kernels: the unprofiled iteration time, not the sum of launch times
        pcg64_gbs = PCG_BYTES_PER_CELL["fp64"] * N / (iter64_ms * 1e-3) / 1e9
    # per-kernel DRAM passes of a 3-component FP64 vector (8 B x 3 per cell per pass): the p update
    # also adds the previous alpha p to x (r, p, x in; p, x out), the update reads r, q and writes r
    kernels64 = {}
    for k, passes in (("pupdate64", 5), ("spmv64", 2), ("update64", 3)):
        ms_k, n_k = prof64[k]
        if n_k:
            avg = ms_k / it64_total
            gbs = passes * 24 * N / (avg * 1e-3) / 1e9
            kernels64[k] = dict(avg_launch_ms=round(avg, 4), bytes_per_cell=passes * 24, gbs=round(gbs, 1),
                                frac_of_hbm=round(gbs / hbm, 4))
    roof = dict(bound="alu", achieved=round(spmv_tflops, 4), peak=round(FP64_PEAK_TFLOPS / 1e3, 4),
                unit="TFLOP/s", frac=round(spmv_tflops / (FP64_PEAK_TFLOPS / 1e3), 4),
                traffic=(int(SPMV64_DRAM_BYTES_PER_CELL * N) if prof64["pupdate64"][1] and not overlap64 else None),
                traffic_algorithmic=int(SPMV_BYTES_PER_CELL["fp64"] * N / (3 if overlap64 else 1)),
                kernel=("k_spmv_dotc<2> (one component per launch, beside the next component's p update)"
                        if overlap64 else "k_spmv_dot<double,2,3>"),
                avg_launch_ms=round(spmv_avg, 4),
                iteration=dict(fp64_instr_per_cell=FP64_INSTR_PER_CELL_ITER, ms=round(iter64_ms, 4),
                               fp64_pipe_frac=round(FP64_INSTR_PER_CELL_ITER * N / (iter64_ms * 1e-3)
                                                    / FP64_INSTR_PEAK, 4),
                               form=form64,
                               note=f"the whole FP64 CG iteration (p update, stencil, update), timed unprofiled "
                                    f"over a {iter_n}-iteration solve of the first step's SI system, against the "
                                    f"part's FP64 instruction rate"),
                peak_source="2 DFMA/clk/SM x 152 SMs x 2.07 GHz (nominal FP64 rate of the part)")
    # ---- mixed (FP32 inner PCG, FP64 refinement)
    def mixed_entry(inner_tol, restart):
        msm, infosm, profm, clkm, dsm = run(P.PREC_MIXED, args.steps, args.warmup, True, inner_tol, restart)
        msm = maxr(msm)
        pcg32_ms = sum(profm[k][0] for k in ("pupdate32", "spmv32", "update32", "pspmv32", "pfold32", "rupd32",
                                              "cgr32", "cgu32"))
        pcg32_n = max(sum(sum(i["iters"]) for i in infosm), 1)   # inner CG iterations actually run
        pcg32_gbs = PCG_BYTES_PER_CELL["fp32"] * N * pcg32_n / (pcg32_ms * 1e-3) / 1e9
        fused = profm["pspmv32"][1] > 0
        recompute = profm["pfold32"][1] > 0 or profm["cgr32"][1] > 0
        tiled = not fused and not recompute and profm["pupdate32"][1] == 0
        # per-kernel DRAM passes of a 3-component FP32 vector (4 B x 3 per cell per pass)
        # split form: the p update also adds the previous alpha p to x (r, p, x in; p, x out) and the
        # update kernel reads r, q and writes r; fused form: r, p, x in, p, x, q out, then the update;
        # recompute pair: r, p_old in, p out; then p, r in, r out, and every second iteration x,
        # p_prev in, x out (4.5 on average); single-reduction pair: r in; then r, p_old in, p, r out,
        # and every second iteration x in and out (5 on average)
        kb = {"spmv32": 3 if tiled else 2, "update32": 5 if tiled else 3, "pupdate32": 5, "pspmv32": 6,
              "pfold32": 3, "rupd32": 4.5, "cgr32": 1, "cgu32": 5}
        kernels = {}
        for k in ("pupdate32", "spmv32", "pspmv32", "update32", "pfold32", "rupd32", "cgr32", "cgu32"):
            ms_k, n_k = profm[k]
            if n_k:
                avg = ms_k / pcg32_n   # one launch per inner iteration that ran
                gbs = kb[k] * 12 * N / (avg * 1e-3) / 1e9
                kernels[k] = dict(avg_launch_ms=round(avg, 4), bytes_per_cell=kb[k] * 12, gbs=round(gbs, 1),
                                  frac_of_hbm=round(gbs / hbm, 4))
        err = {k: float(torch.linalg.norm(dsm[k] - ds64[k]) / torch.linalg.norm(ds64[k])) for k in ds64}
        return dict(inner_tol=inner_tol, refinement=("restarted" if restart else "reliable updates"),
                    ms_per_step=round(msm, 3), speedup_vs_fp64=round(ms64 / msm, 3),
                    pcg_iters_per_step=sum(sum(i["iters"]) for i in infosm) / len(infosm),
                    outer_per_step=sum(sum(i["outer"]) for i in infosm) / len(infosm),
                    max_relres=max(max(i["relres"]) for i in infosm),
                    pcg_gbs=round(pcg32_gbs, 1), pcg_frac_of_hbm=round(pcg32_gbs / hbm, 4),
                    kernels=kernels, fp32_kernels=("plane-marching pair (A: p update + stencil, B: stencil + "
                                                   "update)" if tiled else
                                                   "single-reduction pair (residual kernel: gamma, delta, "
                                                   "stop norm; update kernel: p, A p, r, x every second "
                                                   "iteration)" if profm["cgr32"][1] > 0 else
                                                   "recompute pair (p update folded into <p, Ap>; r update "
                                                   "with Ap recomputed, x every second iteration)" if recompute
                                                   else
                                                   "p update folded into the stencil, then the update" if fused
                                                   else "split (p update, stencil, update)"),
                    rel_l2_vs_fp64_gpu_after_steps=err, clocks=clkm,
                    kernel_ms={k: round(v[0], 3) for k, v in profm.items() if v[1]})

    mixed = mixed_reliable = None
    if not args.no_mixed:
        mixed = mixed_entry(1e-5, 1)            # FP32 inner PCG to 1e-5, restarted FP64 refinement
        mixed_reliable = mixed_entry(0.1, 0)    # FP32 CG with reliable FP64 updates every 10x

    # ---- viscosity by RKL2 super time-stepping (the SI solves unchanged)
    def sts_entry(precision, inner_tol=0.1, restart=0):
        mss, infoss, profs, clks, dss = run(precision, psteps, 1, True, inner_tol, restart, sts=1)
        mss = maxr(mss)
        stages = sum(i["iters"][2] for i in infoss)
        st_ms, st_n = profs["sts"]
        per_stage = st_ms / max(stages, 1)
        tflops = STS_FLOPS_PER_CELL * N / (per_stage * 1e-3) / 1e12
        gbs = STS_BYTES_PER_CELL * N / (per_stage * 1e-3) / 1e9
        err = {k: float(torch.linalg.norm(dss[k] - ds64p[k]) / torch.linalg.norm(ds64p[k])) for k in ds64p}
        return dict(si_precision=("fp64" if precision == P.PREC_FP64 else "mixed, reliable updates, inner_tol "
                                  f"{inner_tol}"),
                    ms_per_step=round(mss, 3), speedup_vs_fp64=round(ms64 / mss, 3),
                    stages_per_step=stages / len(infoss),
                    si_pcg_iters_per_step=sum(i["iters"][0] + i["iters"][1] for i in infoss) / len(infoss),
                    sts_ms_per_step=round(st_ms / len(infoss), 3), ms_per_stage=round(per_stage, 4),
                    stage_roofline=dict(bound="alu", achieved=round(tflops, 4), peak=round(FP64_PEAK_TFLOPS / 1e3, 4),
                                        unit="TFLOP/s", frac=round(tflops / (FP64_PEAK_TFLOPS / 1e3), 4),
                                        gbs=round(gbs, 1), frac_of_hbm=round(gbs / hbm, 4)),
                    pcg_viscous_ms_per_step_fp64=round(visc64_ms, 3),
                    rel_l2_vs_fp64_pcg_viscosity_after_steps=err, clocks=clks,
                    kernel_ms={k: round(v[0], 3) for k, v in profs.items() if v[1]})

    # ---- FP64 with the single-reduction (Chronopoulos-Gear) PCG form
    pcg_cg = None
    if not args.no_cg:
        msc, infosc, profc, clkc, dsc = run(P.PREC_FP64, psteps, 1, True, variant=1)
        msc = maxr(msc)
        itc = sum(sum(i["iters"]) for i in infosc) / len(infosc)
        c_ms = profc["spmv64"][0] + profc["update64"][0]
        c_n = profc["spmv64"][1]
        pcg_cg = dict(ms_per_step=round(msc, 3), speedup_vs_fp64=round(ms64 / msc, 3), pcg_iters_per_step=itc,
                      ms_per_iteration=round(c_ms / max(sum(sum(i["iters"]) for i in infosc), 1), 4),
                      ms_per_iteration_hestenes_stiefel=round(iter64_ms, 4),
                      kernels_per_iteration=2,
                      rel_l2_vs_fp64_after_steps={k: float(torch.linalg.norm(dsc[k] - ds64p[k]) /
                                                           torch.linalg.norm(ds64p[k])) for k in ds64p},
                      clocks=clkc, kernel_ms={k: round(v[0], 3) for k, v in profc.items() if v[1]})

    # ---- PC2: block-Jacobi ILU(0) on phi lines (FP64), alone and with RKL2 viscosity
    # mixed PC2 runs reliable updates at inner tol 1e-3: a PC2 iteration is cheap against an FP64
    # correction, so fewer corrections win (the refinement study's PC2 rows: 1e-3 fastest)
    def pc2_entry(sts_flag, precision=P.PREC_FP64):
        msp, infosp, profp, clkp, dsp = run(precision, psteps, 1, True, inner_tol=1e-3, restart=0,
                                            sts=sts_flag, pc=1)
        msp = maxr(msp)
        if precision == P.PREC_MIXED:
            n_it = max(sum(sum(i["iters"]) for i in infosp), 1)
            return dict(viscosity="PCG+PC2", si_precision="mixed, reliable updates, inner_tol 1e-3",
                        ms_per_step=round(msp, 3), speedup_vs_fp64=round(ms64 / msp, 3),
                        pcg_iters_per_step=[sum(i["iters"][q] for i in infosp) / len(infosp) for q in range(3)],
                        outer_per_step=sum(sum(i["outer"]) for i in infosp) / len(infosp),
                        max_relres=max(max(i["relres"]) for i in infosp),
                        kernel_ms_per_iteration={k: round(profp[k][0] / n_it, 4)
                                                 for k in ("pupdate32", "spmv32", "pspmv32", "pc2") if profp[k][1]},
                        rel_l2_vs_fp64_after_steps={k: float(torch.linalg.norm(dsp[k] - ds64p[k]) /
                                                             torch.linalg.norm(ds64p[k])) for k in ds64p},
                        clocks=clkp, kernel_ms={k: round(v[0], 3) for k, v in profp.items() if v[1]})
        # per iteration: summed kernel time over the CG iterations actually run (launches that return
        # at once after convergence last a few microseconds and are not iterations)
        n_it = sum(sum(i["iters"][:2] if sts_flag else i["iters"]) for i in infosp)
        per_it = {k: round(profp[k][0] / max(n_it, 1), 4) for k in ("pupdate64", "spmv64", "pc2")}
        line_ms = profp["pc2"][0] / max(n_it, 1)
        return dict(viscosity=("RKL2" if sts_flag else "PCG+PC2"), ms_per_step=round(msp, 3),
                    speedup_vs_fp64=round(ms64 / msp, 3),
                    pcg_iters_per_step=[sum(i["iters"][q] for i in infosp) / len(infosp) for q in range(3)],
                    pcg_iters_per_step_pc1=[sum(i["iters"][q] for i in infos64) / len(infos64) for q in range(3)],
                    ms_per_iteration=round(sum(per_it.values()), 4), ms_per_iteration_pc1=round(iter64_ms, 4),
                    kernel_ms_per_iteration=per_it,
                    line_kernel_gbs=round(PC2_LINE_BYTES_PER_CELL * N / (line_ms * 1e-3) / 1e9, 1),
                    rel_l2_vs_fp64_after_steps={k: float(torch.linalg.norm(dsp[k] - ds64p[k]) /
                                                         torch.linalg.norm(ds64p[k])) for k in ds64p},
                    clocks=clkp, kernel_ms={k: round(v[0], 3) for k, v in profp.items() if v[1]})

    pc2 = pc2_sts = pc2_mixed = None
    if not args.no_pc2:
        pc2 = pc2_entry(0)
        if not args.no_sts:
            pc2_sts = pc2_entry(1)
        if not args.no_mixed:
            pc2_mixed = pc2_entry(0, P.PREC_MIXED)

    # ---- resistivity eta = RES_ETA: explicit (eta J in E) against the implicit face solve, PC2 solves
    res_entry = None
    if not args.no_res:
        mse, infose, profe, clke, dse = run(P.PREC_FP64, psteps, 1, True, pc=1, eta=RES_ETA, res=0)
        msi, infosi, profi, clki, dsi = run(P.PREC_FP64, psteps, 1, True, pc=1, eta=RES_ETA, res=1)
        mse, msi = maxr(mse), maxr(msi)
        n_res = max(sum(i["iters_res"] for i in infosi), 1)
        res_entry = dict(eta=RES_ETA, cell_solves="FP64 PC2",
                         ms_per_step_explicit_resistivity=round(mse, 3), ms_per_step_implicit_resistivity=round(msi, 3),
                         resistive_iters_per_step=n_res / len(infosi),
                         resistive_solve_ms_per_step=round(profi["res"][0] / len(infosi), 3),
                         ms_per_resistive_iteration=round(profi["res"][0] / n_res, 4),
                         max_resistive_relres=max(i["relres_res"] for i in infosi),
                         rel_l2_implicit_vs_explicit_after_steps={k: float(torch.linalg.norm(dsi[k] - dse[k]) /
                                                                          torch.linalg.norm(dse[k])) for k in dse},
                         clocks=clki)

    sts = sts_mixed = None
    if not args.no_sts:
        sts = sts_entry(P.PREC_FP64)
        if not args.no_mixed:
            sts_mixed = sts_entry(P.PREC_MIXED)
    # ---- end to end through the C ABI with host buffers: every step uploads the state at the
    # start of the timed region from pinned host memory, runs mhd_step and reads the new state back
    e2e = None
    if not args.no_e2e:
        ds = dev_state()
        # the caller's host buffers: page-locked, allocated here (as a user of the library would own
        # them), holding the state at the start of the timed region
        host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in snap.items()}
        for k in host:
            host[k].copy_(snap[k])
        out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in snap.items()}
        f = P.make_fields(ds["br"], ds["bt"], ds["bp"], ds["vr"], ds["vt"], ds["vp"])
        # copy bandwidth of one buffer before the timed region (a check on the host memory, reported)
        torch.cuda.synchronize()
        pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ds["vp"].copy_(host["vp"], non_blocking=True)
            pa.record(stream)
            ds["vp"].copy_(host["vp"], non_blocking=True)
            pb.record(stream)
        stream.synchronize()
        probe_gbs = host["vp"].numel() * 8 / (pa.elapsed_time(pb) * 1e6)
        prm = P.make_params(nu=w["nu"], eta=w["eta"], cfl=w["cfl"], tol=w["tol"])
        ke = max(1, args.steps)
        h2d = sum(t.numel() * 8 for t in snap.values())
        barrier()
        ev = lambda: torch.cuda.Event(enable_timing=True)
        e0, e1 = ev(), ev()
        parts = {"h2d_ms": 0.0, "step_ms": 0.0, "d2h_ms": 0.0}
        e0.record(stream)
        for _ in range(ke):
            a, b_, c_, d_ = ev(), ev(), ev(), ev()
            a.record(stream)
            with torch.cuda.stream(stream):
                for k in ds:
                    ds[k].copy_(host[k], non_blocking=True)
            b_.record(stream)
            st_e, info_e = P.mhd_step(g, prm, f)
            c_.record(stream)
            with torch.cuda.stream(stream):
                for k in ds:
                    out[k].copy_(ds[k], non_blocking=True)
            d_.record(stream)
            stream.synchronize()
            parts["h2d_ms"] += a.elapsed_time(b_) / ke
            parts["step_ms"] += b_.elapsed_time(c_) / ke
            parts["d2h_ms"] += c_.elapsed_time(d_) / ke
        e1.record(stream)
        barrier()
        e2e = dict(value=round(maxr(e0.elapsed_time(e1) / ke), 3), unit="ms/step", h2d_bytes_per_step=h2d,
                   d2h_bytes_per_step=h2d, **{k: round(v, 3) for k, v in parts.items()},
                   h2d_probe_gbs=round(probe_gbs, 1),
                   pcg_iters_per_step=sum(info_e["iters"]),
                   note="each step starts from the state at the start of the timed region (host copy); "
                        "step_ms is that step alone, so it differs from the timed steps' mean by the "
                        "iteration count of that one step")
    # ---- CPU baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        iters, iters_src = cpu_baseline_iters(args, it64)
        ms_cpu, sample, used, parts = oracle_sample(w, st0, iters, pcg_iters=3)
        one, _, _, _ = oracle_sample(w, st0, iters, pcg_iters=2, threads=1)
        cpu = dict(value=round(ms_cpu, 1), unit="ms/step", cores=used, kind="oracle", sample=sample,
                   single_thread_value=round(one, 1), iters_per_step=iters, iters_source=iters_src,
                   parts_ms={k: round(v, 2) for k, v in parts.items()},
                   note="the same sample and iteration count as the reference arm (bench.py --impl reference), "
                        "which also prints measured whole oracle steps at 32x32x64 and 128x128x256")
    launches = sum(v[1] for v in prof64.values())
    if overlap64:   # the one-thread alpha kernel of each overlapped iteration has no profiling slot
        launches += it64_total
    if rank == 0:
        line = dict(metric=METRIC, value=round(ms64, 3), unit="ms/step", n_gpus=ws, steps=args.steps,
                    warmup=args.warmup, ms_per_step=round(ms64, 3), higher_is_better=False, scaling="weak",
                    vs_baseline=None, dtype="f64", data="synthetic",
                    config=dict(workload=args.workload, grid=f"{d.nr}x{d.nt}x{d.np}", precision="fp64",
                                parallelism=("replicas" if ws > 1 else "single"),
                                l2="inputs larger than L2 (no flush)",
                                pcg_iters_per_step=it64,
                                dt=[i["dt"] for i in infos64u]),
                    profiled=dict(steps=psteps, ms_per_step=round(ms64p, 3),
                                  pcg_iters_per_step=sum(sum(i["iters"]) for i in infos64) / len(infos64),
                                  clocks=clk64p,
                                  note="the same workload after one warm-up step (the headline's timed steps "
                                       "start after W), with CUDA events around every launch (PCG kernels "
                                       "launched directly instead of from graphs); kernel_ms and the roofline "
                                       "kernel come from this run; value is the unprofiled run"),
                    pcg_gbs=dict(fp64=round(pcg64_gbs, 1), fp64_frac_of_hbm=round(pcg64_gbs / hbm, 4),
                                 peak_gbs=hbm, peak_source=peak_src, kernels=kernels64),
                    roofline=roof, mixed=mixed, mixed_reliable=mixed_reliable, sts=sts, sts_mixed_reliable=sts_mixed, pcg_single_reduction=pcg_cg,
                    pc2=pc2, pc2_sts=pc2_sts, pc2_mixed_reliable=pc2_mixed, resistivity=res_entry,
                    e2e=e2e, cpu_baseline=cpu, clocks=clk64,
                    gpu_launches=int(launches), kernel_ms={k: round(v[0], 3) for k, v in prof64.items() if v[1]})
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def ktilde2_max(d):
    """max over cells of 1/dr^2 + 1/(r dtheta)^2 + 1/(r sin(theta) dphi)^2 (the SI coefficient's
    grid factor), for choosing each batched system's alpha."""
    import numpy as np
    from paper_1811_02605_gb300 import inputs as I
    r = I.radial_nodes(d)
    rc = 0.5 * (r[1:] + r[:-1])
    dr = r[1:] - r[:-1]
    sc = np.sin((np.arange(d.nt) + 0.5) * math.pi / d.nt)
    k2 = (1 / dr ** 2)[:, None] + (1 / (rc * math.pi / d.nt) ** 2)[:, None] + \
        1 / (rc[:, None] * sc[None, :] * 2 * math.pi / d.np) ** 2
    return float(k2.max())


def run_batched(args):
    """64 independent FP64 solves on grids of uneven size (nt in {32, 48, ..., 128}, nr = nt,
    np = 2 nt, stretch in [1.02, 1.08]) with smooth seeded right-hand sides, in one persistent
    launch, against the same 64 solves one after another. Each alpha gives its system the
    conditioning of the 32x32x64 parity workload's semi-implicit solve at step 0."""
    import numpy as np
    import torch
    from paper_1811_02605_gb300 import build as B
    B.build()
    import paper_1811_02605_gb300 as P
    from paper_1811_02605_gb300 import inputs as I
    X0 = 4623.0
    items = I.batched_items(args.batch)
    grids, bs, alphas, cells = [], [], [], 0
    for it in items:
        d = it["desc"]
        g = P.mhd_grid_create(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch)
        f = I.smooth_field(d, it["modes"])
        r = I.radial_nodes(d)
        th = np.arange(d.nt + 1) * math.pi / d.nt
        c = np.cos(th)
        c[0], c[-1] = 1.0, -1.0
        vol = ((r[1:] ** 3 - r[:-1] ** 3) / 3)[:, None] * (c[:-1] - c[1:])[None, :] * (2 * math.pi / d.np)
        bs.append(torch.from_numpy(np.ascontiguousarray(f * vol[None, :, :, None])).cuda())
        grids.append(g)
        alphas.append(X0 / ktilde2_max(d))
        cells += d.nr * d.nt * d.np
    prm = P.make_params(tol=1e-9, max_iter=50000)
    xs = [torch.zeros_like(b) for b in bs]
    t0 = time.perf_counter()
    st, its, rr = P.pcg_solve_batched(grids, alphas, bs, xs, prm)  # first call: plan + autotune
    t_first = time.perf_counter() - t0
    times = []
    for _ in range(args.steps):
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, its, rr = P.pcg_solve_batched(grids, alphas, bs, xs, prm)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    seq = []
    for _ in range(max(1, args.steps // 2)):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for g, a, b in zip(grids, alphas, bs):
            x = torch.zeros_like(b)
            P.pcg_solve(g, a, b, x, prm)
        e1.record()
        torch.cuda.synchronize()
        seq.append(e0.elapsed_time(e1))
    ms = min(times)
    # algorithmic bytes: 144 B per cell per CG iteration, summed over systems
    bytes_alg = sum(144.0 * it["desc"].nr * it["desc"].nt * it["desc"].np * n for it, n in zip(items, its))
    print(json.dumps(dict(workload=f"batched{args.batch}", status=P.STATUS_NAMES[st], ms_per_batch=round(ms, 3),
                          ms_sequential_single_solves=round(min(seq), 3), speedup=round(min(seq) / ms, 3),
                          first_call_ms_incl_autotune=round(1e3 * t_first, 1), total_cells=cells,
                          iters_min=min(its), iters_max=max(its), max_relres=max(rr),
                          pcg_gbs_algorithmic=round(bytes_alg / (ms * 1e-3) / 1e9, 1))), flush=True)


def run_adjoint(args):
    """20 FP64 steps at 128x128x256 with a checkpoint every 5 steps, loss = misfit of the final
    outer-shell B_r against a smooth seeded target; gradient with respect to the inner-boundary
    B_r and the initial v by the adjoint chain, checked against central differences of the same
    frozen-coefficient map on `--fd-dirs` seeded unit directions (h = 1e-6 relative)."""
    import numpy as np
    import torch
    from paper_1811_02605_gb300 import build as B
    B.build()
    import paper_1811_02605_gb300 as P
    from paper_1811_02605_gb300 import inputs as I
    from paper_1811_02605_gb300.autograd import simulate
    name = "adjoint_128x128x256"
    w, st = gen_state(name, args.grid)
    d = w["desc"]
    nsteps = args.adj_steps
    g = P.mhd_grid_create(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch)
    target = torch.from_numpy(I.outer_target(d, 1811 * 4)).cuda()
    kw = dict(nu=w["nu"], eta=w["eta"], cfl=w["cfl"], tol=1e-13, max_iter=500000)
    x0 = {k: torch.from_numpy(v).cuda().requires_grad_(k in ("vr", "vt", "vp", "br")) for k, v in st.items()}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = simulate(g, x0, nsteps, checkpoint_every=5, **kw)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss = 0.5 * torch.sum((out["br"][-1] - target) ** 2)
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    gv = [x0[k].grad.cpu().numpy() for k in ("vr", "vt", "vp")]
    gb = x0["br"].grad[0].cpu().numpy()
    # frozen per-step coefficients of the base trajectory
    base = {k: torch.from_numpy(v).cuda() for k, v in st.items()}
    f = P.make_fields(base["br"], base["bt"], base["bp"], base["vr"], base["vt"], base["vp"])
    dts, als = [], []
    for _ in range(nsteps):
        s_, info = P.mhd_step(g, P.make_params(**kw), f)
        dts.append(info["dt"])
        als.append(info["alpha_si"])

    def L(x):
        ds = {k: torch.from_numpy(v).cuda() for k, v in x.items()}
        ff = P.make_fields(ds["br"], ds["bt"], ds["bp"], ds["vr"], ds["vt"], ds["vp"])
        for n in range(nsteps):
            P.mhd_step(g, P.make_params(**dict(kw, dt_fixed=dts[n], alpha_si_fixed=als[n])), ff)
        return 0.5 * float(torch.sum((ds["br"][-1] - target) ** 2))

    errs, errs_g = [], []
    gnorm = math.sqrt(sum(float(np.sum(a * a)) for a in gv) + float(np.sum(gb * gb)))
    xn = math.sqrt(sum(float(np.sum(st[k] ** 2)) for k in ("vr", "vt", "vp")) + float(np.sum(st["br"][0] ** 2)))
    h = 1e-6 * xn
    t3 = time.perf_counter()
    for q in range(args.fd_dirs):
        rng = np.random.default_rng(1811 * 400 + q)
        dv = [rng.normal(size=st["vr"].shape) for _ in range(3)]
        db = rng.normal(size=st["br"][0].shape)
        nrm = math.sqrt(sum(float(np.sum(a * a)) for a in dv) + float(np.sum(db * db)))
        dv = [a / nrm for a in dv]
        db = db / nrm

        def pert(sg):
            x = {k: v.copy() for k, v in st.items()}
            for a, k in zip(dv, ("vr", "vt", "vp")):
                x[k] = x[k] + sg * h * a
            x["br"][0] = x["br"][0] + sg * h * db
            return x

        fd = (L(pert(1.0)) - L(pert(-1.0))) / (2 * h)
        ad = sum(float(np.sum(a * b)) for a, b in zip(gv, dv)) + float(np.sum(gb * db))
        errs.append(abs(fd - ad) / max(abs(fd), abs(ad), 1e-300))
        errs_g.append(abs(fd - ad) / gnorm)   # |d| = 1: error on the gradient's own scale
    t4 = time.perf_counter()
    print(json.dumps(dict(workload=name, grid=f"{d.nr}x{d.nt}x{d.np}", steps=nsteps, checkpoint_every=5,
                          tol=kw["tol"], loss=float(loss), forward_s=round(t1 - t0, 3),
                          backward_s=round(t2 - t1, 3), ms_per_step_fwd_adj=round(1e3 * (t2 - t0) / nsteps, 1),
                          fd_dirs=args.fd_dirs, fd_rel_err_max=max(errs), fd_rel_err_median=float(np.median(errs)),
                          fd_err_over_grad_norm_max=max(errs_g),
                          fd_seconds=round(t4 - t3, 1), grad_norm_v=math.sqrt(sum(float(np.sum(a * a)) for a in gv)),
                          grad_norm_br_inner=float(np.linalg.norm(gb)))), flush=True)


def run_refinement_study(args):
    """The workload's first semi-implicit solve in FP64 and in mixed precision with restarted
    refinement and with reliable updates over a range of inner tolerances (iterations, FP64
    corrections, wall time)."""
    import torch
    from paper_1811_02605_gb300 import build as B
    B.build()
    import paper_1811_02605_gb300 as P
    w, st0 = gen_state(args.workload, args.grid)
    d = w["desc"]
    g = P.mhd_grid_create(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch)
    ds = {k: torch.from_numpy(v).cuda() for k, v in st0.items()}
    f = P.make_fields(ds["br"], ds["bt"], ds["bp"], ds["vr"], ds["vt"], ds["vp"])
    c = P.mhd_step_coeffs(g, P.make_params(nu=w["nu"], cfl=w["cfl"]), f)
    b = torch.empty((3, d.nr, d.nt, d.np), dtype=torch.float64, device="cuda")
    P.mhd_force(g, f, c["dt"], b)
    rows = []

    def one(name, **kw):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t = time.perf_counter()
        s, it, ou, rr = P.pcg_solve(g, c["alpha_si"], b, x, P.make_params(tol=w["tol"], **kw))
        torch.cuda.synchronize()
        rows.append(dict(variant=name, status=P.STATUS_NAMES[s], iters=it, corrections=ou, relres=rr,
                         seconds=round(time.perf_counter() - t, 4), **{k: v for k, v in kw.items() if k != "precision"}))

    one("fp64")
    one("mixed warm-up", precision=1, inner_tol=0.1, max_outer=200)   # first mixed solve tunes kernels
    if not args.pc2_only:
        for restart in (1, 0):
            for itol in (1e-5, 1e-3, 1e-2, 1e-1, 0.3):
                one("restarted" if restart else "reliable", precision=1, inner_tol=itol, max_outer=200,
                    max_iter=20000, mixed_restart=restart)
    # the same first solve with PC2 (phi-line block-Jacobi ILU(0)), FP64 and mixed
    one("fp64 pc2", preconditioner=1)
    one("mixed pc2 warm-up", precision=1, inner_tol=0.1, max_outer=200, preconditioner=1)
    for itol in (1e-3, 1e-2, 3e-2, 1e-1, 0.3):
        one("reliable pc2", precision=1, inner_tol=itol, max_outer=200, max_iter=20000, mixed_restart=0,
            preconditioner=1)
    print(json.dumps(dict(workload=args.workload, grid=f"{d.nr}x{d.nt}x{d.np}", alpha_si=c["alpha_si"],
                          rows=rows)), flush=True)


def run_accuracy_study(args):
    """`--acc-steps` steps (default 20) of the workload from its initial state with each solver
    form; per-field relative L2 distance to the FP64 point-Jacobi run after every 5 steps, the
    largest final relative residual of any solve, and ms per step (CUDA events)."""
    import torch
    from paper_1811_02605_gb300 import build as B
    B.build()
    import paper_1811_02605_gb300 as P
    w, st0 = gen_state(args.workload, args.grid)
    d = w["desc"]
    stream = torch.cuda.Stream()
    g = P.mhd_grid_create(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch, stream)
    marks = [s for s in range(5, args.acc_steps + 1, 5)] or [args.acc_steps]
    if marks[-1] != args.acc_steps:
        marks.append(args.acc_steps)
    variants = [
        ("fp64_pc1", dict()),
        ("mixed_restarted_1e-5", dict(precision=P.PREC_MIXED, inner_tol=1e-5, mixed_restart=1)),
        ("mixed_reliable_0.1", dict(precision=P.PREC_MIXED, inner_tol=0.1, mixed_restart=0)),
        ("fp64_pc2", dict(preconditioner=1)),
        ("mixed_pc2_reliable_1e-3", dict(precision=P.PREC_MIXED, inner_tol=1e-3, mixed_restart=0,
                                         preconditioner=1)),
        # viscosity by RKL2 super time-stepping instead of the implicit solve: a different time
        # discretisation of the viscous term (the comparison the paper makes with its energies)
        ("fp64_sts", dict(viscosity_sts=1)),
        ("mixed_reliable_0.1_sts", dict(precision=P.PREC_MIXED, inner_tol=0.1, mixed_restart=0, viscosity_sts=1)),
    ]
    ref = {}
    rows = []
    for name, kw in variants:
        with torch.cuda.stream(stream):
            ds = {k: torch.from_numpy(v).to("cuda") for k, v in st0.items()}
        torch.cuda.synchronize()
        f = P.make_fields(ds["br"], ds["bt"], ds["bp"], ds["vr"], ds["vt"], ds["vp"])
        prm = P.make_params(nu=w["nu"], eta=w["eta"], cfl=w["cfl"], tol=w["tol"], max_outer=200,
                            max_iter=20000, **kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        errs, iters, worst, ms = {}, 0, 0.0, 0.0
        for s in range(1, args.acc_steps + 1):
            e0.record(stream)
            st, info = P.mhd_step(g, prm, f)
            e1.record(stream)
            torch.cuda.synchronize()
            if st != P.MHD_OK:
                raise RuntimeError(f"{name} step {s}: {P.STATUS_NAMES[st]} {P.mhd_last_error(g)}")
            ms += e0.elapsed_time(e1)
            iters += sum(info["iters"])
            worst = max(worst, max(info["relres"]))
            if s in marks:
                if name == "fp64_pc1":
                    ref[s] = {k: v.clone() for k, v in ds.items()}
                else:
                    errs[s] = {k: float(torch.linalg.norm(ds[k] - ref[s][k]) / torch.linalg.norm(ref[s][k]))
                               for k in ds}
        diag = P.mhd_diagnostics(g, f)   # Sec. 3.1: the paper compares such integrals between solver forms
        rows.append(dict(variant=name, ms_per_step=round(ms / args.acc_steps, 3),
                         pcg_iters_per_step=round(iters / args.acc_steps, 2), max_final_relres=worst,
                         rel_l2_vs_fp64_pc1={str(s): e for s, e in errs.items()},
                         diagnostics_after_steps=diag))
        del ds, f
    print(json.dumps(dict(accuracy_study=f"{d.nr}x{d.nt}x{d.np}", workload=args.workload,
                          steps=args.acc_steps, reference="FP64 point-Jacobi PCG on the GPU (the same "
                          "path matches the oracle's record of the first step at this size)", rows=rows)),
          flush=True)


def run_profile_case(args):
    """A short, fixed piece of the hot path for profilers: the first SI system of the workload,
    `--profile-iters` FP64 CG iterations, then one mixed-precision outer pass with the same cap."""
    import torch
    from paper_1811_02605_gb300 import build as B
    B.build()
    import paper_1811_02605_gb300 as P
    w, st0 = gen_state(args.workload, args.grid)
    d = w["desc"]
    g = P.mhd_grid_create(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch)
    ds = {k: torch.from_numpy(v).cuda() for k, v in st0.items()}
    f = P.make_fields(ds["br"], ds["bt"], ds["bp"], ds["vr"], ds["vt"], ds["vp"])
    c = P.mhd_step_coeffs(g, P.make_params(nu=w["nu"], cfl=w["cfl"]), f)
    b = torch.empty((3, d.nr, d.nt, d.np), dtype=torch.float64, device="cuda")
    P.mhd_force(g, f, c["dt"], b)
    out = {}
    legs = args.profile_legs.split(",")
    for name, prec, pc in (("fp64", P.PREC_FP64, 0), ("mixed", P.PREC_MIXED, 0), ("pc2", P.PREC_FP64, 1),
                           ("pc2mixed", P.PREC_MIXED, 1)):
        if name not in legs:
            continue
        x = torch.zeros_like(b)
        prm = P.make_params(tol=1e-30, max_iter=args.profile_iters, precision=prec, max_outer=1, preconditioner=pc)
        st, it, ou, rr = P.pcg_solve(g, c["alpha_si"], b, x, prm)
        out[name] = dict(status=P.STATUS_NAMES[st], iters=it, outer=ou, relres=rr)
    # whole steps with capped cell solves: the RKL2 stages (sts) or the implicit resistive solve (res)
    for name, kw in (("sts", dict(viscosity_sts=1)), ("res", dict(resistivity_implicit=1, eta=1e-2))):
        if name not in legs:
            continue
        dsc = {k: v.clone() for k, v in ds.items()}
        fc = P.make_fields(dsc["br"], dsc["bt"], dsc["bp"], dsc["vr"], dsc["vt"], dsc["vp"])
        prm = P.make_params(nu=w["nu"], cfl=w["cfl"], tol=1e-30, max_iter=args.profile_iters, **kw)
        st, info = P.mhd_step(g, prm, fc)
        out[name] = dict(status=P.STATUS_NAMES[st], stages=info["iters"][2], res_iters=info["iters_res"])
    torch.cuda.synchronize()
    print(json.dumps(dict(profile_case=f"{d.nr}x{d.nt}x{d.np}", alpha_si=c["alpha_si"], **out)), flush=True)


def run_iteration_forms(args):
    """Time each kernel form of the FP64 and FP32 CG iterations on the workload's first SI system:
    every form forced in turn (MHD_FORCE_SLAB) on its own grid. FP64: a fixed-count solve
    (--form-iters iterations, tol 1e-30); FP32: the mixed solve to tol 1e-9 with reliable updates at
    inner tol 0.1. Each once unprofiled (CUDA events around the solve) and once with per-kernel
    events. One JSON line per form."""
    import torch
    from paper_1811_02605_gb300 import build as B
    B.build()
    import paper_1811_02605_gb300 as P
    w, st0 = gen_state(args.workload, args.grid)
    d = w["desc"]
    N = d.nr * d.nt * d.np
    hbm, _ = peaks()
    ds = {k: torch.from_numpy(v).cuda() for k, v in st0.items()}
    del st0
    legs = [("fp64", c) for c in args.forms64.split(",") if c] + [("fp32", c) for c in args.forms32.split(",") if c]
    for prec, code in legs:
        os.environ["MHD_FORCE_SLAB"] = code
        g = P.mhd_grid_create(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch)
        f = P.make_fields(ds["br"], ds["bt"], ds["bp"], ds["vr"], ds["vt"], ds["vp"])
        c = P.mhd_step_coeffs(g, P.make_params(nu=w["nu"], cfl=w["cfl"]), f)
        b = torch.empty((3, d.nr, d.nt, d.np), dtype=torch.float64, device="cuda")
        P.mhd_force(g, f, c["dt"], b)
        if prec == "fp64":
            prm = P.make_params(tol=1e-30, max_iter=args.form_iters)
        else:
            prm = P.make_params(tol=1e-9, inner_tol=0.1, precision=P.PREC_MIXED, max_outer=200, max_iter=20000)
        x = torch.zeros_like(b)
        P.pcg_solve(g, c["alpha_si"], b, x, prm)   # the autotuner's set-up and a warm-up
        row = dict(precision=prec, form=code, forms_chosen=P.mhd_grid_kernel_forms(g))
        for prof in (False, True):
            x.zero_()
            torch.cuda.synchronize()
            P.mhd_profile_enable(g, prof)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st, it, ou, rr = P.pcg_solve(g, c["alpha_si"], b, x, prm)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if prof:
                pr = {k: v for k, v in P.mhd_profile_read(g).items() if v[1]}
                row["kernel_ms_per_iteration"] = {k: round(v[0] / it, 4) for k, v in pr.items()}
                P.mhd_profile_enable(g, False)
            else:
                row.update(iters=it, outer=ou, relres=rr, ms=round(ms, 3), ms_per_iteration=round(ms / it, 4))
        if prec == "fp32":
            inner = sum(v for k, v in row["kernel_ms_per_iteration"].items() if k.endswith("32"))
            row["inner_kernels_ms_per_iteration"] = round(inner, 4)
            row["inner_frac_of_hbm"] = round(PCG_BYTES_PER_CELL["fp32"] * N / (inner * 1e-3) / 1e9 / hbm, 4)
            row["solve_frac_of_hbm"] = round(PCG_BYTES_PER_CELL["fp32"] * N / (row["ms_per_iteration"] * 1e-3)
                                             / 1e9 / hbm, 4)
        else:
            row["fp64_pipe_frac"] = round(FP64_INSTR_PER_CELL_ITER * N / (row["ms_per_iteration"] * 1e-3)
                                          / FP64_INSTR_PEAK, 4)
        del g
        print(json.dumps(row), flush=True)
    os.environ.pop("MHD_FORCE_SLAB", None)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--grid", default=None, help="NRxNTxNP: the workload's physics on another grid")
    ap.add_argument("--profile-case", action="store_true",
                    help="run a few CG iterations of the first SI solve (for ncu captures) and exit")
    ap.add_argument("--profile-iters", type=int, default=6)
    ap.add_argument("--profile-legs", default="fp64,mixed",
                    help="--profile-case pieces: fp64, mixed, pc2, pc2mixed (capped solves), sts, res (capped steps)")
    ap.add_argument("--iteration-forms", action="store_true",
                    help="time every kernel form of the FP64 and FP32 CG iterations on the first SI system and exit")
    ap.add_argument("--forms64", default="-1,-64")
    ap.add_argument("--forms32", default="-1,-2,-3,-4,-6,-7,-8")
    ap.add_argument("--form-iters", type=int, default=300)
    ap.add_argument("--batched", action="store_true", help="time the 64-system batched solve and exit")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--adjoint", action="store_true", help="time and check the adjoint workload and exit")
    ap.add_argument("--refinement-study", action="store_true",
                    help="first SI solve: FP64 vs mixed (restarted / reliable updates) over inner tolerances")
    ap.add_argument("--accuracy-study", action="store_true",
                    help="--acc-steps steps with each solver form; per-field error against FP64 point-Jacobi")
    ap.add_argument("--acc-steps", type=int, default=20)
    ap.add_argument("--adj-steps", type=int, default=20)
    ap.add_argument("--fd-dirs", type=int, default=16)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-sts", action="store_true", help="skip the RKL2-viscosity entries")
    ap.add_argument("--no-cg", action="store_true", help="skip the single-reduction PCG entry")
    ap.add_argument("--no-pc2", action="store_true", help="skip the PC2 entries")
    ap.add_argument("--no-res", action="store_true", help="skip the resistivity entry")
    ap.add_argument("--pc2-only", action="store_true", help="--refinement-study: only the PC2 rows")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--all-entries", action="store_true",
                    help="with N > 1 ranks, also time the mixed, RKL2, single-reduction, PC2 and resistivity entries")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=3,
                    help="steps (after one warm-up) of the profiled FP64 run beside the unprofiled headline; "
                         "the RKL2, single-reduction, PC2 and resistivity entries run as many and compare "
                         "with it")
    ap.add_argument("--no-anchors", action="store_true",
                    help="reference arm: skip the measured whole oracle steps at 32x32x64 and 128x128x256")
    ap.add_argument("--ref-iters", type=int, default=1000,
                    help="PCG iterations per step assumed by the reference arm if no oracle record exists")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
    elif args.iteration_forms:
        run_iteration_forms(args)
    elif args.batched:
        run_batched(args)
    elif args.adjoint:
        run_adjoint(args)
    elif args.refinement_study:
        run_refinement_study(args)
    elif args.accuracy_study:
        run_accuracy_study(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
