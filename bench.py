#!/usr/bin/env python
"""Benchmark of the batched hot path: one step = the misfit gradient of a batch of (source,
frequency) problems.

Default workload (`vti512`): 512 x 512 VTI cells of 5 m, FFT grid 1024 x 1024, 64 surface sources x
6 frequencies (3-18 Hz) = 384 problems, 256 receivers, a smooth random contrast of +/-10 %. One
step: Green's tables for the 6 frequencies, incident fields, the batched complex64 BiCGSTAB
forward solve of A u = u0 to a relative residual of 1e-6 (every iteration two fused LS-operator
passes), the data residual at the receivers, and the adjoint: conj(residual) injected at the
receivers, convolved with G, solved in the background and imaged against u into the misfit
gradient for (rho, C11, C13, C33, C55). The metric counts LS-operator cell-applies (cells x
problems x operator passes, the Green's convolution of the adjoint source included) per second
of device time. The line also carries the same step on the 256 x 256 workload (32 sources x 8
frequencies, 5-20 Hz), the accuracy of sampled wavefields, data, residuals and a sub-batch
gradient against the FP64 CPU oracle, and the oracle's own rate on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --workload vti256       # the 256^2 gradient step alone
    python bench.py --workload uneven40     # the 40-problem uneven batch (grids 64^2 .. 512^2)
    python bench.py --workload op384        # operator passes over 384^2 problems on FFT length 768
    python bench.py --workload formk256     # operator passes in the paper-literal form of Eq. 9
    python bench.py --workload gmres256     # batched forward solves by GMRES(30) beside BiCGSTAB
    python bench.py --workload hess3d       # 3D operator passes and GMRES solves, 80 x 40 x 32 cells

With N > 1 (torchrun, one rank per GPU) every rank runs its own sources x all frequencies (weak
scaling) and the gradients are summed across ranks with one all-reduce per step.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload, one
process per host core.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2402_02116_gb300 import inputs  # noqa: E402

METRIC = "LS operator cell-applies/s (cells x sources x frequencies)"
UNIT = "cell-applies/s"
TOL = 1e-6          # BiCGSTAB relative residual of the benchmark's solves
MAX_ITER = 3000
ORACLE_TOL = 1e-12  # the FP64 oracle's solves that the accuracy block compares against


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle sample")
    ap.add_argument("--no-plain", action="store_true", help="skip the complex128 plain-path sample")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the accuracy block (FP64 oracle)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 256^2 line inside the 512^2 one")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparator")
    ap.add_argument("--cores", type=int, default=0, help="host processes for the oracle (0: every core)")
    ap.add_argument("--check-every", type=int, default=4,
                    help="BiCGSTAB iterations between host convergence checks (each check also "
                         "compacts the launches to the problems still active)")
    ap.add_argument("--workload", choices=["vti512", "vti256", "uneven40", "op384", "formk256", "gmres256", "hess3d"],
                    default="vti512",
                    help="vti512: the gradient step on 512^2 cells, 64 sources x 6 frequencies (default); "
                         "vti256: the gradient step on 256^2 cells, 32 sources x 8 frequencies; uneven40: "
                         "operator passes over the 40-problem uneven batch (persistent launches, autotuned), "
                         "plus one graph-captured solve; op384: operator passes over one 384^2 member of "
                         "the uneven recipe (96 problems) on FFT length 768 beside 1024; formk256: operator "
                         "passes over the 256^2 "
                         "batch in the paper-literal form (derivatives on G, Eq. 9) beside the "
                         "divergence form; gmres256: batched forward solves of the 256^2 batch by "
                         "restarted GMRES beside BiCGSTAB; hess3d: 3D operator passes and GMRES "
                         "solves on 80 x 40 x 32 cells (16 sources x 4 frequencies)")
    ap.add_argument("--restart", type=int, default=30, help="GMRES restart length (gmres256)")
    ap.add_argument("--sources", type=int, default=0,
                    help="sources per GPU (0: the workload's own, 64 at 512^2 and 32 at 256^2; fewer make a "
                         "smaller batch of the same grid for profiler captures)")
    return ap.parse_args()


def default_sources(name: str) -> int:
    return 64 if name == "vti512" else 32


def workload(name: str, rank: int = 0, world: int = 1, sources: int = 0):
    """The gradient workloads: `vti512` (512 x 512 cells, smooth random contrast, 6 frequencies
    3-18 Hz) or `vti256` (256 x 256 cells, layers and anomalies, 8 frequencies 5-20 Hz). With
    several ranks the job has `sources` surface sources per rank and every rank keeps its
    round-robin shard of them (weak scaling)."""
    full = default_sources(name)
    n = sources or full
    if name == "vti512":
        w = inputs.config4_misfit(n_src=n * world)
    else:
        w = inputs.config2_batched_forward()
        if n * world != full:
            cols = inputs.surface_line(w.nx, n * world)
            w.src_cells = np.stack([np.zeros_like(cols), cols], axis=1)
            w.src_force = np.tile([0.0, 1.0], (len(cols), 1))
    if world > 1:
        from paper_2402_02116_gb300.shard import shard_workload
        w = shard_workload(w, rank, world)
    if n != full:
        w.name = f"vti{w.nz}x{w.nx}_{n}src_{w.nf}f"
    return w


def config_dict(w, world):
    return {"workload": w.name, "nz": w.nz, "nx": w.nx, "lz": w.lz, "lx": w.lx, "h_m": w.h,
            "sources": w.n_src * world, "frequencies_hz": [round(float(f), 3) for f in w.freqs_hz],
            "receivers": int(len(w.rec_cells)), "problems_per_gpu": w.n_problems,
            "krylov": f"BiCGSTAB to {TOL:g} relative residual", "precision": "complex64 operator, FP64 reductions",
            "step": "greens_tabulate + incident_field + ls_solve + data_residual + adjoint_apply (gradient)",
            "l2": f"inputs larger than L2: each wavefield batch is {w.n_problems * 16 * w.nz * w.nx / 1e6:.0f} MB "
                  "(the L2 holds 129 MB)",
            "parallelism": f"dp{world} (sources sharded, gradient all-reduce)" if world > 1 else "single GPU"}


def synthetic_data(w, seed=7):
    """Observed data of the same shape as the receiver data, at the scale of the incident field
    (|d| ~ 1e-10 m for a unit force): seeded Gaussian, rounded to complex64 so that the GPU and the
    oracle read the same values."""
    return (inputs.seeded_complex((w.n_problems, len(w.rec_cells), 2), seed) * 1e-10).astype(np.complex64)


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index  # nvidia-smi --id: an index or a GPU UUID
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------
class GradientStep:
    """One gradient step of a workload on one device: every call goes through the library's C ABI
    (binding in paper_2402_02116_gb300/dbi.py)."""

    def __init__(self, w, dev, check_every, precision=None):
        from paper_2402_02116_gb300 import dbi
        from paper_2402_02116_gb300.problem import DeviceProblem
        self.dbi = dbi
        self.w = w
        self.P = DeviceProblem(w, dbi.C64 if precision is None else precision, device=dev)
        self.check_every = check_every
        self.cells = w.nz * w.nx

    def __call__(self, m, d_obs):
        dbi, P = self.dbi, self.P
        Ghat, Gspace = dbi.greens_tabulate(P.grid, P.ref, P.omega, P.precision)
        u0 = dbi.incident_field(P.grid, P.omega, P.fidx, Gspace, P.src_cells, P.forces)
        u, it_f, _, code_f = dbi.ls_solve(P.grid, P.ref, m, P.omega, P.fidx, Ghat, u0, tol=TOL,
                                          max_iter=MAX_ITER, check_every=self.check_every)
        r, phi = dbi.data_residual(P.grid, P.omega, P.fidx, P.rec_cells, u, d_obs)
        g, (it_a, _, code_a) = dbi.adjoint_apply(P.grid, P.ref, m, P.omega, P.fidx, Ghat, u, P.rec_cells, r,
                                                 tol=TOL, max_iter=MAX_ITER, check_every=self.check_every,
                                                 with_status=True)
        return {"phi": phi, "g": g, "it_f": it_f, "it_a": it_a, "code_f": code_f, "code_a": code_a, "u": u, "r": r}

    @staticmethod
    def applies(out):
        # two operator passes per BiCGSTAB iteration, plus the adjoint source's convolution
        return int(2 * out["it_f"].sum().item() + 2 * out["it_a"].sum().item() + out["it_a"].numel())


def timed_steps(step, m, d_obs, steps, warmup, dev, barrier, stage=None):
    """warmup untimed steps, then `steps` steps between CUDA events on the launching stream; returns
    (ms, applies, last output, launches, (stage ms, stage launches), clocks)."""
    import torch
    from paper_2402_02116_gb300 import dbi
    for _ in range(warmup):
        step(m, d_obs)
    barrier()
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = dbi.kernel_launches()
    if stage:
        dbi.profile_begin(stage)
    outs = []
    with ClockSampler(gpu_id(dev)) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(steps):
            outs.append(step(m, d_obs))
        ev1.record(stream)
        barrier()
    prof = dbi.profile_end() if stage else (0.0, 0)
    launches = dbi.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    applies = sum(GradientStep.applies(o) for o in outs)
    return ms, applies, outs[-1], launches, prof, clk.summary()


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2402_02116_gb300 import build, dbi
    from paper_2402_02116_gb300.shard import reduce_gradient

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    dbi.load()

    w = workload(args.workload, rank, world, args.sources)
    step_fn = GradientStep(w, dev, args.check_every)
    P = step_fn.P
    d_obs_host = synthetic_data(w, seed=7 + rank)
    d_obs = P.to_field(d_obs_host)
    cells = step_fn.cells

    def step(m, d):
        out = step_fn(m, d)
        reduce_gradient(out["g"], out["phi"])  # sum over ranks (no-op on one GPU)
        return out

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ms, total_applies, last, launches, (cols_ms, cols_launches), clocks = timed_steps(
        step, P.m, d_obs, args.steps, args.warmup, dev, barrier, stage=dbi.PROF_COLS)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    a = torch.tensor([total_applies], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(a, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    job_applies = float(a.item())
    value = job_applies * cells / (ms_max * 1e-3)
    ok = bool((last["code_f"] == dbi.CONVERGED).all().item() and (last["code_a"] == dbi.CONVERGED).all().item())

    # roofline of the column-pass kernel (the largest share of the step's device time)
    props = torch.cuda.get_device_properties(dev)
    sms = int(props.multi_processor_count)
    fp32 = fp32_peak_probe(dev, sms)
    roof = column_roofline(w, cells * total_applies, cols_ms, cols_launches, ms, clocks, fp32, sms)

    # end to end through the public API with host buffers (copies inside the timed region)
    e2e = run_e2e(args, P, step, d_obs_host, w, world, dev, barrier)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 (fp32 complex operator; fp64 inner products and scalars)",
        "data": "synthetic (seeded VTI model and contrast; seeded observed data)",
        "config": config_dict(w, world),
        "roofline": roof, "e2e": e2e, "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / args.steps, "clocks": clocks,
        "all_converged": ok,
        "krylov_iterations_per_step": {"forward_mean": float(last["it_f"].float().mean()),
                                       "forward_max": int(last["it_f"].max()),
                                       "adjoint_mean": float(last["it_a"].float().mean()),
                                       "adjoint_max": int(last["it_a"].max())},
        "device": {"name": props.name, "sms": sms},
    }
    solo = rank == 0 and world == 1
    if solo:
        result["operator_hbm"] = operator_stages(P, w, dev)
        result["path_roofline"] = path_roofline(w, result["operator_hbm"]["stages"]["pass"]["us_per_problem"],
                                                value, fp32["tflops"], result["operator_hbm"]["hbm_peak_gbs"])
    if solo and not args.no_cufft:
        result["cufft_c64"] = cufft_comparator(P, w, dev)
    if solo and not args.no_plain:
        result["plain_c128"] = plain_c128_sample(w, dev, cells, value)
    if solo and args.workload == "vti512" and not args.no_secondary:
        w2 = workload("vti256")
        s2 = GradientStep(w2, dev, args.check_every)
        d2 = s2.P.to_field(synthetic_data(w2))
        ms2, ap2, last2, _, _, clk2 = timed_steps(s2, s2.P.m, d2, max(3, min(args.steps, 10)), 2, dev, barrier)
        n2 = max(3, min(args.steps, 10))
        result["vti256"] = {"value": ap2 * s2.cells / (ms2 * 1e-3), "unit": UNIT, "ms_per_step": ms2 / n2,
                            "steps": n2, "config": config_dict(w2, 1), "clocks": clk2,
                            "all_converged": bool((last2["code_f"] == dbi.CONVERGED).all().item()
                                                  and (last2["code_a"] == dbi.CONVERGED).all().item())}
        del s2, d2, last2
    if solo and not (args.no_accuracy and args.no_cpu_baseline):
        acc_problems = accuracy_problems(w)
        gpu_acc = None if args.no_accuracy else gpu_accuracy_side(P, last, acc_problems)
        acc_res, base = run_cpp_oracle(w, d_obs_host, [] if args.no_accuracy else acc_problems,
                                       not args.no_cpu_baseline, args.cores)
        if acc_res is not None:
            result["accuracy"] = accuracy_block(w, gpu_acc, acc_res[0], acc_res[1], d_obs_host)
        if base is not None:
            result["cpu_baseline"] = base
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def fp32_peak_probe(dev, sms, iters=1 << 16, reps=10):
    """Measured FP32 FMA throughput (TFLOP/s): the library's FMA-only probe over 8 CTAs of 256
    threads per SM (the resident maximum), best of `reps` launches timed with CUDA events on the
    launching stream."""
    import torch
    from paper_2402_02116_gb300 import dbi
    blocks = 8 * sms
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        dbi.fma_probe(blocks, iters, dev)
    best = None
    flops = 0
    for _ in range(reps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        flops, _ = dbi.fma_probe(blocks, iters, dev)
        ev1.record(stream)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1)
        best = t if best is None else min(best, t)
    return {"tflops": flops / (best * 1e-3) / 1e12, "ms": best, "blocks": blocks, "flops": flops,
            "how": f"dbi_fma_probe: {blocks} CTAs x 256 threads x 8 FMA chains x {iters} steps, best of {reps}"}


def measured_alu_peak(dev, clocks):
    """The FP32 peak of the secondary workloads' ALU rooflines: the FMA probe (as for the default
    line), with the nominal figure from the device's SM count and the sampled clock beside it."""
    import torch
    sms = int(torch.cuda.get_device_properties(dev).multi_processor_count)
    fp32 = fp32_peak_probe(dev, sms)
    sm_mhz = clocks["sm_mhz"] or load_peaks().get("sm_max_mhz", 2070.0)
    return fp32["tflops"], "measured: " + fp32["how"], sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# DRAM bytes of one k_cols launch from ncu captures (dram__bytes_read.sum + dram__bytes_write.sum):
# (nz, nx, lz, lx) -> (problems in the captured launch, frequencies, bytes). The Green's spectra
# [nf][3][lx][lz] are read once per launch; the rest grows with the problems a launch processes.
COLS_DRAM = {
    # one k_cols_split launch over 6 sources x 6 frequencies (profiles/operator_kernels_vti512_6src_6f.md)
    (512, 512, 1024, 1024): (36, 6, 473_260_032 + 252_288_768),
}


def column_roofline(w, cell_applies, cols_ms, cols_launches, step_ms, clocks, fp32, sms):
    cols_algo_bytes = cols_bytes_per_cell_apply(w) * cell_applies
    cols_flops = cols_flops_per_cell_apply(w) * cell_applies
    cols_s = cols_ms * 1e-3
    peaks = load_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0) * 1e9
    sm_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    nominal = sms * 128 * 2 * sm_mhz * 1e6
    roof = {"bound": "alu", "achieved": cols_flops / cols_s / 1e12, "peak": fp32["tflops"], "unit": "TFLOP/s",
            "peak_source": "measured: " + fp32["how"],
            "peak_nominal": nominal / 1e12,
            "peak_nominal_source": f"{sms} SMs (device query) x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (sampled median)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["frac_of_nominal"] = roof["achieved"] / roof["peak_nominal"]
    roof["kernel"] = ("k_cols_split (column FFTs as pairs of 512-point transforms x Green's tensor x inverse)"
                      if w.lz == 1024 else "k_cols (column FFTs x Green's tensor x inverse column FFTs)")
    roof["flops_per_cell_apply"] = cols_flops_per_cell_apply(w)
    roof["algorithmic_bytes_per_cell_apply"] = cols_bytes_per_cell_apply(w)
    per_launch_problems = cell_applies / (w.nz * w.nx) / max(cols_launches, 1)
    cap = COLS_DRAM.get((w.nz, w.nx, w.lz, w.lx))
    if cap:
        nb, nf, byts = cap
        tables = 3 * w.lz * w.lx * 8 * nf
        roof["traffic"] = tables * w.nf / nf + (byts - tables) / nb * per_launch_problems
        roof["traffic_source"] = (f"ncu capture of one k_cols launch over {nb} problems ({nf} frequencies): "
                                  f"{byts / 1e6:.1f} MB, scaled to the {per_launch_problems:.0f} problems of an "
                                  "average timed launch (the tables once per launch)")
    else:
        roof["traffic"] = None
    roof["hbm_frac_of_algorithmic_bytes"] = cols_algo_bytes / cols_s / hbm_peak
    roof["launches_timed"] = cols_launches
    roof["avg_launch_ms"] = cols_ms / max(cols_launches, 1)
    roof["avg_launch_problems"] = per_launch_problems
    roof["share_of_step_time"] = cols_ms / step_ms if step_ms > 0 else None
    return roof


def gpu_id(dev):
    """nvidia-smi id of the device: its UUID when torch exposes it, else the visible index."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev.index] if vis else str(dev.index)


def run_e2e(args, P, step, d_obs_host, w, world, dev, barrier):
    """Same step, with the model and observed data copied from pinned host memory each step and
    the gradient and misfit read back. The public entry points (dbi.*) hand device pointers of
    these copies to the C ABI."""
    import torch
    m_host = torch.as_tensor(np.asarray(w.model, dtype=np.float32)).pin_memory()
    d_host = torch.as_tensor(np.asarray(d_obs_host, dtype=np.complex64)).pin_memory()
    g_host = torch.empty((5, w.nz, w.nx), dtype=torch.float32).pin_memory()
    phi_host = torch.empty((), dtype=torch.float64).pin_memory()
    m_dev = torch.empty(m_host.shape, dtype=torch.float32, device=dev)
    d_dev = torch.empty(d_host.shape, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    total = 0
    outs = []
    for _ in range(args.steps):
        m_dev.copy_(m_host, non_blocking=True)
        d_dev.copy_(d_host, non_blocking=True)
        out = step(m_dev, d_dev)
        g_host.copy_(out["g"], non_blocking=True)
        phi_host.copy_(out["phi"], non_blocking=True)
        outs.append((out["it_f"], out["it_a"]))
    ev1.record(stream)
    barrier()
    total = sum(int(2 * f.sum() + 2 * a.sum() + a.numel()) for f, a in outs)
    ms = ev0.elapsed_time(ev1)
    cells = w.nz * w.nx
    h2d = m_host.numel() * 4 + d_host.numel() * 8
    d2h = g_host.numel() * 4 + 8
    return {"value": total * world * cells / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms / args.steps,
            "api": "dbi.greens_tabulate/incident_field/ls_solve/data_residual/adjoint_apply (ctypes C ABI; the model "
                   "and data are copied from pinned host memory to device tensors whose pointers the C ABI receives)"}


def plain_c128_sample(w, dev, cells, value_c64):
    """The plain unbatched complex128 path (same kernels, one problem per call, FP64 throughout)
    on a sample of the problems: per-problem forward + adjoint time, scaled to the batch."""
    import torch

    from paper_2402_02116_gb300 import dbi
    from paper_2402_02116_gb300.problem import DeviceProblem
    P = DeviceProblem(w, dbi.C128, device=dev)
    d_obs = P.to_field(synthetic_data(w))
    sample = [0, w.n_problems // 2 + 3, w.n_problems - 1]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot_ms, tot_applies = 0.0, 0
    for b in sample:
        fidx = P.fidx[b:b + 1].contiguous()
        src, frc = P.src_cells[b:b + 1].contiguous(), P.forces[b:b + 1].contiguous()
        torch.cuda.synchronize()
        ev0.record()
        Ghat, Gspace = dbi.greens_tabulate(P.grid, P.ref, P.omega, dbi.C128)
        u0 = dbi.incident_field(P.grid, P.omega, fidx, Gspace, src, frc)
        u, it_f, _, _ = dbi.ls_solve(P.grid, P.ref, P.m, P.omega, fidx, Ghat, u0, tol=TOL, max_iter=MAX_ITER)
        r, phi = dbi.data_residual(P.grid, P.omega, fidx, P.rec_cells, u, d_obs[b:b + 1].contiguous())
        g, (it_a, _, _) = dbi.adjoint_apply(P.grid, P.ref, P.m, P.omega, fidx, Ghat, u, P.rec_cells, r, tol=TOL,
                                            max_iter=MAX_ITER, with_status=True)
        ev1.record()
        torch.cuda.synchronize()
        tot_ms += ev0.elapsed_time(ev1)
        tot_applies += int(2 * it_f.sum() + 2 * it_a.sum() + 1)
    rate = tot_applies * cells / (tot_ms * 1e-3)
    return {"value": rate, "unit": UNIT, "sample": f"problems {sample} of the batch, one per call",
            "ms_per_problem_gradient": tot_ms / len(sample),
            "est_ms_per_step": tot_ms / len(sample) * w.n_problems,
            "speedup_c64_batched": value_c64 / rate}


def operator_stage_bytes(w, precision_c64=True):
    """Algorithmic bytes per cell-apply of each stage of one ls_apply pass (complex64: 8-byte
    points; r = lx / nx, the spectra per domain cell): rows forward (with the contrast-source kernel
    where the row stage is split: u in, the source field out and back in), the spectra T written;
    cols: T read and written, the Green's spectra [3][lz][lx] once per frequency shared by its
    sources; rows inverse: T read, the identity term u read, the output written. The model (shared
    by the whole batch) is not counted."""
    r = w.lx / w.nx
    split = precision_c64 and w.lx in (768, 1024)
    g = 3 * w.lz * w.lx * 8 * w.nf / (w.n_problems * w.nz * w.nx)
    return {"rows_forward": (16 + 16 + 16 if split else 16) + 16 * r,
            "cols": 32 * r + g,
            "rows_inverse": 16 * r + 16 + 16}


def operator_stages(P, w, dev, passes=5):
    """Each stage of ls_apply over the whole batch timed by the library's stage events (CUDA events
    on the launching stream around every launch of the stage), `passes` passes per stage after a
    warm-up, and the pass as a whole; achieved bandwidth on the stage's algorithmic bytes against
    the measured copy bandwidth."""
    import torch
    from paper_2402_02116_gb300 import dbi
    u = P.incident()
    out = torch.empty_like(u)
    work, _ = dbi._work(P.grid, P.B, P.precision, dbi.OP_APPLY, u.device)

    def f():
        dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u, out=out, work=work)
    for _ in range(3):
        f()
    torch.cuda.synchronize()
    peak = load_peaks().get("hbm_gbs", 6800.0)
    cells = w.nz * w.nx
    bpc = operator_stage_bytes(w)
    stages = {}
    for stage, name in ((dbi.PROF_ROWS_FORWARD, "rows_forward"), (dbi.PROF_COLS, "cols"),
                        (dbi.PROF_ROWS_INVERSE, "rows_inverse"), (dbi.PROF_OPERATOR, "pass")):
        dbi.profile_begin(stage)
        for _ in range(passes):
            f()
        ms, n = dbi.profile_end()
        us = ms / n / P.B * 1e3  # per problem
        b = sum(bpc.values()) if name == "pass" else bpc[name]
        gbs = b * cells / (us * 1e-6) / 1e9
        stages[name] = {"us_per_problem": us, "bytes_per_cell_apply": b, "achieved_gbs": gbs,
                        "hbm_frac": gbs / peak}
    del work, out, u
    torch.cuda.empty_cache()
    return {"stages": stages, "hbm_peak_gbs": peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)",
            "passes_per_stage": passes, "grid": [w.nz, w.nx, w.lz, w.lx], "problems": P.B,
            "bytes": "algorithmic bytes per cell-apply: rows forward u 16 (+ the source field 16 out and 16 "
                     "in where the row stage is split) + spectra 16 lx/nx out; cols spectra 2 x 16 lx/nx + "
                     "Green's spectra once per frequency; rows inverse spectra 16 lx/nx + u 16 + out 16"}


def cufft_comparator(P, w, dev, reps=5):
    """A cuFFT-based complex64 LS operator pass on the same batch, for comparison only (it is not
    part of the library): the contrast source by the same central differences in torch
    elementwise ops, zero padding and 2D FFTs by torch.fft (cuFFT), the symmetric 2 x 2 product
    with the library's Green's spectra (transposed to row-major once, outside the timing), inverse
    2D FFTs, crop, u - K u. Timed per pass with CUDA events beside the library's ls_apply on the
    same input; the two outputs are compared."""
    import torch
    from paper_2402_02116_gb300 import dbi
    nz, nx, lz, lx, h = w.nz, w.nx, w.lz, w.lx, w.h
    nf, ns = w.nf, w.n_src
    u = P.incident()
    ref = torch.tensor(reference_values(w), dtype=torch.float32, device=dev)
    dm = (P.m - ref[:, None, None]).contiguous()
    w2 = (P.omega.to(torch.float32) ** 2)[P.fidx.long()].view(-1, 1, 1)
    G = P.Ghat.transpose(-1, -2).contiguous().view(nf, 1, 3, lz, lx)  # [nf][1][3][lz][lx]
    inv2h = 1.0 / (2.0 * h)

    def d1(v):  # central difference along x, zero outside the grid
        o = torch.zeros_like(v)
        o[..., 1:-1] = v[..., 2:] - v[..., :-2]
        o[..., 0] = v[..., 1]
        o[..., -1] = -v[..., -2]
        return o * inv2h

    def d3(v):
        o = torch.zeros_like(v)
        o[..., 1:-1, :] = v[..., 2:, :] - v[..., :-2, :]
        o[..., 0, :] = v[..., 1, :]
        o[..., -1, :] = -v[..., -2, :]
        return o * inv2h

    def apply(u):
        u1, u3 = u[:, 0], u[:, 1]
        e1, e3, e5 = d1(u1), d3(u3), d3(u1) + d1(u3)
        s1 = dm[1] * e1 + dm[2] * e3
        s3 = dm[2] * e1 + dm[3] * e3
        s5 = dm[4] * e5
        src = torch.stack([w2 * dm[0] * u1 + d1(s1) + d3(s5), w2 * dm[0] * u3 + d1(s5) + d3(s3)], dim=1)
        S = torch.fft.fft2(src, s=(lz, lx)).view(nf, ns, 2, lz, lx)
        O = torch.stack([G[:, :, 0] * S[:, :, 0] + G[:, :, 1] * S[:, :, 1],
                         G[:, :, 1] * S[:, :, 0] + G[:, :, 2] * S[:, :, 1]], dim=2)
        o = torch.fft.ifft2(O.view(-1, 2, lz, lx), norm="forward")[..., :nz, :nx]
        return u - o

    stream = torch.cuda.current_stream(dev)

    def time_it(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            out = fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps, out

    out_buf = torch.empty_like(u)
    ms_lib, a_lib = time_it(lambda: dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u, out=out_buf))
    a_lib = a_lib.clone()
    ms_fft, a_fft = time_it(lambda: apply(u))
    ms_fft_only, _ = time_it(lambda: torch.fft.ifft2(torch.fft.fft2(u, s=(lz, lx)), norm="forward"))
    diff = float(torch.linalg.norm(a_fft - a_lib) / torch.linalg.norm(a_lib - u))
    cells = nz * nx * P.B
    del a_fft
    torch.cuda.empty_cache()
    return {"value": cells / (ms_fft * 1e-3), "unit": UNIT, "ms_per_pass": ms_fft,
            "library_ls_apply": {"value": cells / (ms_lib * 1e-3), "ms_per_pass": ms_lib},
            "cufft_transforms_only_ms": ms_fft_only,
            "speedup_library_over_cufft": ms_fft / ms_lib,
            "relative_difference_to_library": diff,
            "what": "one operator pass over every problem: torch elementwise stencil + torch.fft.fft2/ifft2 (cuFFT, "
                    f"{lz}x{lx}, 2 components) + 2x2 product; transforms_only = forward + inverse 2D FFTs of the field"}


def reference_values(w):
    """(rho, C11, C13, C33, C55) of the isotropic reference medium of a workload (Eq. 4)."""
    a2, b2 = w.alpha0 ** 2, w.beta0 ** 2
    return [w.rho0, w.rho0 * a2, w.rho0 * (a2 - 2 * b2), w.rho0 * a2, w.rho0 * b2]


# ---------------------------------------------------------------------------------------------
# roofline arithmetic of the column pass (per D-cell per operator pass)
# ---------------------------------------------------------------------------------------------
COLS_DRAM_BYTES_PER_PROBLEM = 4.35e6  # ncu, k_cols before the per-exchange line layout


def cols_bytes_per_cell_apply(w):
    """Compulsory bytes of k_cols: the row-transformed field T[2][nz][lx] read once and written
    once (complex64), plus the Green's spectrum [3][lz][lx] read once per frequency and shared by
    the sources of that frequency."""
    cells = w.nz * w.nx
    t = 2 * 2 * w.nz * w.lx * 8
    g = 3 * w.lz * w.lx * 8 * w.nf / w.n_problems
    return (t + g) / cells


def cols_flops_per_cell_apply(w):
    """Nominal flops of k_cols: 5 L log2 L per complex FFT of length lz (2 components, forward
    and inverse, lx columns) plus the symmetric 2x2 complex multiply (4 complex products and 2
    sums, 28 flops) at each of the lz x lx wavenumbers."""
    cells = w.nz * w.nx
    fft = 2 * 2 * w.lx * 5 * w.lz * math.log2(w.lz)
    mult = 28 * w.lz * w.lx
    return (fft + mult) / cells


def pass_flops_per_cell_apply(w):
    """Nominal flops of one operator pass: 5 L log2 L per complex FFT (the rows forward and inverse
    over the nz non-zero rows, 2 components each; the columns forward and inverse over all lx
    columns, 2 components each) plus the symmetric 2x2 Green's multiply (28 flops per wavenumber).
    The stencil, the contrast contraction and the epilogue (a few dozen flops per cell) are left
    out."""
    rows = 2 * 2 * w.nz * 5 * w.lx * math.log2(w.lx)
    return rows / (w.nz * w.nx) + cols_flops_per_cell_apply(w)


def compulsory_bytes_per_cell_apply(w):
    """Bytes one operator pass cannot avoid (complex64): the input field read and the output field
    written (16 B each per cell), the Green's spectra [3][lz][lx] once per frequency and the five
    float32 contrast parameters once per batch."""
    cells = w.nz * w.nx
    return 16 + 16 + 3 * w.lz * w.lx * 8 * w.nf / (w.n_problems * cells) + 20 / w.n_problems


def path_roofline(w, pass_us_per_problem, step_value, fp32_tflops, hbm_gbs):
    """The operator pass and the whole gradient step against the path's own roofline: cell-applies
    per second ÷ min(HBM bandwidth / compulsory bytes, FP32 peak / pass flops), both per
    cell-apply. With every transpose on chip the pass would be bound by the smaller of the two; the
    built pass moves its spectra through HBM between stages (operator_hbm gives that fraction)."""
    flops = pass_flops_per_cell_apply(w)
    byts = compulsory_bytes_per_cell_apply(w)
    alu = fp32_tflops * 1e12 / flops
    hbm = hbm_gbs * 1e9 / byts
    bound = min(alu, hbm)
    achieved = w.nz * w.nx / (pass_us_per_problem * 1e-6)
    return {"flops_per_cell_apply": flops, "compulsory_bytes_per_cell_apply": byts,
            "alu_bound": alu, "hbm_bound": hbm, "bound": "alu" if alu <= hbm else "hbm",
            "unit": "cell-applies/s", "pass_achieved": achieved, "pass_frac": achieved / bound,
            "step_frac": step_value / bound,
            "peaks": {"fp32_tflops": fp32_tflops, "hbm_gbs": hbm_gbs, "source": "measured (FMA probe; copy)"}}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}


# ---------------------------------------------------------------------------------------------
# the FP64 CPU oracle: accuracy of sampled problems and the CPU baseline, one process per core
# ---------------------------------------------------------------------------------------------
def accuracy_problems(w):
    """Problems whose wavefields, data and gradient the accuracy block compares with the FP64
    oracle: the first source at the lowest frequency and the middle source at the highest."""
    return [0, (w.nf - 1) * w.n_src + w.n_src // 2]


def run_cpp_oracle(w, d_obs_host, acc_problems, baseline, cores=0):
    """The C++17 FP64 oracle (OpenMP, one problem per thread) on the host cores, two jobs at once:
    the accuracy reference (the sampled problems solved to ORACLE_TOL) on one thread per sampled
    problem, and the CPU baseline (one gradient contribution per remaining core at the benchmark's
    tolerance, the lowest frequency, distinct sources). Returns (accuracy results or None, baseline
    line or None)."""
    import threading
    from oracle import cpp_oracle as C
    cores = cores or (os.cpu_count() or 1)
    model = np.asarray(w.model, dtype=np.float32).astype(np.float64)  # as the GPU reads it
    d_obs = np.asarray(d_obs_host).astype(np.complex128)
    fidx_all, src_all = w.problem_fidx(), w.problem_src()
    out = {}

    def acc_job():
        b = np.asarray(acc_problems)
        fs = sorted(set(int(f) for f in fidx_all[b]))
        orc = C.Oracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, model, w.omegas[fs],
                       threads=len(b))
        fidx = np.array([fs.index(int(f)) for f in fidx_all[b]], dtype=np.int32)
        t0 = time.perf_counter()
        g, r, passes, relres, u = orc.gradient(fidx, w.src_cells[src_all[b]], w.src_force[src_all[b]], w.rec_cells,
                                               d_obs[b], tol=ORACLE_TOL, threads=len(b), keep_fields=True)
        dt = time.perf_counter() - t0
        out["acc"] = ([{"b": int(bb), "u": u[k], "d": r[k] + d_obs[bb], "r": r[k], "passes": int(passes[k]),
                        "relres": tuple(float(x) for x in relres[k]), "seconds": dt,
                        "freq_hz": float(w.freqs_hz[fidx_all[bb]]), "source": int(src_all[bb])}
                       for k, bb in enumerate(b)], g)

    def base_job(n):
        bs = [int(k * w.n_src // n) % w.n_src for k in range(n)]  # lowest frequency, distinct sources
        orc = C.Oracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, model, w.omegas[:1], threads=n)
        t0 = time.perf_counter()
        g, r, passes, relres, _ = orc.gradient(np.zeros(n, dtype=np.int32), w.src_cells[bs], w.src_force[bs],
                                               w.rec_cells, d_obs[bs], tol=TOL, threads=n)
        dt = time.perf_counter() - t0
        out["base"] = {"value": float(passes.sum()) * w.nz * w.nx / dt, "unit": UNIT, "cores": n, "kind": "oracle",
                       "sample": f"C++17 FP64 oracle (own radix-2 FFT, OpenMP, one problem per thread) on {n} host "
                                 f"cores: the gradient contributions (forward solve, residual, adjoint solve, imaging) "
                                 f"of {n} problems of {w.name} at {w.freqs_hz[0]:g} Hz, BiCGSTAB to {TOL:g}, "
                                 f"{int(passes.sum())} operator passes in {dt:.1f} s (tables built before)",
                       "seconds": dt, "host_cpu_count": os.cpu_count()}

    jobs = []
    if acc_problems:
        jobs.append(threading.Thread(target=acc_job))
    n_base = max(1, cores - len(acc_problems))
    if baseline:
        jobs.append(threading.Thread(target=base_job, args=(n_base,)))
    for j in jobs:
        j.start()
    for j in jobs:
        j.join()
    return out.get("acc"), out.get("base")


def gpu_accuracy_side(P, last, problems):
    """GPU values of the sampled problems from the last timed step (wavefield, residual), and the
    gradient of the sub-batch of those problems by one more adjoint_apply at the benchmark's
    tolerance."""
    import torch
    from paper_2402_02116_gb300 import dbi
    idx = torch.tensor(problems, dtype=torch.long, device=P.device)
    u = last["u"].index_select(0, idx).contiguous()
    r = last["r"].index_select(0, idx).contiguous()
    fidx = P.fidx.index_select(0, idx).contiguous()
    g = dbi.adjoint_apply(P.grid, P.ref, P.m, P.omega, fidx, P.Ghat, u, P.rec_cells, r, tol=TOL, max_iter=MAX_ITER)
    torch.cuda.synchronize()
    return {"u": u.cpu().numpy().astype(np.complex128), "r": r.cpu().numpy().astype(np.complex128),
            "g": g.cpu().numpy().astype(np.float64)}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def accuracy_block(w, gpu, res, g_or, d_obs_host):
    """Relative L2 errors against the FP64 oracle (solved to ORACLE_TOL): every sampled problem's
    wavefield, receiver data (P u) and data residual, and the sub-batch gradient (g_or: the oracle's
    gradient summed over the sampled problems) per parameter."""
    per = []
    for k, r in enumerate(res):
        d_gpu = gpu["r"][k] + d_obs_host[r["b"]].astype(np.complex128)
        per.append({"problem": r["b"], "source": r["source"], "freq_hz": r["freq_hz"],
                    "wavefield": _rel(gpu["u"][k], r["u"]), "data": _rel(d_gpu, r["d"]),
                    "residual": _rel(gpu["r"][k], r["r"]),
                    "oracle_passes": r["passes"], "oracle_relres": r["relres"], "oracle_seconds": r["seconds"]})
    grad = {p: _rel(gpu["g"][i], g_or[i]) for i, p in enumerate(inputs.PARAMS)}
    return {"reference": f"C++17 FP64 oracle, BiCGSTAB to {ORACLE_TOL:g} (same seeded inputs: model rounded to "
                         "float32, observed data to complex64, as the GPU reads them)",
            "gpu": f"complex64 BiCGSTAB to {TOL:g} (the timed step's last solutions; the gradient by adjoint_apply "
                   "on the sub-batch of the sampled problems)",
            "problems": per,
            "wavefield_max": max(p["wavefield"] for p in per), "data_max": max(p["data"] for p in per),
            "residual_max": max(p["residual"] for p in per),
            "gradient_subbatch": grad, "gradient_max": max(grad.values()),
            "gradient_all": _rel(gpu["g"], g_or),
            "tolerances": {"wavefield": 1e-5, "data": 1e-5, "residual": 1e-5, "gradient": 1e-4}}


def _oracle_rate(passes, cells, dt, sample):
    return {"value": passes * cells / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
            "seconds": dt}


def oracle_formk_sample(w, b, passes=16):
    """Operator passes of the paper-literal form (Eq. 9) on problem b by the FP64 oracle as it stands;
    its derivative tables are built before the timed passes, as the GPU line times passes only."""
    import oracle as O
    f, s = int(w.problem_fidx()[b]), int(w.problem_src()[b])
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas[f:f + 1])
    u = orc.incident(0, w.src_cells[s], w.src_force[s])
    orc.apply_k(u, w.model, 0)
    t0 = time.perf_counter()
    for _ in range(passes):
        orc.apply_k(u, w.model, 0)
    dt = time.perf_counter() - t0
    return _oracle_rate(passes, w.nz * w.nx, dt, f"problem {b} (source {s}, {w.freqs_hz[f]:.2f} Hz) of {w.name}: "
                        f"{passes} paper-literal operator passes in {dt:.1f} s (tables built before)")


def oracle_gmres_sample(w, b, restart=30):
    """One GMRES(restart) forward solve of problem b to the bench tolerance by the FP64 oracle; every
    operator pass it makes (Arnoldi steps, the residual of each cycle, the final check) is counted."""
    import oracle as O
    f, s = int(w.problem_fidx()[b]), int(w.problem_src()[b])
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas[f:f + 1])
    u0 = orc.incident(0, w.src_cells[s], w.src_force[s])
    calls, apply = [0], orc.apply

    def counted(u, model, fi):
        calls[0] += 1
        return apply(u, model, fi)

    orc.apply = counted
    t0 = time.perf_counter()
    _, info = orc.solve_gmres(u0, w.model, 0, restart=restart, tol=TOL)
    dt = time.perf_counter() - t0
    return _oracle_rate(calls[0], w.nz * w.nx, dt, f"problem {b} (source {s}, {w.freqs_hz[f]:.2f} Hz) of {w.name}: "
                        f"GMRES({restart}) to {TOL:g}, {info['iters']} Arnoldi steps, {calls[0]} operator passes "
                        f"in {dt:.1f} s")


def oracle_3d_sample(w, b, passes=4):
    """3D operator passes on wavefield b by the FP64 3D oracle as it stands (tables built before)."""
    import oracle as O
    f, s = int(w.problem_fidx()[b]), int(w.problem_src()[b])
    orc = O.o3d.LSOracle3D(w.nz, w.ny, w.nx, w.h, w.lz, w.ly, w.lx, w.rho0, w.alpha0, w.beta0,
                           w.omegas[f:f + 1])
    u = orc.incident(0, tuple(w.src_cells[s]), w.src_force[s])
    t0 = time.perf_counter()
    for _ in range(passes):
        orc.apply(u, w.model, 0)
    dt = time.perf_counter() - t0
    return _oracle_rate(passes, w.nz * w.ny * w.nx, dt, f"wavefield {b} (source {s}, {w.freqs_hz[f]:.2f} Hz) of "
                        f"{w.name}: {passes} 3D operator passes in {dt:.1f} s (tables built before)")


def oracle_uneven_sample(ws):
    """One operator pass by the FP64 oracle on one problem of each grid size of the uneven batch; each
    size's time per cell is weighted by its share of the batch's cells, so the rate is the oracle's
    on this mix of sizes."""
    import oracle as O
    by_size = {}
    for w in ws:
        by_size.setdefault((w.nz, w.nx, w.lz, w.lx), []).append(w)
    t_mix, cells_mix, seconds, parts = 0.0, 0, 0.0, []
    for key in sorted(by_size):
        w = by_size[key][0]
        orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas[:1])
        u = orc.incident(0, w.src_cells[0], w.src_force[0])
        t0 = time.perf_counter()
        orc.apply(u, w.model, 0)
        dt = time.perf_counter() - t0
        cells = sum(g.n_problems * g.nz * g.nx for g in by_size[key])
        t_mix += dt / (w.nz * w.nx) * cells
        cells_mix += cells
        seconds += dt
        parts.append(f"{w.nz}x{w.nx} (L {w.lz}): {dt * 1e3:.0f} ms")
    return {"value": cells_mix / t_mix, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one oracle operator pass per grid size (" + ", ".join(parts)
                      + "), weighted by each size's cells in the batch", "seconds": seconds}


def run_reference(args):
    """The C++17 FP64 oracle as it stands on every host core (OpenMP, one problem per thread): each
    step runs two LS-operator passes (one BiCGSTAB iteration's worth) on each of `cores` problems of
    the workload (lowest frequency, distinct sources); the oracle's tables are built before the
    warm-up steps."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from oracle import cpp_oracle as C
    name = args.workload if args.workload in ("vti512", "vti256") else "vti512"
    w = workload(name, 0, 1, args.sources)
    cores = args.cores or (os.cpu_count() or 1)
    model = np.asarray(w.model, dtype=np.float32).astype(np.float64)
    orc = C.Oracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, model, w.omegas[:1], threads=cores)
    bs = [int(k * w.n_src // cores) % w.n_src for k in range(cores)]
    fidx = np.zeros(cores, dtype=np.int32)
    u = np.stack([np.asarray(inputs.seeded_complex((2, w.nz, w.nx), 100 + b)) for b in bs])
    for _ in range(args.warmup):
        orc.apply(fidx, u, threads=cores)
    t_sec, t_applies = 0.0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        v = orc.apply(fidx, u, threads=cores)
        orc.apply(fidx, v, threads=cores)
        t_sec += time.perf_counter() - t0
        t_applies += 2.0 * cores * w.nz * w.nx
    value = t_applies / t_sec
    sample = (f"C++17 FP64 oracle (own radix-2 FFT, OpenMP, one problem per thread) on {cores} host cores: each step "
              f"2 LS-operator passes on each of {cores} problems of {w.name} (lowest frequency, distinct sources)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_sec / max(args.steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex128)",
            "data": "synthetic", "config": config_dict(w, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cores, "sample": sample,
                             "host_cpu_count": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_uneven(args):
    """Operator passes over the 40-problem uneven batch (3074 wavefields on grids of 64^2 .. 512^2),
    after the autotuner; one step = one pass over every wavefield. Also times one graph-captured
    BiCGSTAB solve of every wavefield from its incident field."""
    import torch
    from paper_2402_02116_gb300 import dbi
    from paper_2402_02116_gb300.group import UnevenBatch
    from paper_2402_02116_gb300.problem import DeviceProblem
    rank, world = 0, 1
    if args.gpus > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        rank, world = dist.get_rank(), dist.get_world_size()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    from paper_2402_02116_gb300 import build
    build.build()
    dbi.load()
    ws = inputs.config5_uneven()
    Ps = [DeviceProblem(w, dbi.C64, device=dev) for w in ws]
    G = UnevenBatch(Ps, dbi.C64)
    u = G.incident()
    out = torch.empty_like(u)
    tuning = G.tune(u)
    cells = sum(P.B * P.w.nz * P.w.nx for P in Ps)
    for _ in range(args.warmup):
        G.apply(u, out=out)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = dbi.kernel_launches()
    with ClockSampler(gpu_id(dev)) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            G.apply(u, out=out)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = dbi.kernel_launches() - launches0
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * cells * args.steps / (ms_max * 1e-3)
    # one graph-captured solve of every wavefield
    torch.cuda.synchronize()
    t0 = time.time()
    _, iters, _, code = G.solve(u, tol=TOL, max_iter=MAX_ITER, check_every=8, graph=True)
    torch.cuda.synchronize()
    solve_s = time.time() - t0
    slot_cells = [P.w.nz * P.w.nx for P in Ps for _ in range(P.B)]
    useful = sum(2 * int(i) * c for i, c in zip(iters.cpu().tolist(), slot_cells))
    sizes = sorted({P.w.nz for P in Ps})
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 (fp32 complex operator; fp64 inner products and scalars)",
        "data": "synthetic (seeded isotropic / VTI models with Gaussian anomalies)",
        "config": {"workload": "uneven40: 40 problems, square grids " + "/".join(f"{n}^2" for n in sizes)
                   + ", 1-32 sources x 1-8 frequencies (2-25 Hz) each", "members": len(Ps),
                   "wavefields": G.slots, "cells_per_pass": cells, "step": "one operator pass over every "
                   "wavefield (per stage one persistent launch for each kernel kind present: ordinary, "
                   "pairs of 512-point and triples of 256-point transforms; the source kernel; input scaling)",
                   "fft_lengths": sorted({P.w.lz for P in Ps} | {P.w.lx for P in Ps}),
                   "l2": f"inputs larger than L2: {cells * 16 / 1e9:.1f} GB per field"},
        "autotuner": tuning, "gpu_launches": int(launches), "gpu_launches_per_step": launches / args.steps,
        "clocks": clk.summary(),
        "solve": {"seconds": solve_s, "all_converged": bool((code == dbi.CONVERGED).all()),
                  "iterations_mean": float(iters.float().mean()), "iterations_max": int(iters.max()),
                  "useful_cell_applies_per_s": useful / solve_s, "graph_captured": True},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = oracle_uneven_sample(ws)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_op384(args):
    """Operator passes over one 384^2 member of the uneven recipe (seed 7, its first 16 sources x 6
    frequencies: 96 problems) on FFT length 768, where every half-pruned transform runs as three
    256-point transforms; one step = one ls_apply pass over the 96 problems. The same batch on
    length 1024 (pairs of 512-point transforms) is timed beside it, and every stage of both by the
    library's stage events."""
    import dataclasses
    import torch
    from paper_2402_02116_gb300 import build, dbi
    from paper_2402_02116_gb300.problem import DeviceProblem
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    build.build()
    dbi.load()
    runs = {}
    for radix3 in (True, False):
        w = inputs.config5_uneven(sizes=(384,), n_members=1, max_src=32, max_f=8, seed=7, radix3=radix3)[0]
        w = dataclasses.replace(w, src_cells=w.src_cells[:16], src_force=w.src_force[:16],
                                name=f"{w.name.split('_')[0]}_16src_{w.nf}f_L{w.lz}")
        P = DeviceProblem(w, dbi.C64, device=dev)
        u = P.incident()
        out = torch.empty_like(u)
        work, _ = dbi._work(P.grid, P.B, dbi.C64, dbi.OP_APPLY, u.device)

        def f():
            dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u, out=out, work=work)
        for _ in range(args.warmup):
            f()
        stream = torch.cuda.current_stream(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = dbi.kernel_launches()
        with ClockSampler(gpu_id(dev)) as clk:
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.steps):
                f()
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        runs[w.lz] = {"w": w, "ms": ms, "launches": dbi.kernel_launches() - n0, "clocks": clk.summary(),
                      "stages": operator_stages(P, w, dev), "cells": P.B * w.nz * w.nx}
        del P, u, out, work
        torch.cuda.empty_cache()
    r, r2 = runs[768], runs[1024]
    w = r["w"]
    result = {
        "metric": METRIC, "value": r["cells"] * args.steps / (r["ms"] * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32 complex operator)",
        "data": "synthetic (seeded model of the uneven recipe: background with Gaussian anomalies)",
        "config": {"workload": f"op384: {w.name}, one ls_apply pass over the {w.n_problems} problems",
                   "nz": w.nz, "nx": w.nx, "lz": w.lz, "lx": w.lx,
                   "l2": f"spectra larger than L2: {w.n_problems * 2 * w.lx * w.nz * 8 / 1e9:.2f} GB per pass"},
        "operator_hbm": r["stages"], "gpu_launches": int(r["launches"]),
        "gpu_launches_per_step": r["launches"] / args.steps, "clocks": r["clocks"],
        "length_1024": {"value": r2["cells"] * args.steps / (r2["ms"] * 1e-3), "unit": UNIT,
                        "ms_per_step": r2["ms"] / args.steps, "operator_hbm": r2["stages"], "clocks": r2["clocks"]},
    }
    print(json.dumps(result), flush=True)


def formk_cols_bytes_per_cell_apply(w):
    """Compulsory bytes of kk_cols: the five row-transformed sources [5][nz][lx] read and the two
    outputs [2][nz][lx] written (complex64), plus Ghat [3][lz][lx] and the derivative tables
    [6][lz][lx] read once per frequency and shared by its sources."""
    t = 7 * w.nz * w.lx * 8
    g = 9 * w.lz * w.lx * 8 * w.nf / w.n_problems
    return (t + g) / (w.nz * w.nx)


def formk_cols_flops_per_cell_apply(w):
    """Nominal flops of kk_cols: 5 L log2 L per complex FFT of length lz (five forward, two
    inverse per column, lx columns) plus the 2 x 5 complex multiply-accumulate (10 products and
    10 sums, 80 flops) at each of the lz x lx wavenumbers."""
    fft = 7 * w.lx * 5 * w.lz * math.log2(w.lz)
    return (fft + 80 * w.lz * w.lx) / (w.nz * w.nx)


def run_formk(args):
    """Operator passes over the 256 x 256 VTI batch (32 sources x 8 frequencies) in the
    paper-literal form of Eq. 9 (ls_apply_k: five sources, the 2 x 5 kernel of G and its central
    differences), one step = one pass over the 256 wavefields; the divergence form (ls_apply) is
    timed the same way on the same inputs, and the two results are compared."""
    import torch
    from paper_2402_02116_gb300 import build, dbi
    from paper_2402_02116_gb300.problem import DeviceProblem
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    build.build()
    dbi.load()
    w = workload("vti256", 0, 1, args.sources)
    P = DeviceProblem(w, dbi.C64, device=dev)
    u = P.incident()
    out = torch.empty_like(u)
    cells = w.nz * w.nx * P.B
    stream = torch.cuda.current_stream(dev)

    def timed(fn, stage):
        for _ in range(args.warmup):
            fn()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = dbi.kernel_launches()
        dbi.profile_begin(stage)
        with ClockSampler(gpu_id(dev)) as clk:
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.steps):
                fn()
            ev1.record(stream)
            torch.cuda.synchronize()
        stage_ms, stage_launches = dbi.profile_end()
        return ev0.elapsed_time(ev1), dbi.kernel_launches() - n0, stage_ms, stage_launches, clk.summary()

    Dhat = P.Dhat
    ms_k, launches_k, cols_ms, cols_launches, clocks = timed(
        lambda: dbi.ls_apply_k(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, Dhat, u, out=out), dbi.PROF_COLS)
    a_k = out.clone()
    out_s = torch.empty_like(u)
    ms_s, launches_s, _, _, clocks_s = timed(
        lambda: dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u, out=out_s), dbi.PROF_OPERATOR)
    diff = float(torch.linalg.norm(a_k - out_s) / torch.linalg.norm(out_s - u))
    value = cells * args.steps / (ms_k * 1e-3)
    peaks = load_peaks()
    peak_tf, peak_src, nominal_tf = measured_alu_peak(dev, clocks)
    cols_s = cols_ms * 1e-3
    flops = formk_cols_flops_per_cell_apply(w) * cells * args.steps
    algo_bytes = formk_cols_bytes_per_cell_apply(w) * cells * args.steps
    # DRAM bytes per launch from one ncu capture of kk_cols over 32 wavefields of this grid (8
    # frequencies): 373.98 MB, of which the nine kernel tables are 151 MB; the rest grows with the
    # wavefields a launch processes
    traffic = None
    if (w.nz, w.nx, w.lz, w.lx, w.nf) == (256, 256, 512, 512, 8):
        tables = 9 * w.lz * w.lx * 8 * w.nf
        traffic = tables + (373.98e6 - tables) / 32 * cells * args.steps / (w.nz * w.nx) / max(cols_launches, 1)
    roof = {"bound": "alu", "achieved": flops / cols_s / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
            "peak_source": peak_src, "peak_nominal": nominal_tf,
            "traffic": traffic, "kernel": "kk_cols (five forward column FFTs, 2 x 5 kernel, two inverse)",
            "hbm_frac_of_algorithmic_bytes": algo_bytes / cols_s / (peaks.get("hbm_gbs", 6800.0) * 1e9),
            "launches_timed": cols_launches, "avg_launch_ms": cols_ms / max(cols_launches, 1),
            "share_of_step_time": cols_ms / ms_k if ms_k > 0 else None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_k / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 (fp32 complex operator)", "data": "synthetic (seeded VTI model with layers and anomalies)",
        "config": {"workload": f"formk: {w.name}, one operator pass over every wavefield in the paper-literal "
                               "form of Eq. 9 (derivatives on G)", "nz": w.nz, "nx": w.nx, "lz": w.lz, "lx": w.lx,
                   "wavefields": P.B, "l2": f"inputs larger than L2: {cells * 16 / 1e9:.2f} GB per field"},
        "roofline": roof, "gpu_launches": int(launches_k), "gpu_launches_per_step": launches_k / args.steps,
        "clocks": clocks,
        "divergence_form": {"value": cells * args.steps / (ms_s * 1e-3), "ms_per_step": ms_s / args.steps,
                            "gpu_launches_per_step": launches_s / args.steps, "clocks": clocks_s},
        "form_difference": {"relative_to_scattered_field": diff,
                            "note": "||A_K u0 - A_S u0|| / ||A_S u0 - u0|| over the batch: the boundary layer "
                                    "the divergence form leaves out where the contrast reaches the edge of D"},
    }
    if not args.no_cpu_baseline:
        result["cpu_baseline"] = oracle_formk_sample(w, w.n_problems // 2 + 3)
    print(json.dumps(result), flush=True)


def run_gmres(args):
    """Forward solves of the 256 x 256 VTI batch (32 sources x 8 frequencies) to 1e-5 from the
    incident fields, one step = one batched solve: restarted GMRES (the paper's solver) and then
    BiCGSTAB on the same right-hand sides. The metric counts the operator passes each solver made
    (Arnoldi steps for GMRES, two per iteration for BiCGSTAB) times the cells, per second."""
    import torch
    from paper_2402_02116_gb300 import build, dbi
    from paper_2402_02116_gb300.problem import DeviceProblem
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    build.build()
    dbi.load()
    w = workload("vti256", 0, 1, args.sources)
    P = DeviceProblem(w, dbi.C64, device=dev)
    u0 = P.incident()
    cells = w.nz * w.nx
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = dbi.kernel_launches()
        dbi.profile_begin(dbi.PROF_OPERATOR)
        with ClockSampler(gpu_id(dev)) as clk:
            torch.cuda.synchronize()
            ev0.record(stream)
            outs = [fn() for _ in range(args.steps)]
            ev1.record(stream)
            torch.cuda.synchronize()
        op_ms, op_n = dbi.profile_end()
        return ev0.elapsed_time(ev1), dbi.kernel_launches() - n0, op_ms, op_n, clk.summary(), outs[-1]

    ms_g, launches_g, op_ms_g, op_n_g, clocks, (u_g, it_g, rr_g, code_g) = timed(
        lambda: P.solve_gmres(u0, restart=args.restart, tol=TOL, max_iter=MAX_ITER, check_every=args.check_every))
    ms_b, launches_b, op_ms_b, _, clocks_b, (u_b, it_b, rr_b, code_b) = timed(
        lambda: P.solve(u0, tol=TOL, max_iter=MAX_ITER, check_every=args.check_every))
    # Arnoldi steps plus the residual pass of every restart (the first cycle starts from x = 0)
    passes_g = int(it_g.sum()) + int(((it_g - 1).clamp(min=0) // args.restart).sum())
    passes_b = 2 * int(it_b.sum())
    value = passes_g * cells * args.steps / (ms_g * 1e-3)
    agree = float(torch.linalg.norm(u_g - u_b) / torch.linalg.norm(u_b))
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_g / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 (fp32 complex operator and basis; fp64 Hessenberg, rotations, reductions)",
        "data": "synthetic (seeded VTI model with layers and anomalies)",
        "config": {"workload": f"gmres: {w.name}, one batched forward solve to {TOL:g} by GMRES({args.restart})",
                   "nz": w.nz, "nx": w.nx, "lz": w.lz, "lx": w.lx, "wavefields": P.B,
                   "l2": f"inputs larger than L2: {P.B * cells * 16 / 1e9:.2f} GB per field"},
        "gpu_launches": int(launches_g), "gpu_launches_per_step": launches_g / args.steps, "clocks": clocks,
        "gmres": {"solve_ms": ms_g / args.steps, "arnoldi_steps_mean": float(it_g.float().mean()),
                  "arnoldi_steps_max": int(it_g.max()), "operator_passes": passes_g,
                  "operator_share": op_ms_g / ms_g, "all_converged": bool((code_g == dbi.CONVERGED).all())},
        "bicgstab": {"solve_ms": ms_b / args.steps, "iterations_mean": float(it_b.float().mean()),
                     "operator_passes": passes_b, "operator_share": op_ms_b / ms_b,
                     "cell_applies_per_s": passes_b * cells * args.steps / (ms_b * 1e-3),
                     "all_converged": bool((code_b == dbi.CONVERGED).all()), "clocks": clocks_b},
        "solutions_relative_difference": agree,
    }
    if not args.no_cpu_baseline:
        result["cpu_baseline"] = oracle_gmres_sample(w, w.n_problems // 2 + 3, args.restart)
    print(json.dumps(result), flush=True)


def run_hess3d(args):
    """3D extension at the size of the paper's modified 3D VTI example (80 x 40 x 32 cells of 25 m,
    FFT grid 256 x 128 x 64), 16 surface sources x 4 frequencies = 64 wavefields, complex64: one
    step = one 3D operator pass over every wavefield; one GMRES(30) solve of the batch to 1e-5 is
    timed after the steps."""
    import torch
    from paper_2402_02116_gb300 import build, dbi
    from paper_2402_02116_gb300.problem import DeviceProblem3D
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    build.build()
    dbi.load()
    w = inputs.hess3d_like()
    P = DeviceProblem3D(w, dbi.C64, device=dev)
    u = P.incident()
    out = torch.empty_like(u)
    cells = w.nz * w.ny * w.nx * P.B
    work, nbytes = dbi._work3(P.grid, P.B, dbi.C64, dbi.OP_APPLY, dev)
    model = dbi._model3(P.grid, P.ref, P.m, dbi.C64)
    batch = dbi._batch(P.omega, P.fidx)
    lib = dbi.load()

    def step():
        dbi._check(lib.ls_apply_3d(ctypes.byref(model), ctypes.byref(batch), dbi._ptr(P.Ghat), dbi._ptr(u),
                                   dbi._ptr(out), dbi.C64, dbi._ptr(work), nbytes, dbi._stream(dev)), "ls_apply_3d")

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = dbi.kernel_launches()
    dbi.profile_begin(dbi.PROF_COLS)
    with ClockSampler(gpu_id(dev)) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    z_ms, z_launches = dbi.profile_end()
    ms = ev0.elapsed_time(ev1)
    launches = dbi.kernel_launches() - n0
    torch.cuda.synchronize()
    t0 = time.time()
    _, iters, _, code = P.solve(u, restart=30, tol=1e-5, max_iter=2000)
    torch.cuda.synchronize()
    solve_s = time.time() - t0
    clocks = clk.summary()
    peaks = load_peaks()
    peak_tf, peak_src, nominal_tf = measured_alu_peak(dev, clocks)
    # the z pass: per (ky, kx) column of every wavefield three forward and three inverse FFTs of
    # length lz (5 L log2 L flops each) and the symmetric 3 x 3 complex product (66 flops) per kz
    cols = P.B * w.ly * w.lx
    z_flops = cols * (6 * 5 * w.lz * math.log2(w.lz) + 66 * w.lz) * args.steps
    z_bytes = (P.B * 2 * 3 * w.nz * w.ly * w.lx * 8 + w.nf * 6 * w.lz * w.ly * w.lx * 8) * args.steps
    z_s = z_ms * 1e-3
    roof = {"bound": "alu", "achieved": z_flops / z_s / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
            "peak_source": peak_src, "peak_nominal": nominal_tf, "traffic": None,
            "kernel": ("k3_fft_z_reg (register z-line FFTs of the three components, 3 x 3 kernel, inverse)"
                       if w.lz <= 256 else
                       "k3_fft_z_mul (z-line FFTs of the three components, 3 x 3 kernel, inverse)"),
            "hbm_frac_of_algorithmic_bytes": z_bytes / z_s / (peaks.get("hbm_gbs", 6800.0) * 1e9),
            "launches_timed": z_launches, "avg_launch_ms": z_ms / max(z_launches, 1),
            "share_of_step_time": z_ms / ms if ms > 0 else None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    result = {
        "metric": METRIC, "value": cells * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 (fp32 complex operator)",
        "data": "synthetic (seeded 3D VTI model with layers and anomalies, the size of the paper's 3D example)",
        "config": {"workload": f"3d: {w.name}, one operator pass over every wavefield", "nz": w.nz, "ny": w.ny,
                   "nx": w.nx, "lz": w.lz, "ly": w.ly, "lx": w.lx, "wavefields": P.B,
                   "l2": f"spectra larger than L2: {P.B * 3 * w.nz * w.ly * w.lx * 8 / 1e9:.2f} GB per pass"},
        "roofline": roof, "gpu_launches": int(launches), "gpu_launches_per_step": launches / args.steps,
        "clocks": clocks,
        "gmres_solve": {"seconds": solve_s, "all_converged": bool((code == dbi.CONVERGED).all()),
                        "arnoldi_steps_mean": float(iters.float().mean()), "arnoldi_steps_max": int(iters.max())},
    }
    if not args.no_cpu_baseline:
        result["cpu_baseline"] = oracle_3d_sample(w, w.n_problems // 2 + 3)
    print(json.dumps(result), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven40":
        run_uneven(args)
    elif args.workload == "op384":
        run_op384(args)
    elif args.workload == "formk256":
        run_formk(args)
    elif args.workload == "gmres256":
        run_gmres(args)
    elif args.workload == "hess3d":
        run_hess3d(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
