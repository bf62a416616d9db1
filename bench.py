#!/usr/bin/env python
"""Benchmark of the batched hot path on the 256 x 256 VTI workload (32 sources x 8 frequencies).

One step = one pass of the whole hot path over the batch: Green's tables for the 8 frequencies,
incident fields, the batched complex64 BiCGSTAB forward solve of A u = u0 (every iteration two
fused LS-operator passes), the data residual at the receivers, and the adjoint: conj(residual)
injected at the receivers, convolved with G, solved in the background and imaged against u into
the misfit gradient for (rho, C11, C13, C33, C55). The metric counts LS-operator cell-applies
(cells x problems x operator passes, the Green's convolution of the adjoint source included) per
second of wall time on the device.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --workload uneven40     # the 40-problem uneven batch (grids 64^2 .. 512^2)
    python bench.py --workload formk256     # operator passes in the paper-literal form of Eq. 9
    python bench.py --workload gmres256     # batched forward solves by GMRES(30) beside BiCGSTAB
    python bench.py --workload hess3d       # 3D operator passes and GMRES solves, 80 x 40 x 32 cells

With N > 1 (torchrun, one rank per GPU) every rank runs its own 32 sources x 8 frequencies
(weak scaling) and the gradients are summed across ranks with one all-reduce per step.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload.
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
from paper_2402_02116_gb300.shard import reduce_gradient, shard_workload  # noqa: E402

METRIC = "LS operator cell-applies/s (cells x sources x frequencies)"
UNIT = "cell-applies/s"
TOL = 1e-5
MAX_ITER = 3000


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle sample")
    ap.add_argument("--no-plain", action="store_true", help="skip the complex128 plain-path sample")
    ap.add_argument("--check-every", type=int, default=4,
                    help="BiCGSTAB iterations between host convergence checks (each check also "
                         "compacts the launches to the problems still active)")
    ap.add_argument("--workload", choices=["vti256", "uneven40", "formk256", "gmres256", "hess3d"],
                    default="vti256",
                    help="vti256: the gradient step of the benchmark (default); uneven40: operator "
                         "passes over the 40-problem uneven batch (persistent launches, autotuned), "
                         "plus one graph-captured solve; formk256: operator passes over the 256^2 "
                         "batch in the paper-literal form (derivatives on G, Eq. 9) beside the "
                         "divergence form; gmres256: batched forward solves of the 256^2 batch by "
                         "restarted GMRES beside BiCGSTAB; hess3d: 3D operator passes and GMRES "
                         "solves on 80 x 40 x 32 cells (16 sources x 4 frequencies)")
    ap.add_argument("--restart", type=int, default=30, help="GMRES restart length (gmres256)")
    ap.add_argument("--sources", type=int, default=32,
                    help="sources per GPU (32 is the benchmark workload; fewer make a smaller batch "
                         "of the same grid for profiler captures)")
    return ap.parse_args()


def workload(rank: int, world: int, sources: int = 32):
    """The 256 x 256 VTI workload; with several ranks the job has `sources` surface sources per
    rank and every rank keeps its round-robin shard of them (weak scaling)."""
    w = inputs.config2_batched_forward()
    if world > 1 or sources != 32:
        cols = inputs.surface_line(w.nx, sources * world)
        w.src_cells = np.stack([np.zeros_like(cols), cols], axis=1)
        w.src_force = np.tile([0.0, 1.0], (len(cols), 1))
        w = shard_workload(w, rank, world)
        if sources != 32:
            w.name = f"vti{w.nz}x{w.nx}_{sources}src_{w.nf}f"
    return w


def config_dict(w, world):
    return {"workload": w.name, "nz": w.nz, "nx": w.nx, "lz": w.lz, "lx": w.lx, "h_m": w.h,
            "sources": w.n_src * world, "frequencies_hz": [round(float(f), 3) for f in w.freqs_hz],
            "receivers": int(len(w.rec_cells)), "problems_per_gpu": w.n_problems,
            "krylov": f"BiCGSTAB to {TOL:g} relative residual", "precision": "complex64 operator, FP64 reductions",
            "step": "greens_tabulate + incident_field + ls_solve + data_residual + adjoint_apply (gradient)",
            "l2": "inputs larger than L2: each wavefield batch is 256 MB (the L2 holds 129 MB)",
            "parallelism": f"dp{world} (sources sharded, gradient all-reduce)" if world > 1 else "single GPU"}


def synthetic_data(w, seed=7):
    """Observed data of the same shape as the receiver data, at the scale of the incident field
    (|d| ~ 1e-10 m for a unit force): seeded Gaussian."""
    return inputs.seeded_complex((w.n_problems, len(w.rec_cells), 2), seed) * 1e-10


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
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2402_02116_gb300 import build, dbi
    from paper_2402_02116_gb300.problem import DeviceProblem

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    dbi.load()

    w = workload(rank, world, args.sources)
    P = DeviceProblem(w, dbi.C64, device=dev)
    d_obs_host = synthetic_data(w, seed=7 + rank)
    d_obs = P.to_field(d_obs_host)
    cells = w.nz * w.nx

    def step(m, d_obs):
        Ghat, Gspace = dbi.greens_tabulate(P.grid, P.ref, P.omega, dbi.C64)
        u0 = dbi.incident_field(P.grid, P.omega, P.fidx, Gspace, P.src_cells, P.forces)
        u, it_f, _, code_f = dbi.ls_solve(P.grid, P.ref, m, P.omega, P.fidx, Ghat, u0, tol=TOL,
                                          max_iter=MAX_ITER, check_every=args.check_every)
        r, phi = dbi.data_residual(P.grid, P.omega, P.fidx, P.rec_cells, u, d_obs)
        g, (it_a, _, code_a) = dbi.adjoint_apply(P.grid, P.ref, m, P.omega, P.fidx, Ghat, u, P.rec_cells, r,
                                                 tol=TOL, max_iter=MAX_ITER, check_every=args.check_every,
                                                 with_status=True)
        reduce_gradient(g, phi)  # sum over ranks (no-op on one GPU)
        return phi, g, it_f, it_a, code_f, code_a

    def applies(it_f, it_a):
        # two operator passes per BiCGSTAB iteration, plus the adjoint source's convolution
        return int(2 * it_f.sum().item() + 2 * it_a.sum().item() + it_a.numel())

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (untimed)
    for _ in range(args.warmup):
        out = step(P.m, d_obs)
    barrier()
    ok = bool((out[4] == dbi.CONVERGED).all().item() and (out[5] == dbi.CONVERGED).all().item())

    # timed region: device events on the launching stream, barrier + synchronize on both sides
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_applies = 0
    launches0 = dbi.kernel_launches()
    dbi.profile_begin(dbi.PROF_COLS)
    with ClockSampler(gpu_id(dev)) as clk:
        barrier()
        ev0.record(stream)
        per_step = []
        for _ in range(args.steps):
            phi, g, it_f, it_a, code_f, code_a = step(P.m, d_obs)
            per_step.append((it_f, it_a))
        ev1.record(stream)
        barrier()
    cols_ms, cols_launches = dbi.profile_end()
    launches = dbi.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    for it_f, it_a in per_step:
        total_applies += applies(it_f, it_a)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    a = torch.tensor([total_applies], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(a, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    job_applies = float(a.item())
    value = job_applies * cells / (ms_max * 1e-3)
    ok = ok and bool((code_f == dbi.CONVERGED).all().item() and (code_a == dbi.CONVERGED).all().item())

    # roofline of the column-pass kernel (the largest share of the step's device time)
    peaks = load_peaks()
    rank_applies = total_applies
    cols_algo_bytes = cols_bytes_per_cell_apply(w) * cells * rank_applies
    cols_flops = cols_flops_per_cell_apply(w) * cells * rank_applies
    cols_s = cols_ms * 1e-3
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6  # FMA lanes x 2 flop x measured SM clock
    hbm_peak = peaks.get("hbm_gbs", 6800.0) * 1e9
    t_hbm, t_alu = cols_algo_bytes / hbm_peak, cols_flops / fp32_peak
    if t_alu >= t_hbm:
        roof = {"bound": "alu", "achieved": cols_flops / cols_s / 1e12, "peak": fp32_peak / 1e12,
                "unit": "TFLOP/s", "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (measured median)"}
    else:
        roof = {"bound": "hbm", "achieved": cols_algo_bytes / cols_s / 1e9, "peak": hbm_peak / 1e9,
                "unit": "GB/s", "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = "k_cols (column FFTs x Green's tensor x inverse column FFTs)"
    # DRAM bytes per launch: null, because k_cols changed (its FFT line layout is now chosen per
    # exchange) after its last ncu DRAM capture on these shapes; that capture is kept as context
    roof["traffic"] = None
    if (w.nz, w.nx, w.lz, w.lx) == (256, 256, 512, 512):
        roof["traffic_note"] = ("null: k_cols changed after its last ncu DRAM capture, which gave "
                                f"{COLS_DRAM_BYTES_PER_PROBLEM / 1e6:.2f} MB per problem (64-problem capture) "
                                "against 4.39 MB algorithmic")
    roof["hbm_frac_of_algorithmic_bytes"] = cols_algo_bytes / cols_s / hbm_peak
    roof["launches_timed"] = cols_launches
    roof["avg_launch_ms"] = cols_ms / max(cols_launches, 1)
    roof["share_of_step_time"] = cols_ms / ms if ms > 0 else None

    # end to end through the public API with host buffers (copies inside the timed region)
    e2e = run_e2e(args, P, step, d_obs_host, w, world, dev, barrier, applies)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 (fp32 complex operator; fp64 inner products and scalars)",
        "data": "synthetic (seeded VTI model with layers and anomalies; seeded observed data)",
        "config": config_dict(w, world),
        "roofline": roof, "e2e": e2e, "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / args.steps, "clocks": clocks,
        "all_converged": ok,
        "krylov_iterations_per_step": {"forward_mean": float(per_step[-1][0].float().mean()),
                                       "adjoint_mean": float(per_step[-1][1].float().mean())},
    }
    if rank == 0 and world == 1 and not args.no_plain:
        result["plain_c128"] = plain_c128_sample(w, dev, cells, value)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = oracle_samples(w, [0, w.n_problems // 2 + 3, w.n_problems - 1])
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def gpu_id(dev):
    """nvidia-smi id of the device: its UUID when torch exposes it, else the visible index."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev.index] if vis else str(dev.index)


def run_e2e(args, P, step, d_obs_host, w, world, dev, barrier, applies):
    """Same step, with the model and observed data copied from pinned host memory each step and
    the gradient and misfit read back."""
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
    its = []
    for _ in range(args.steps):
        m_dev.copy_(m_host, non_blocking=True)
        d_dev.copy_(d_host, non_blocking=True)
        phi, g, it_f, it_a, _, _ = step(m_dev, d_dev)
        g_host.copy_(g, non_blocking=True)
        phi_host.copy_(phi, non_blocking=True)
        its.append((it_f, it_a))
    ev1.record(stream)
    barrier()
    total = sum(applies(it_f, it_a) for it_f, it_a in its)
    ms = ev0.elapsed_time(ev1)
    cells = w.nz * w.nx
    h2d = m_host.numel() * 4 + d_host.numel() * 8
    d2h = g_host.numel() * 4 + 8
    return {"value": total * world * cells / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms / args.steps,
            "api": "dbi.greens_tabulate/incident_field/ls_solve/data_residual/adjoint_apply"}


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


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}


# ---------------------------------------------------------------------------------------------
# the FP64 CPU oracle on a bounded sample
# ---------------------------------------------------------------------------------------------
def oracle_samples(w, problems):
    """oracle_sample over several problems, merged into one rate."""
    res = [oracle_sample(w, b) for b in problems]
    sec = sum(r["seconds"] for r in res)
    applies = sum(r["value"] * r["seconds"] for r in res)
    return {"value": applies / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": " | ".join(r["sample"] for r in res), "seconds": sec}


def oracle_sample(w, problems=None):
    """One gradient contribution (forward solve, residual, adjoint solve, imaging) of one problem
    of the workload, by the FP64 CPU oracle as it stands (numpy, one core)."""
    import oracle as O
    b = w.n_problems // 2 + 3 if problems is None else problems
    f = int(w.problem_fidx()[b])
    s = int(w.problem_src()[b])
    t0 = time.perf_counter()
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas[f:f + 1])
    u0 = orc.incident(0, w.src_cells[s], w.src_force[s])
    u, info_f = orc.solve_info(u0, w.model, 0, tol=TOL)
    r = orc.sample(u, w.rec_cells) - synthetic_data(w)[b]
    q = orc.inject(np.conj(r), w.rec_cells)
    ua, info_a = orc.solve_info(orc.convolve(q, 0), w.model, 0, tol=TOL)
    orc.imaging(ua, u, orc.omegas[0], orc.h)
    dt = time.perf_counter() - t0
    # the oracle's solve_info applies A once more to report the true residual
    applies = 2 * info_f["iters"] + 1 + 2 * info_a["iters"] + 1 + 1
    return {"value": applies * w.nz * w.nx / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"problem {b} (source {s}, {w.freqs_hz[f]:.2f} Hz) of {w.name}: forward solve, residual, "
                      f"adjoint solve, imaging; {applies} operator passes in {dt:.1f} s",
            "seconds": dt}


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
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(0, 1)
    # each step is one problem's gradient contribution (a bounded sample of the batch)
    problems = [w.n_problems // 2 + 3, 0, w.n_problems - 1]
    if args.warmup > 0:  # one untimed sample warms numpy/scipy; more would only add minutes
        oracle_sample(w, problems[0])
    t_applies, t_sec = 0.0, 0.0
    samples = []
    for k in range(args.steps):
        res = oracle_sample(w, problems[k % len(problems)])
        t_applies += res["value"] * res["seconds"]
        t_sec += res["seconds"]
        samples.append(res["sample"])
    value = t_applies / t_sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_sec / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex128)",
            "data": "synthetic", "config": config_dict(w, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1,
                             "sample": "one problem's gradient contribution per step (FP64 numpy oracle): "
                                       + "; ".join(samples[:3])},
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
                   "wavefield (3 persistent launches + input scaling)",
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
    w = workload(0, 1, args.sources)
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
    sm_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6
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
    roof = {"bound": "alu", "achieved": flops / cols_s / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
            "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (measured median)",
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
    w = workload(0, 1, args.sources)
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
    sm_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6
    # the z pass: per (ky, kx) column of every wavefield three forward and three inverse FFTs of
    # length lz (5 L log2 L flops each) and the symmetric 3 x 3 complex product (66 flops) per kz
    cols = P.B * w.ly * w.lx
    z_flops = cols * (6 * 5 * w.lz * math.log2(w.lz) + 66 * w.lz) * args.steps
    z_bytes = (P.B * 2 * 3 * w.nz * w.ly * w.lx * 8 + w.nf * 6 * w.lz * w.ly * w.lx * 8) * args.steps
    z_s = z_ms * 1e-3
    roof = {"bound": "alu", "achieved": z_flops / z_s / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
            "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (measured median)", "traffic": None,
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
