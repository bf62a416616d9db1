"""Uneven batches (include/dbi_group.h) on the GPU: problems of different grid sizes, models,
frequencies and source counts in one persistent launch per operator stage, against the FP64 oracle
(every slot of a small mixed batch), against the single-grid path (the same tile bodies), with
graph-captured Krylov iterations, after autotuning, and on
the full 40-problem uneven workload (64^2 .. 512^2; sampled slots against the oracle, every slot
by its residual)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2402_02116_gb300 import build, dbi, inputs
from paper_2402_02116_gb300.group import UnevenBatch
from paper_2402_02116_gb300.problem import DeviceProblem

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = {dbi.C64: 1e-5, dbi.C128: 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dbi.load()


def npy(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# A small mixed batch: ragged shapes, non-square and oversized FFT grids, one-row and one-slot
# members, isotropic and VTI backgrounds, several row and column tiles, FFT lengths 1024 and 768.
MINI = [
    dict(nz=12, nx=10, n_src=2, freqs=(8.0, 14.0), seed=71),
    dict(nz=5, nx=9, lz=16, lx=32, n_src=1, freqs=(11.0,), seed=72),
    dict(nz=40, nx=24, vti=True, n_src=3, freqs=(6.0, 9.0), seed=73),
    dict(nz=1, nx=8, n_src=1, freqs=(10.0,), seed=74),
    dict(nz=20, nx=20, vti=True, lz=64, lx=64, n_src=2, freqs=(12.0,), seed=75),
    dict(nz=30, nx=60, n_src=2, freqs=(5.0, 7.0), seed=76),
    # FFT length 1024 along one or both axes: complex64 runs these stages on the split kernels
    # (pairs of 512-point transforms, the source kernel in 32-row tiles) beside the others
    dict(nz=35, nx=33, lz=1024, lx=1024, vti=True, n_src=1, freqs=(9.0,), seed=77),
    dict(nz=9, nx=50, lz=32, lx=1024, n_src=1, freqs=(13.0,), seed=78),
    dict(nz=40, nx=7, lz=1024, lx=16, n_src=1, freqs=(6.0,), seed=79),
    # FFT length 768 (complex64: triples of 256-point transforms), alone and beside 1024
    dict(nz=29, nx=300, lz=768, lx=768, vti=True, n_src=1, freqs=(8.0,), seed=81),
    dict(nz=33, nx=257, lz=1024, lx=768, n_src=1, freqs=(12.0,), seed=82),
    dict(nz=300, nx=12, lz=768, lx=32, n_src=1, freqs=(7.0,), seed=83),
]


def mini_workloads(precision=dbi.C64):
    """The small mixed batch (complex128: without the length-768 members, a complex64 length)."""
    return [inputs.small_case(amp=0.1, **kw) for kw in MINI
            if precision == dbi.C64 or 768 not in (kw.get("lz"), kw.get("lx"))]


def member_oracle(w, omegas=None):
    return O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0,
                      w.omegas if omegas is None else omegas)


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_group_apply_matches_oracle(precision):
    ws = mini_workloads(precision)
    Ps = [DeviceProblem(w, precision) for w in ws]
    G = UnevenBatch(Ps, precision)
    u = G.join([torch.as_tensor(inputs.seeded_complex((P.B, 2, P.w.nz, P.w.nx), 80 + k)).to(P.device, P.cdt)
                for k, P in enumerate(Ps)])
    out = G.split(G.apply(u))
    uin = G.split(u)
    for k, (w, P) in enumerate(zip(ws, Ps)):
        orc = member_oracle(w)
        fidx = w.problem_fidx()
        for q in range(P.B):
            want = orc.apply(npy(uin[k][q]).astype(np.complex128), w.model, fidx[q])
            assert rel(npy(out[k][q]), want) < TOL[precision], (k, q)


def test_group_apply_equals_single_grid_path():
    """Each slot of the uneven batch equals the single-grid batched call to FP32 rounding (the same
    tile bodies, compiled into another kernel, may contract multiply-adds differently)."""
    ws = mini_workloads() + inputs.config5_uneven(sizes=(64, 128, 256, 384, 512), n_members=6, max_src=3,
                                                  max_f=2, seed=15)
    Ps = [DeviceProblem(w, dbi.C64) for w in ws]
    G = UnevenBatch(Ps, dbi.C64)
    u = G.join([P.incident() for P in Ps])
    out = G.split(G.apply(u))
    for k, (P, uk) in enumerate(zip(Ps, G.split(u))):
        assert rel(npy(out[k]), npy(P.apply(uk.contiguous()))) < 1e-6, k


@pytest.mark.parametrize("precision,graph", [(dbi.C128, True), (dbi.C128, False), (dbi.C64, True)])
def test_group_solve_matches_oracle(precision, graph):
    ws = mini_workloads(precision)
    Ps = [DeviceProblem(w, precision) for w in ws]
    G = UnevenBatch(Ps, precision)
    rhs = G.incident()
    tol = 1e-11 if precision == dbi.C128 else 1e-6
    u, iters, relres, code = G.solve(rhs, tol=tol, max_iter=500, check_every=4, graph=graph)
    assert bool((code == dbi.CONVERGED).all()) and float(relres.max()) <= tol
    uk = G.split(u)
    for k, (w, P) in enumerate(zip(ws, Ps)):
        orc = member_oracle(w)
        fidx, srcs = w.problem_fidx(), w.problem_src()
        for q in range(P.B):
            u0 = orc.incident(fidx[q], w.src_cells[srcs[q]], w.src_force[srcs[q]])
            want = orc.solve(u0, w.model, fidx[q], tol=1e-13)
            assert rel(npy(uk[k][q]), want) < (1e-8 if precision == dbi.C128 else 1e-5), (k, q)


def test_graph_replay_gives_the_same_bits_and_launch_count():
    ws = mini_workloads()
    Ps = [DeviceProblem(w, dbi.C64) for w in ws]
    G = UnevenBatch(Ps, dbi.C64)
    rhs = G.incident()
    G.bind(dbi.OP_SOLVE)  # (binding launches the twiddle kernel once)
    torch.cuda.synchronize()
    n0 = dbi.kernel_launches()
    u1, it1, rr1, c1 = G.solve(rhs, tol=1e-6, max_iter=400, check_every=4, graph=False)
    torch.cuda.synchronize()
    n1 = dbi.kernel_launches()
    u2, it2, rr2, c2 = G.solve(rhs, tol=1e-6, max_iter=400, check_every=4, graph=True)
    torch.cuda.synchronize()
    n2 = dbi.kernel_launches()
    assert torch.equal(u1, u2) and torch.equal(it1, it2) and torch.equal(c1, c2)
    assert n2 - n1 == n1 - n0  # every replayed kernel is counted


def test_group_apply_can_be_captured_by_the_caller():
    """After binding, ls_apply_group allocates nothing and never synchronises: a torch CUDA graph of
    it replays to the eager result on new inputs."""
    ws = mini_workloads()
    Ps = [DeviceProblem(w, dbi.C64) for w in ws]
    G = UnevenBatch(Ps, dbi.C64)
    u_static = G.incident()
    out_static = torch.empty_like(u_static)
    G.bind(dbi.OP_APPLY)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        G.apply(u_static, out=out_static)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        G.apply(u_static, out=out_static)
    u_new = G.join([torch.as_tensor(inputs.seeded_complex((P.B, 2, P.w.nz, P.w.nx), 90 + k)).to(P.device, P.cdt)
                    for k, P in enumerate(Ps)])
    u_static.copy_(u_new)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out_static, G.apply(u_new))


def test_autotuner_reports_and_keeps_the_result():
    ws = inputs.config5_uneven(sizes=(64, 128, 256), n_members=8, max_src=4, max_f=2, seed=25)
    Ps = [DeviceProblem(w, dbi.C64) for w in ws]
    G = UnevenBatch(Ps, dbi.C64)
    u = G.incident()
    before = G.apply(u)
    rep = G.tune(u)
    lens = sorted(L for L, _, _ in rep["lengths"])
    assert lens == sorted({w.lx for w in ws} | {w.lz for w in ws})
    for L, plan, (t0, t1) in rep["lengths"]:
        if L not in (64, 512):
            assert plan in (0, 1) and t0 > 0 and t1 > 0 and (t1 < t0) == (plan == 1)
    assert all(1 <= c <= m for c, m in zip(rep["ctas_per_sm"], rep["max_ctas"]))
    after = G.apply(u)
    for k in range(len(Ps)):  # a different radix order changes only the rounding
        assert rel(npy(G.split(after)[k]), npy(G.split(before)[k])) < 1e-6


def test_uneven_workload_40_problems():
    """The 40-problem uneven batch (grids 64^2 .. 512^2, 1-32 sources, 1-8 frequencies in 2-25 Hz,
    isotropic or VTI): tuned, then solved to 1e-5 with graph-captured iterations. Every slot
    converges and its true residual, by an independent operator pass, stays near the tolerance;
    one slot of each grid size is checked against the oracle's operator and its solution's
    residual under the oracle's operator."""
    ws = inputs.config5_uneven()
    Ps = [DeviceProblem(w, dbi.C64) for w in ws]
    G = UnevenBatch(Ps, dbi.C64)
    rhs = G.incident()
    rep = G.tune(rhs)
    assert rep["apply_ms"] > 0
    u, iters, relres, code = G.solve(rhs, tol=1e-5, max_iter=3000, check_every=8, graph=True)
    assert bool((code == dbi.CONVERGED).all()), np.unique(npy(code), return_counts=True)
    Au = G.apply(u)
    r = (Au - rhs)
    offs = G.offsets
    for b in range(G.slots):
        a, e = offs[b], offs[b + 1]
        assert float(torch.linalg.norm(r[a:e]) / torch.linalg.norm(rhs[a:e])) < 3e-5, b
    # one slot per grid size against the oracle
    seen = set()
    uk, rk, ak = G.split(u), G.split(rhs), G.split(Au)
    for k, (w, P) in enumerate(zip(ws, Ps)):
        if w.nz in seen:
            continue
        seen.add(w.nz)
        q = P.B - 1
        f = int(w.problem_fidx()[q])
        orc = member_oracle(w, omegas=[w.omegas[f]])
        x = npy(uk[k][q]).astype(np.complex128)
        A_x = orc.apply(x, w.model, 0)
        assert rel(npy(ak[k][q]), A_x) < 1e-5, (w.nz, "operator")
        assert rel(A_x, npy(rk[k][q])) < 3e-5, (w.nz, "residual")
    assert seen == {64, 128, 256, 384, 512}
