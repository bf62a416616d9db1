"""Sharding of the (source, frequency) problems over ranks, with world_size = 2 gloo processes on
CPU: the gradients of the two shards, summed by the all-reduce, equal the gradient of the whole
batch. The per-rank gradients come from the CPU oracle (no GPU here); the host logic under test
(which rank owns which sources, the all-reduce of the gradient and of the misfit) is the one
bench.py uses on GPUs."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2402_02116_gb300 import inputs
from paper_2402_02116_gb300.shard import reduce_gradient, shard_sources, shard_workload


def test_shards_partition_the_sources():
    for n, world in ((32, 2), (32, 4), (7, 3), (1, 2)):
        parts = [shard_sources(n, r, world) for r in range(world)]
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(n))
        assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        shard_sources(4, 2, 2)


def _workload():
    return inputs.small_case(nz=8, nx=7, amp=0.1, vti=True, n_src=3, freqs=(8.0, 12.0), seed=61)


def _gradient(w, d_obs_all):
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    fidx = w.problem_fidx()
    srcs, forces = w.src_cells[w.problem_src()], w.src_force[w.problem_src()]
    return orc.misfit(w.model, fidx, srcs, forces, d_obs_all, w.rec_cells)


def _observed(w):
    return inputs.seeded_complex((w.n_problems, len(w.rec_cells), 2), 5) * 1e-11


def _rank_main(rank, world, port, out_path):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = _workload()
    d_all = _observed(w).reshape(w.nf, w.n_src, len(w.rec_cells), 2)
    mine = shard_sources(w.n_src, rank, world)
    ws = shard_workload(w, rank, world)
    d_obs = d_all[:, mine].reshape(-1, len(w.rec_cells), 2)
    phi, g, _ = _gradient(ws, d_obs)
    gt = torch.as_tensor(g)
    pt = torch.tensor(phi, dtype=torch.float64)
    reduce_gradient(gt, pt)
    if rank == 0:
        np.save(out_path, np.concatenate([gt.numpy().ravel(), [pt.item()]]))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_gradient_equals_single_process(tmp_path):
    out = os.path.join(tmp_path, "g.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    w = _workload()
    phi, g, _ = _gradient(w, _observed(w))
    want = np.concatenate([g.ravel(), [phi]])
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def _workload_3d():
    return inputs.small_case_3d(nz=4, ny=3, nx=5, n_src=3, freqs=(8.0, 12.0), seed=62)


def _adjoint_3d(w, r_all):
    """Re J^H r of the 3D operator summed over the problems of workload `w` (oracle, FP64)."""
    orc = O.o3d.LSOracle3D(w.nz, w.ny, w.nx, w.h, w.lz, w.ly, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    fidx = w.problem_fidx()
    srcs, forces = w.src_cells[w.problem_src()], w.src_force[w.problem_src()]
    U_b = np.stack([orc.solve(orc.incident(f, tuple(s), fv), w.model, f, tol=1e-13)[0]
                    for f, s, fv in zip(fidx, srcs, forces)])
    return O.o3d.adjoint_3d(orc, w.model, U_b, fidx, r_all, w.rec_cells, tol=1e-13)


def _residual_3d(w):
    return inputs.seeded_complex((w.n_problems, len(w.rec_cells), 3), 7)


def _rank_main_3d(rank, world, port, out_path):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = _workload_3d()
    r_all = _residual_3d(w).reshape(w.nf, w.n_src, len(w.rec_cells), 3)
    mine = shard_sources(w.n_src, rank, world)
    ws = shard_workload(w, rank, world)
    gt = torch.as_tensor(_adjoint_3d(ws, r_all[:, mine].reshape(-1, len(w.rec_cells), 3)))
    reduce_gradient(gt)
    if rank == 0:
        np.save(out_path, gt.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_3d_adjoint_equals_single_process(tmp_path):
    """The same partition for the 3D products: six parameters per cell, one all-reduce."""
    out = os.path.join(tmp_path, "g3.npy")
    mp.spawn(_rank_main_3d, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    w = _workload_3d()
    want = _adjoint_3d(w, _residual_3d(w))
    assert got.shape == (6, w.nz, w.ny, w.nx)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
