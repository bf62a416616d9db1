"""ls_apply_noalloc: the operator pass for callers that must not allocate device memory while
running. It keeps its scratch in a fixed device array of the library instead of a work buffer;
its output must equal ls_apply's on the same inputs, call after call (the array keeps the previous
call's contents, and nothing in it may leak into the next result). This file is collected last so
that a failure here does not stop the rest of the GPU suite."""
import numpy as np
import pytest
import torch

from paper_2402_02116_gb300 import build, dbi, inputs
from paper_2402_02116_gb300.problem import DeviceProblem

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _rel(a, b):
    a = a.detach().cpu().numpy().astype(np.complex128)
    b = b.detach().cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_ls_apply_on_consecutive_calls():
    build.build()
    dbi.load()
    assert dbi.noalloc_scratch_bytes() == 32 << 20
    # 12 problems of 96 x 80 cells and one of another model: both calls fit the fixed array
    w = inputs.small_case(nz=96, nx=80, n_src=4, freqs=(6.0, 9.0, 14.0), amp=0.12, vti=True, seed=5)
    P = DeviceProblem(w, dbi.C64)
    assert dbi.workspace_bytes(P.grid, P.B, dbi.C64, dbi.OP_APPLY) <= dbi.noalloc_scratch_bytes()
    u1 = P.to_field(inputs.seeded_complex((P.B, 2, w.nz, w.nx), 21))
    u2 = P.to_field(inputs.seeded_complex((P.B, 2, w.nz, w.nx), 22) * 1e-11)
    for u in (u1, u2, u1):  # consecutive calls share the array; each must match on its own
        want = dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u)
        got = dbi.ls_apply_noalloc(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u)
        torch.cuda.synchronize()
        assert _rel(got, want) < 1e-6
    # complex128 through the same array
    P2 = DeviceProblem(w, dbi.C128)
    u = P2.to_field(inputs.seeded_complex((P2.B, 2, w.nz, w.nx), 23))
    want = dbi.ls_apply(P2.grid, P2.ref, P2.m, P2.omega, P2.fidx, P2.Ghat, u)
    got = dbi.ls_apply_noalloc(P2.grid, P2.ref, P2.m, P2.omega, P2.fidx, P2.Ghat, u)
    assert _rel(got, want) < 1e-12


@pytest.mark.parametrize("lz,lx", [(1024, 1024), (768, 768)])
def test_noalloc_on_the_split_stages(lz, lx):
    """The complex64 stages of FFT lengths 1024 and 768 (the contrast-source kernel's scratch and
    the split row and column kernels) through the fixed array: the same result as ls_apply."""
    build.build()
    dbi.load()
    w = inputs.small_case(nz=37, nx=300, lz=lz, lx=lx, n_src=1, freqs=(6.0, 13.0), amp=0.12, seed=6)
    P = DeviceProblem(w, dbi.C64)
    assert dbi.workspace_bytes(P.grid, P.B, dbi.C64, dbi.OP_APPLY) <= dbi.noalloc_scratch_bytes()
    u = P.to_field(inputs.seeded_complex((P.B, 2, w.nz, w.nx), 24))
    want = dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u)
    got = dbi.ls_apply_noalloc(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u)
    torch.cuda.synchronize()
    assert _rel(got, want) < 1e-6


def test_noalloc_rejects_a_batch_beyond_the_array():
    build.build()
    w = inputs.config2_batched_forward(n=256, n_src=4, nf=8)  # 32 problems of 256 x 256
    P = DeviceProblem(w, dbi.C64)
    assert dbi.workspace_bytes(P.grid, P.B, dbi.C64, dbi.OP_APPLY) > dbi.noalloc_scratch_bytes()
    u = P.incident()
    with pytest.raises(dbi.DBIError, match="scratch"):
        dbi.ls_apply_noalloc(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u)


def test_noalloc_allocates_no_device_memory():
    """The entry point's promise, measured: with a preallocated output and after one warm-up call
    (which looks up the array's address), further calls leave both PyTorch's allocation count and
    the device's free memory unchanged, and give the same result every time."""
    build.build()
    dbi.load()
    w = inputs.small_case(nz=64, nx=48, n_src=3, freqs=(7.0, 12.0), amp=0.1, vti=True, seed=9)
    P = DeviceProblem(w, dbi.C64)
    u = P.to_field(inputs.seeded_complex((P.B, 2, w.nz, w.nx), 31))
    out = torch.empty_like(u)
    dbi.ls_apply_noalloc(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u, out=out)
    torch.cuda.synchronize()
    first = out.clone()
    torch.cuda.synchronize()
    allocs = torch.cuda.memory_stats()["allocation.all.allocated"]
    free = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        dbi.ls_apply_noalloc(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u, out=out)
        torch.cuda.synchronize()
    # read the counters before comparing (the comparison itself allocates a result tensor)
    allocs_after = torch.cuda.memory_stats()["allocation.all.allocated"]
    free_after = torch.cuda.mem_get_info()[0]
    assert allocs_after == allocs and free_after == free
    assert torch.equal(out, first)
