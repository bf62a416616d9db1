"""The binding's checks on field and table arguments (CPU only): every wrapper that hands
wavefields, receiver data, Green's tables or per-cell parameters to the library checks that each
holds one block per problem (B = the length of fidx) or the table's nf x components x FFT-grid
points, in the call's dtype, before anything reaches the device, so a wrongly sized or typed tensor
is an error, not a read or write past its end. With CPU tensors a correctly sized and typed call
gets as far as the CUDA check."""
import pytest
import torch

from paper_2402_02116_gb300 import dbi

B, NZ, NX, NY, NREC = 3, 4, 5, 2, 6
C = torch.complex64


def f(*shape):
    return torch.zeros(shape, dtype=C)


def common2d():
    g = dbi.make_grid(NZ, NX, 16, 16, 10.0)
    ref = dbi.make_medium(2000.0, 2000.0, 1155.0)
    m = torch.zeros((5, NZ, NX), dtype=torch.float32)
    omega = torch.ones(1, dtype=torch.float64)
    fidx = torch.zeros(B, dtype=torch.int32)
    rec = torch.zeros((NREC, 2), dtype=torch.int32)
    return g, ref, m, omega, fidx, f(1, 3, 16, 16), rec


def common3d():
    g = dbi.make_grid3(NZ, NY, NX, 16, 16, 16, 10.0)
    ref = dbi.make_medium(2000.0, 2000.0, 1155.0)
    m = torch.zeros((6, NZ, NY, NX), dtype=torch.float32)
    omega = torch.ones(1, dtype=torch.float64)
    fidx = torch.zeros(B, dtype=torch.int32)
    rec = torch.zeros((NREC, 3), dtype=torch.int32)
    return g, ref, m, omega, fidx, f(1, 6, 16, 16, 16), rec


def calls():
    g, ref, m, om, fi, G, rec = common2d()
    u, bad = f(B, 2, NZ, NX), f(B - 1, 2, NZ, NX)
    d, dbad = f(B, NREC, 2), f(B, NREC - 1, 2)
    dm = torch.zeros((5, NZ, NX), dtype=torch.float32)
    g3, ref3, m3, om3, fi3, G3, rec3 = common3d()
    u3, bad3 = f(B, 3, NZ, NY, NX), f(B, 3, NZ, NY, NX - 1)
    d3, d3bad = f(B, NREC, 3), f(B + 1, NREC, 3)
    dm3 = torch.zeros((6, NZ, NY, NX), dtype=torch.float32)
    yield "ls_apply", lambda x: dbi.ls_apply(g, ref, m, om, fi, G, x), u, bad
    yield "ls_apply out", lambda x: dbi.ls_apply(g, ref, m, om, fi, G, u, out=x), u, bad
    yield "ls_apply_noalloc", lambda x: dbi.ls_apply_noalloc(g, ref, m, om, fi, G, x), u, bad
    yield "ls_solve", lambda x: dbi.ls_solve(g, ref, m, om, fi, G, x), u, bad
    yield "ls_solve u0", lambda x: dbi.ls_solve(g, ref, m, om, fi, G, u, u0=x), u, bad
    yield "ls_solve_gmres", lambda x: dbi.ls_solve_gmres(g, ref, m, om, fi, G, x), u, bad
    yield "green_convolve", lambda x: dbi.green_convolve(g, om, fi, G, x), u, bad
    D = f(1, 6, 16, 16)
    yield "ls_apply_k", lambda x: dbi.ls_apply_k(g, ref, m, om, fi, G, D, x), u, bad
    yield "ls_solve_k", lambda x: dbi.ls_solve_k(g, ref, m, om, fi, G, D, x), u, bad
    yield "frechet_apply", lambda x: dbi.frechet_apply(g, ref, m, om, fi, G, x, rec, dm), u, bad
    yield "adjoint_apply u_b", lambda x: dbi.adjoint_apply(g, ref, m, om, fi, G, x, rec, d), u, bad
    yield "adjoint_apply r", lambda x: dbi.adjoint_apply(g, ref, m, om, fi, G, u, rec, x), d, dbad
    yield "data_residual u", lambda x: dbi.data_residual(g, om, fi, rec, x, d), u, bad
    yield "data_residual d_obs", lambda x: dbi.data_residual(g, om, fi, rec, u, x), d, dbad
    yield "normal_cg u_b", lambda x: dbi.normal_cg(g, ref, m, om, fi, G, x, rec, d), u, bad
    yield "normal_cg dd", lambda x: dbi.normal_cg(g, ref, m, om, fi, G, u, rec, x), d, dbad
    yield "ls_apply_3d", lambda x: dbi.ls_apply_3d(g3, ref3, m3, om3, fi3, G3, x), u3, bad3
    yield "ls_solve_3d", lambda x: dbi.ls_solve_3d(g3, ref3, m3, om3, fi3, G3, x), u3, bad3
    yield "frechet_apply_3d", lambda x: dbi.frechet_apply_3d(g3, ref3, m3, om3, fi3, G3, x, rec3, dm3), u3, bad3
    yield "adjoint_apply_3d r", lambda x: dbi.adjoint_apply_3d(g3, ref3, m3, om3, fi3, G3, u3, rec3, x), d3, d3bad
    yield "normal_cg_3d u_b", lambda x: dbi.normal_cg_3d(g3, ref3, m3, om3, fi3, G3, x, rec3, d3), u3, bad3
    yield "normal_cg_3d dd", lambda x: dbi.normal_cg_3d(g3, ref3, m3, om3, fi3, G3, u3, rec3, x), d3, d3bad


CALLS = list(calls())


@pytest.mark.parametrize("name, call, good, bad", CALLS, ids=[c[0] for c in CALLS])
def test_field_sizes_are_checked_before_the_device(name, call, good, bad):
    with pytest.raises(dbi.DBIError, match="holds .* elements"):
        call(bad)
    with pytest.raises(dbi.DBIError, match="CUDA tensor"):
        call(good)


def test_uneven_batch_fields_are_checked_before_the_device():
    """UnevenBatch.apply / solve / tune take flat fields of every slot: a tensor of another size or
    dtype is an error before the work buffer is bound or anything reaches the device."""
    from paper_2402_02116_gb300.group import UnevenBatch
    G = UnevenBatch.__new__(UnevenBatch)  # the checks need only the field size and dtype
    G.field_elems, G.cdt = 40, torch.complex64
    good, short, wide = f(40), f(39), torch.zeros(40, dtype=torch.complex128)
    for call in (lambda x: G.apply(x), lambda x: G.apply(good, out=x), lambda x: G.solve(x),
                 lambda x: G.solve(good, u0=x), lambda x: G.tune(x)):
        for bad in (short, wide):
            with pytest.raises(dbi.DBIError, match="holds .* elements"):
                call(bad)
        with pytest.raises(dbi.DBIError, match="CUDA tensor"):
            call(good)


def typed_calls():
    """(name, call taking the checked argument, a correct value, a wrong value, expected message)."""
    g, ref, m, om, fi, G, rec = common2d()
    u = f(B, 2, NZ, NX)
    wide = torch.zeros((B, 2, NZ, NX), dtype=torch.complex128)
    d = f(B, NREC, 2)
    dm = torch.zeros((5, NZ, NX), dtype=torch.float32)
    D = f(1, 6, 16, 16)
    Gshort, Gwide = f(1, 3, 16, 15), torch.zeros((1, 3, 16, 16), dtype=torch.complex128)
    yield "ls_apply out dtype", lambda x: dbi.ls_apply(g, ref, m, om, fi, G, u, out=x), u, wide, "needs"
    yield "ls_apply_noalloc out dtype", lambda x: dbi.ls_apply_noalloc(g, ref, m, om, fi, G, u, out=x), u, wide, "needs"
    yield "ls_solve u0 dtype", lambda x: dbi.ls_solve(g, ref, m, om, fi, G, u, u0=x), u, wide, "needs"
    yield "ls_solve out dtype", lambda x: dbi.ls_solve(g, ref, m, om, fi, G, u, out=x), u, wide, "needs"
    for name, bad, msg in (("size", Gshort, "FFT-grid points"), ("dtype", Gwide, "needs")):
        yield f"ls_apply Ghat {name}", lambda x: dbi.ls_apply(g, ref, m, om, fi, x, u), G, bad, msg
        yield f"ls_apply_noalloc Ghat {name}", lambda x: dbi.ls_apply_noalloc(g, ref, m, om, fi, x, u), G, bad, msg
        yield f"ls_solve Ghat {name}", lambda x: dbi.ls_solve(g, ref, m, om, fi, x, u), G, bad, msg
        yield f"green_convolve Ghat {name}", lambda x: dbi.green_convolve(g, om, fi, x, u), G, bad, msg
        yield f"frechet_apply Ghat {name}", lambda x: dbi.frechet_apply(g, ref, m, om, fi, x, u, rec, dm), G, bad, msg
        yield f"adjoint_apply Ghat {name}", lambda x: dbi.adjoint_apply(g, ref, m, om, fi, x, u, rec, d), G, bad, msg
        yield f"normal_cg Ghat {name}", lambda x: dbi.normal_cg(g, ref, m, om, fi, x, u, rec, d), G, bad, msg
        yield f"ls_apply_k Ghat {name}", lambda x: dbi.ls_apply_k(g, ref, m, om, fi, x, D, u), G, bad, msg
    yield "ls_apply_k Dhat size", lambda x: dbi.ls_apply_k(g, ref, m, om, fi, G, x, u), D, G, "FFT-grid points"
    yield "incident_field Gspace size", (lambda x: dbi.incident_field(
        g, om, fi, x, torch.zeros((B, 2), dtype=torch.int32), torch.zeros((B, 2), dtype=torch.float64))), \
        G, Gshort, "FFT-grid points"
    yield "frechet_apply dm size", (lambda x: dbi.frechet_apply(g, ref, m, om, fi, G, u, rec, x)), dm, \
        torch.zeros((5, NZ, NX - 1), dtype=torch.float32), "holds"
    yield "frechet_apply dm dtype", (lambda x: dbi.frechet_apply(g, ref, m, om, fi, G, u, rec, x)), dm, \
        torch.zeros((5, NZ, NX), dtype=torch.float64), "needs"
    yield "normal_cg power_start size", (lambda x: dbi.normal_cg(g, ref, m, om, fi, G, u, rec, d, power_start=x)), \
        dm, torch.zeros((4, NZ, NX), dtype=torch.float32), "holds"


TYPED = list(typed_calls())


@pytest.mark.parametrize("name, call, good, bad, msg", TYPED, ids=[c[0] for c in TYPED])
def test_dtypes_and_tables_are_checked_before_the_device(name, call, good, bad, msg):
    """A wrong dtype of an output or initial guess, and a Green's table or per-cell argument of the
    wrong size or dtype, are errors before the device; the correct value reaches the CUDA check."""
    with pytest.raises(dbi.DBIError, match=msg):
        call(bad)
    with pytest.raises(dbi.DBIError, match="CUDA tensor"):
        call(good)


def test_misaligned_complex_tensors_are_errors_before_the_device():
    """A complex view whose start is off a 16-byte boundary (the kernels read complex64 pairs and
    Green's tables with 16-byte loads, which would fault there) is rejected before any device work,
    as a field, an output and a table; an aligned tensor gets as far as the CUDA check."""
    g, ref, m, om, fi, G, rec = common2d()
    u = f(B, 2, NZ, NX)
    shifted = torch.zeros(u.numel() + 1, dtype=torch.complex64)[1:].view(B, 2, NZ, NX)
    assert shifted.data_ptr() % 16 == 8
    Gs = torch.zeros(G.numel() + 1, dtype=torch.complex64)[1:].view(G.shape)
    for call in (lambda: dbi.ls_apply(g, ref, m, om, fi, G, shifted),
                 lambda: dbi.ls_apply(g, ref, m, om, fi, G, u, out=shifted),
                 lambda: dbi.ls_solve(g, ref, m, om, fi, G, shifted),
                 lambda: dbi.ls_solve_gmres(g, ref, m, om, fi, G, shifted),
                 lambda: dbi.green_convolve(g, om, fi, G, shifted),
                 lambda: dbi.ls_apply(g, ref, m, om, fi, Gs, u),
                 lambda: dbi.ls_solve(g, ref, m, om, fi, Gs, u)):
        with pytest.raises(dbi.DBIError, match="multiple of 16 bytes"):
            call()
    with pytest.raises(dbi.DBIError, match="CUDA tensor"):
        dbi.ls_apply(g, ref, m, om, fi, G, u)


def test_caller_work_buffers_are_checked():
    """A work buffer the caller passes to ls_apply / ls_solve must be a contiguous, 16-byte aligned
    tensor on the call's device; its size is counted in bytes whatever its element type."""
    dev = torch.device("cuda", 0)
    with pytest.raises(dbi.DBIError, match="multiple of 16 bytes"):
        dbi._caller_work(torch.zeros(65, dtype=torch.uint8)[1:], dev)
    with pytest.raises(dbi.DBIError, match="CUDA tensor"):
        dbi._caller_work(torch.zeros(64, dtype=torch.uint8), dev)
    with pytest.raises(dbi.DBIError, match="torch tensor"):
        dbi._caller_work(bytearray(64), dev)
