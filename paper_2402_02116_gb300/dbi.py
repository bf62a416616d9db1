"""Python binding of the C ABI in include/dbi.h (ctypes; argument marshalling only).

Every function here allocates its outputs and the work buffer with PyTorch on the inputs' CUDA
device, passes raw pointers and the current CUDA stream to `libdbi.so`, and raises DBIError when
the library returns a non-zero code. All arithmetic runs in the library's CUDA kernels; there is
no CPU path. The library must have been built (`paper_2402_02116_gb300.build.build()`); loading
fails loudly otherwise.

Precision follows the tensors: complex64 fields use the DBI_C64 path (float model arrays),
complex128 fields the DBI_C128 path (double model arrays).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_size_t, c_void_p

import torch

from . import build as _build

C64, C128 = 0, 1
OP_GREENS, OP_CONVOLVE, OP_APPLY, OP_SOLVE, OP_FRECHET, OP_ADJOINT, OP_NORMAL_CG = range(7)
OP_GREENS_K, OP_APPLY_K, OP_SOLVE_K = 7, 8, 9
CONVERGED, NOT_CONVERGED, BREAKDOWN, NONFINITE = 0, 1, 2, 3


class DBIError(RuntimeError):
    pass


class Grid(ctypes.Structure):
    _fields_ = [("nz", c_int), ("nx", c_int), ("lz", c_int), ("lx", c_int), ("h", c_double)]


class Medium(ctypes.Structure):
    _fields_ = [("rho0", c_double), ("alpha0", c_double), ("beta0", c_double),
                ("c11", c_double), ("c13", c_double), ("c33", c_double), ("c55", c_double)]


class Model(ctypes.Structure):
    _fields_ = [("grid", Grid), ("ref", Medium), ("m", c_void_p)]


class Grid3(ctypes.Structure):
    _fields_ = [("nz", c_int), ("ny", c_int), ("nx", c_int), ("lz", c_int), ("ly", c_int), ("lx", c_int),
                ("h", c_double)]


class Model3(ctypes.Structure):
    _fields_ = [("grid", Grid3), ("ref", Medium), ("m", c_void_p)]


class Batch(ctypes.Structure):
    _fields_ = [("B", c_int), ("nf", c_int), ("omega", c_void_p), ("fidx", c_void_p)]


class Receivers(ctypes.Structure):
    _fields_ = [("n", c_int), ("cells", c_void_p)]


class KrylovOpts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_iter", c_int), ("check_every", c_int), ("zero_guess", c_int)]


class Status(ctypes.Structure):
    _fields_ = [("iters", c_void_p), ("relres", c_void_p), ("code", c_void_p)]


class CGOpts(ctypes.Structure):
    _fields_ = [("iters", c_int), ("lam", c_double), ("lambda_rel", c_double), ("power_iters", c_int)]


class GroupMember(ctypes.Structure):
    _fields_ = [("model", Model), ("Ghat", c_void_p), ("omega", c_void_p), ("nf", c_int), ("B", c_int),
                ("fidx", c_void_p)]


class GroupTuning(ctypes.Structure):
    _fields_ = [("lengths", c_int * 8), ("plan", c_int * 8), ("plan_ms", (c_double * 2) * 8),
                ("ctas_per_sm", c_int * 3), ("max_ctas", c_int * 3), ("apply_ms", c_double)]


GROUP_GRAPH = 1

# (name, restype, argtypes) of every entry point declared in include/dbi.h and include/dbi_group.h
SIGNATURES = {
    "dbi_last_error": (ctypes.c_char_p, []),
    "dbi_version": (c_int, []),
    "dbi_workspace_bytes": (c_size_t, [POINTER(Grid), c_int, c_int, c_int]),
    "dbi_kernel_launches": (ctypes.c_ulonglong, []),
    "dbi_profile_begin": (c_int, [c_int]),
    "dbi_profile_end": (c_int, [POINTER(c_double), POINTER(ctypes.c_longlong)]),
    "dbi_fma_probe": (ctypes.c_longlong, [c_int, c_int, c_void_p, c_void_p]),
    "greens_tabulate": (c_int, [POINTER(Grid), POINTER(Medium), c_void_p, c_int, c_int, c_void_p,
                                c_void_p, c_void_p, c_size_t, c_void_p]),
    "incident_field": (c_int, [POINTER(Grid), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_void_p,
                               c_int, c_void_p]),
    "green_convolve": (c_int, [POINTER(Grid), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_int,
                               c_void_p, c_size_t, c_void_p]),
    "ls_apply": (c_int, [POINTER(Model), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_int, c_void_p,
                         c_size_t, c_void_p]),
    "ls_apply_noalloc": (c_int, [POINTER(Model), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "dbi_noalloc_scratch_bytes": (c_size_t, []),
    "dbi_group_create": (c_int, [POINTER(GroupMember), c_int, c_int, POINTER(c_void_p)]),
    "dbi_group_destroy": (None, [c_void_p]),
    "dbi_group_slots": (c_int, [c_void_p]),
    "dbi_group_field_elems": (ctypes.c_longlong, [c_void_p]),
    "dbi_group_offsets": (c_int, [c_void_p, POINTER(ctypes.c_longlong)]),
    "dbi_group_workspace_bytes": (c_size_t, [c_void_p, c_int]),
    "dbi_group_bind": (c_int, [c_void_p, c_void_p, c_size_t, c_int, c_void_p]),
    "ls_apply_group": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ls_solve_group": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(KrylovOpts), POINTER(Status), c_int,
                               c_void_p]),
    "dbi_group_tune": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(GroupTuning)]),
    "dbi_set_radix_plan": (c_int, [c_int, c_int, c_int]),
    "ls_solve": (c_int, [POINTER(Model), POINTER(Batch), c_void_p, c_void_p, c_void_p, POINTER(KrylovOpts),
                         POINTER(Status), c_int, c_void_p, c_size_t, c_void_p]),
    "dbi_gmres_workspace_bytes": (c_size_t, [POINTER(Grid), c_int, c_int, c_int]),
    "ls_solve_gmres": (c_int, [POINTER(Model), POINTER(Batch), c_void_p, c_void_p, c_void_p, POINTER(KrylovOpts),
                               c_int, POINTER(Status), c_int, c_void_p, c_size_t, c_void_p]),
    "dbi_workspace_bytes_3d": (c_size_t, [POINTER(Grid3), c_int, c_int, c_int, c_int]),
    "greens_tabulate_3d": (c_int, [POINTER(Grid3), POINTER(Medium), c_void_p, c_int, c_int, c_void_p, c_void_p,
                                   c_void_p, c_size_t, c_void_p]),
    "incident_field_3d": (c_int, [POINTER(Grid3), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                                  c_void_p]),
    "ls_apply_3d": (c_int, [POINTER(Model3), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_int, c_void_p,
                            c_size_t, c_void_p]),
    "ls_solve_3d": (c_int, [POINTER(Model3), POINTER(Batch), c_void_p, c_void_p, c_void_p, POINTER(KrylovOpts),
                            c_int, POINTER(Status), c_int, c_void_p, c_size_t, c_void_p]),
    "dbi_products_workspace_bytes_3d": (c_size_t, [POINTER(Grid3), c_int, c_int, c_int]),
    "frechet_apply_3d": (c_int, [POINTER(Model3), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_int, c_void_p,
                                 c_void_p, POINTER(KrylovOpts), c_int, POINTER(Status), c_int, c_void_p, c_size_t,
                                 c_void_p]),
    "adjoint_apply_3d": (c_int, [POINTER(Model3), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_int, c_void_p,
                                 c_void_p, POINTER(KrylovOpts), c_int, POINTER(Status), c_int, c_void_p, c_size_t,
                                 c_void_p]),
    "dbi_normal_cg_workspace_bytes_3d": (c_size_t, [POINTER(Grid3), c_int, c_int, c_int, c_int, c_int]),
    "normal_cg_3d": (c_int, [POINTER(Model3), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_int, c_void_p,
                             POINTER(CGOpts), c_void_p, c_void_p, POINTER(c_double), POINTER(c_double),
                             POINTER(KrylovOpts), c_int, POINTER(Status), c_int, c_void_p, c_size_t, c_void_p]),
    "sample_3d": (c_int, [POINTER(Grid3), c_int, c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p]),
    "greens_tabulate_k": (c_int, [POINTER(Grid), POINTER(Medium), c_void_p, c_int, c_int, c_void_p, c_void_p,
                                  c_size_t, c_void_p]),
    "ls_apply_k": (c_int, [POINTER(Model), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                           c_void_p, c_size_t, c_void_p]),
    "ls_solve_k": (c_int, [POINTER(Model), POINTER(Batch), c_void_p, c_void_p, c_void_p, c_void_p,
                           POINTER(KrylovOpts), POINTER(Status), c_int, c_void_p, c_size_t, c_void_p]),
    "frechet_apply": (c_int, [POINTER(Model), POINTER(Batch), c_void_p, c_void_p, POINTER(Receivers),
                              c_void_p, c_void_p, POINTER(KrylovOpts), POINTER(Status), c_int, c_void_p,
                              c_size_t, c_void_p]),
    "adjoint_apply": (c_int, [POINTER(Model), POINTER(Batch), c_void_p, c_void_p, POINTER(Receivers),
                              c_void_p, c_void_p, POINTER(KrylovOpts), POINTER(Status), c_int, c_void_p,
                              c_size_t, c_void_p]),
    "data_residual": (c_int, [POINTER(Grid), POINTER(Batch), POINTER(Receivers), c_void_p, c_void_p,
                              c_void_p, c_void_p, c_int, c_void_p]),
    "normal_cg": (c_int, [POINTER(Model), POINTER(Batch), c_void_p, c_void_p, POINTER(Receivers), c_void_p,
                          POINTER(CGOpts), c_void_p, c_void_p, POINTER(c_double), POINTER(c_double),
                          POINTER(KrylovOpts), POINTER(Status), c_int, c_void_p, c_size_t, c_void_p]),
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libdbi.so (once) and declare its entry points; raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or library_path()
    if not os.path.exists(path):
        raise DBIError(f"CUDA library not built: {path} is missing; run paper_2402_02116_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(rc: int, name: str):
    if rc != 0:
        msg = load().dbi_last_error().decode(errors="replace")
        raise DBIError(f"{name} returned {rc}: {msg}")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _precision(t: torch.Tensor) -> int:
    if t.dtype == torch.complex64:
        return C64
    if t.dtype == torch.complex128:
        return C128
    raise DBIError(f"fields must be complex64 or complex128, got {t.dtype}")


def real_dtype(precision: int):
    return torch.float32 if precision == C64 else torch.float64


def complex_dtype(precision: int):
    return torch.complex64 if precision == C64 else torch.complex128


def _aligned16(name, t):
    """The kernels read and write complex64 fields and tables, and the work buffer's carves, with
    16-byte accesses (pairs of complex64 values, 16-byte table loads and asynchronous copies), which
    a misaligned address turns into a device fault. PyTorch's allocations are aligned; a view whose
    storage offset moves its start off a 16-byte boundary is an error here."""
    if t.numel() and t.data_ptr() % 16:
        raise DBIError(f"{name} starts at an address that is not a multiple of 16 bytes (storage offset "
                       f"{t.storage_offset()}); the kernels need 16-byte aligned complex and work buffers")


def _need_cuda(*ts):
    for t in ts:
        if t is not None and t.is_complex():
            _aligned16("a complex tensor", t)
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise DBIError("every tensor must be a contiguous CUDA tensor")


def _caller_work(work, device) -> int:
    """A work buffer supplied by the caller: a contiguous tensor on the call's device, 16-byte
    aligned; returns its size in bytes (the library checks that it covers the call's carves)."""
    if not isinstance(work, torch.Tensor):
        raise DBIError("work must be a torch tensor")
    _aligned16("work", work)
    if not work.is_cuda or not work.is_contiguous() or work.device != device:
        raise DBIError(f"work must be a contiguous CUDA tensor on {device}")
    return work.numel() * work.element_size()


def _fields(fidx, comps: int, cells: int, dtype, **named) -> list:
    """Every field argument is a tensor of the call's complex dtype holding one [comps][cells] block
    per problem (B = the length of fidx), which the kernels index from its first element: a tensor
    of another size or element type would be read or written past its end. Returns the tensors,
    which the caller then passes to _need_cuda with the others (a host tensor would hand the kernels
    a host address): every size and dtype is checked before any device."""
    B = int(fidx.numel())
    ts = {k: t for k, t in named.items() if t is not None}
    for name, t in ts.items():
        if not isinstance(t, torch.Tensor):
            raise DBIError(f"{name} must be a torch tensor")
        if t.numel() != B * comps * cells:
            raise DBIError(f"{name} holds {t.numel()} elements; {B} problems x {comps} components x "
                           f"{cells} cells need {B * comps * cells}")
    for name, t in ts.items():
        if t.dtype != dtype:
            raise DBIError(f"{name} is {t.dtype}; this call needs {dtype}")
    return list(ts.values())


def _checked(name, t, n: int, dtype, what: str):
    if not isinstance(t, torch.Tensor):
        raise DBIError(f"{name} must be a torch tensor")
    if t.numel() != n:
        raise DBIError(f"{name} holds {t.numel()} elements; {what} need {n}")
    if t.dtype != dtype:
        raise DBIError(f"{name} is {t.dtype}; this call needs {dtype}")


def _table(name, t, nf: int, comps: int, cells: int, dtype):
    """A Green's table argument (Ghat, Dhat, Gspace): a tensor of the call's complex dtype with
    nf x comps x cells elements (cells = the FFT grid's points); the caller checks the device."""
    _checked(name, t, nf * comps * cells, dtype, f"{nf} frequencies x {comps} components x {cells} FFT-grid points")


def _real(name, t, n: int, dtype):
    """A real per-cell argument (a model perturbation, a CG start): dtype and n elements; the caller
    checks the device."""
    _checked(name, t, n, dtype, "the parameters x cells")


def make_grid(nz, nx, lz, lx, h) -> Grid:
    return Grid(int(nz), int(nx), int(lz), int(lx), float(h))


def make_medium(rho0, alpha0, beta0) -> Medium:
    return Medium(float(rho0), float(alpha0), float(beta0), 0.0, 0.0, 0.0, 0.0)


def make_medium_vti(rho0, c11, c13, c33, c55) -> Medium:
    """A homogeneous VTI reference (its Green's tensor is tabulated from the spectral
    representation); alpha0, beta0 are filled with the mean P and the S velocity for reference."""
    a0 = ((c11 + c33) / (2.0 * rho0)) ** 0.5
    b0 = (c55 / rho0) ** 0.5
    return Medium(float(rho0), float(a0), float(b0), float(c11), float(c13), float(c33), float(c55))


def workspace_bytes(grid: Grid, B: int, precision: int, op: int) -> int:
    return int(load().dbi_workspace_bytes(ctypes.byref(grid), int(B), int(precision), int(op)))


def _work(grid, B, precision, op, device):
    n = workspace_bytes(grid, B, precision, op)
    if n == 0:
        raise DBIError("invalid grid or precision for the workspace query")
    return torch.empty(n, dtype=torch.uint8, device=device), n


def _batch(omega: torch.Tensor, fidx: torch.Tensor) -> Batch:
    if omega.dtype != torch.float64 or fidx.dtype != torch.int32:
        raise DBIError("omega must be float64 and fidx int32")
    _need_cuda(omega, fidx)
    return Batch(int(fidx.numel()), int(omega.numel()), omega.data_ptr(), fidx.data_ptr())


def _model(grid, ref, m, precision) -> Model:
    if m.dtype != real_dtype(precision):
        raise DBIError(f"model must be {real_dtype(precision)} for this precision, got {m.dtype}")
    _need_cuda(m)
    if tuple(m.shape) != (5, grid.nz, grid.nx):
        raise DBIError(f"model shape {tuple(m.shape)} != (5, {grid.nz}, {grid.nx})")
    return Model(grid, ref, m.data_ptr())


def _receivers(cells: torch.Tensor) -> Receivers:
    if cells.dtype != torch.int32:
        raise DBIError("receiver cells must be int32 [n][2]")
    _need_cuda(cells)
    return Receivers(int(cells.shape[0]), cells.data_ptr())


def _kopts(tol, max_iter, check_every, zero_guess=False) -> KrylovOpts:
    return KrylovOpts(float(tol), int(max_iter), int(check_every), int(bool(zero_guess)))


def _status(B, device):
    iters = torch.zeros(B, dtype=torch.int32, device=device)
    relres = torch.zeros(B, dtype=torch.float64, device=device)
    code = torch.zeros(B, dtype=torch.int32, device=device)
    return (iters, relres, code), Status(iters.data_ptr(), relres.data_ptr(), code.data_ptr())


PROF_ROWS_FORWARD, PROF_COLS, PROF_ROWS_INVERSE, PROF_OPERATOR = 1, 2, 3, 4


def set_radix_plan(precision: int, L: int, plan: int):
    """Radix plan (0: radix-8 passes first, 1: the smaller radix first) of FFT length L for the
    single-grid entry points."""
    _check(load().dbi_set_radix_plan(int(precision), int(L), int(plan)), "dbi_set_radix_plan")


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().dbi_kernel_launches())


def profile_begin(stage: int):
    _check(load().dbi_profile_begin(int(stage)), "dbi_profile_begin")


def fma_probe(blocks: int, iters: int, device) -> tuple:
    """Launch the FP32 FMA probe on the current stream of `device`; returns (flops, output tensor)."""
    out = torch.empty(int(blocks) * 256, dtype=torch.float32, device=device)
    n = int(load().dbi_fma_probe(int(blocks), int(iters), _ptr(out), _stream(out.device)))
    if n < 0:
        _check(n, "dbi_fma_probe")
    return n, out


def profile_end():
    """(summed ms, launches) of the stage timed since profile_begin."""
    ms, n = c_double(0.0), ctypes.c_longlong(0)
    _check(load().dbi_profile_end(ctypes.byref(ms), ctypes.byref(n)), "dbi_profile_end")
    return float(ms.value), int(n.value)


# ---------------------------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------------------------
def greens_tabulate(grid: Grid, ref: Medium, omega: torch.Tensor, precision: int = C64,
                    with_space: bool = True):
    """Ghat [nf][3][lx][lz] (h^2/(lz lx) FFT(G), column-major) and, if asked, Gspace
    [nf][3][lz][lx]."""
    _need_cuda(omega)
    dev = omega.device
    nf = int(omega.numel())
    cd = complex_dtype(precision)
    Ghat = torch.empty((nf, 3, grid.lx, grid.lz), dtype=cd, device=dev)
    Gspace = torch.empty((nf, 3, grid.lz, grid.lx), dtype=cd, device=dev) if with_space else None
    work, n = _work(grid, nf, precision, OP_GREENS, dev)
    _check(load().greens_tabulate(ctypes.byref(grid), ctypes.byref(ref), _ptr(omega), nf, precision,
                                  _ptr(Ghat), _ptr(Gspace), _ptr(work), n, _stream(dev)), "greens_tabulate")
    return Ghat, Gspace


def incident_field(grid: Grid, omega, fidx, Gspace, src_cells, forces):
    """u0 [B][2][nz][nx] = G_h(x - x_s) f for every problem."""
    precision = _precision(Gspace)
    _table("Gspace", Gspace, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    _need_cuda(Gspace, src_cells, forces)
    if src_cells.dtype != torch.int32 or forces.dtype != torch.float64:
        raise DBIError("src_cells must be int32 [B][2] and forces float64 [B][2]")
    batch = _batch(omega, fidx)
    u0 = torch.empty((batch.B, 2, grid.nz, grid.nx), dtype=Gspace.dtype, device=Gspace.device)
    _check(load().incident_field(ctypes.byref(grid), ctypes.byref(batch), _ptr(Gspace), _ptr(src_cells),
                                 _ptr(forces), _ptr(u0), precision, _stream(Gspace.device)), "incident_field")
    return u0


def green_convolve(grid: Grid, omega, fidx, Ghat, src):
    """h^2 G * src for every problem."""
    precision = _precision(src)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), src=src)
    _table("Ghat", Ghat, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, src)
    batch = _batch(omega, fidx)
    out = torch.empty_like(src)
    work, n = _work(grid, batch.B, precision, OP_CONVOLVE, src.device)
    _check(load().green_convolve(ctypes.byref(grid), ctypes.byref(batch), _ptr(Ghat), _ptr(src), _ptr(out),
                                 precision, _ptr(work), n, _stream(src.device)), "green_convolve")
    return out


def ls_apply(grid: Grid, ref: Medium, m, omega, fidx, Ghat, u, out=None, work=None):
    """A u (Eq. 10) for every problem."""
    precision = _precision(u)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), u=u, out=out)
    _table("Ghat", Ghat, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, u)
    model = _model(grid, ref, m, precision)
    batch = _batch(omega, fidx)
    out = torch.empty_like(u) if out is None else out
    if work is None:
        work, n = _work(grid, batch.B, precision, OP_APPLY, u.device)
    else:
        n = _caller_work(work, u.device)
    _check(load().ls_apply(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(u), _ptr(out), precision,
                           _ptr(work), n, _stream(u.device)), "ls_apply")
    return out


def ls_apply_noalloc(grid: Grid, ref: Medium, m, omega, fidx, Ghat, u, out=None):
    """A u like ls_apply, with the library's fixed scratch array instead of a work buffer."""
    precision = _precision(u)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), u=u, out=out)
    _table("Ghat", Ghat, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, u)
    model = _model(grid, ref, m, precision)
    batch = _batch(omega, fidx)
    out = torch.empty_like(u) if out is None else out
    _check(load().ls_apply_noalloc(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(u), _ptr(out),
                                   precision, _stream(u.device)), "ls_apply_noalloc")
    return out


def noalloc_scratch_bytes() -> int:
    return int(load().dbi_noalloc_scratch_bytes())


def ls_solve(grid: Grid, ref: Medium, m, omega, fidx, Ghat, rhs, u0=None, tol=1e-6, max_iter=1000,
             check_every=8, work=None, out=None):
    """Solve A u = rhs for every problem (from u0, or from zero); returns (u, iters, relres, code)."""
    precision = _precision(rhs)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), rhs=rhs, u0=u0, out=out)
    _table("Ghat", Ghat, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, rhs)
    model = _model(grid, ref, m, precision)
    batch = _batch(omega, fidx)
    if out is None:
        u = torch.empty_like(rhs) if u0 is None else u0.clone()
    else:
        u = out
        if u0 is not None:
            u.copy_(u0)
    if work is None:
        work, n = _work(grid, batch.B, precision, OP_SOLVE, rhs.device)
    else:
        n = _caller_work(work, rhs.device)
    (iters, relres, code), st = _status(batch.B, rhs.device)
    opts = _kopts(tol, max_iter, check_every, zero_guess=u0 is None)
    _check(load().ls_solve(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(rhs), _ptr(u),
                           ctypes.byref(opts), ctypes.byref(st), precision, _ptr(work), n,
                           _stream(rhs.device)), "ls_solve")
    return u, iters, relres, code


def gmres_workspace_bytes(grid: Grid, B: int, precision: int, restart: int) -> int:
    return int(load().dbi_gmres_workspace_bytes(ctypes.byref(grid), B, precision, restart))


def ls_solve_gmres(grid: Grid, ref: Medium, m, omega, fidx, Ghat, rhs, u0=None, restart=30, tol=1e-6,
                   max_iter=1000, check_every=8):
    """Solve A u = rhs by restarted GMRES(restart); returns (u, iters, relres, code), iters in Arnoldi
    steps (operator passes inside the cycles)."""
    precision = _precision(rhs)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), rhs=rhs, u0=u0)
    _table("Ghat", Ghat, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, rhs)
    model = _model(grid, ref, m, precision)
    batch = _batch(omega, fidx)
    u = torch.empty_like(rhs) if u0 is None else u0.clone()
    n = gmres_workspace_bytes(grid, batch.B, precision, restart)
    if n == 0 and batch.B > 0:
        raise DBIError(f"invalid GMRES workspace query (restart {restart})")
    work = torch.empty(max(n, 1), dtype=torch.uint8, device=rhs.device)
    (iters, relres, code), st = _status(batch.B, rhs.device)
    opts = _kopts(tol, max_iter, check_every, zero_guess=u0 is None)
    _check(load().ls_solve_gmres(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(rhs), _ptr(u),
                                 ctypes.byref(opts), int(restart), ctypes.byref(st), precision, _ptr(work), n,
                                 _stream(rhs.device)), "ls_solve_gmres")
    return u, iters, relres, code


# ---------------------------------------------------------------------------------------------
# 3D extension
# ---------------------------------------------------------------------------------------------
def make_grid3(nz, ny, nx, lz, ly, lx, h) -> Grid3:
    return Grid3(int(nz), int(ny), int(nx), int(lz), int(ly), int(lx), float(h))


def workspace_bytes_3d(grid: Grid3, B: int, precision: int, op: int, restart: int = 30) -> int:
    return int(load().dbi_workspace_bytes_3d(ctypes.byref(grid), int(B), int(precision), int(op), int(restart)))


def _work3(grid, B, precision, op, device, restart=30):
    n = workspace_bytes_3d(grid, B, precision, op, restart)
    if n == 0:
        raise DBIError("invalid 3D grid, precision or restart for the workspace query")
    return torch.empty(n, dtype=torch.uint8, device=device), n


def _model3(grid, ref, m, precision) -> Model3:
    if m.dtype != real_dtype(precision):
        raise DBIError(f"model must be {real_dtype(precision)} for this precision, got {m.dtype}")
    _need_cuda(m)
    if tuple(m.shape) != (6, grid.nz, grid.ny, grid.nx):
        raise DBIError(f"model shape {tuple(m.shape)} != (6, {grid.nz}, {grid.ny}, {grid.nx})")
    return Model3(grid, ref, m.data_ptr())


def greens_tabulate_3d(grid: Grid3, ref: Medium, omega: torch.Tensor, precision: int = C64, with_space=True):
    """Ghat [nf][6][lz][ly][lx] (h^3 / (lz ly lx) FFT(G)) and, if asked, Gspace of the same shape."""
    _need_cuda(omega)
    dev = omega.device
    nf = int(omega.numel())
    cd = complex_dtype(precision)
    Ghat = torch.empty((nf, 6, grid.lz, grid.ly, grid.lx), dtype=cd, device=dev)
    Gspace = torch.empty_like(Ghat) if with_space else None
    work, n = _work3(grid, nf, precision, OP_GREENS, dev)
    _check(load().greens_tabulate_3d(ctypes.byref(grid), ctypes.byref(ref), _ptr(omega), nf, precision, _ptr(Ghat),
                                     _ptr(Gspace), _ptr(work), n, _stream(dev)), "greens_tabulate_3d")
    return Ghat, Gspace


def incident_field_3d(grid: Grid3, omega, fidx, Gspace, src_cells, forces):
    precision = _precision(Gspace)
    _table("Gspace", Gspace, int(omega.numel()), 6, grid.lz * grid.ly * grid.lx, complex_dtype(precision))
    _need_cuda(Gspace, src_cells, forces)
    batch = _batch(omega, fidx)
    u0 = torch.empty((batch.B, 3, grid.nz, grid.ny, grid.nx), dtype=Gspace.dtype, device=Gspace.device)
    _check(load().incident_field_3d(ctypes.byref(grid), ctypes.byref(batch), _ptr(Gspace), _ptr(src_cells),
                                    _ptr(forces), _ptr(u0), precision, _stream(Gspace.device)), "incident_field_3d")
    return u0


def ls_apply_3d(grid: Grid3, ref: Medium, m, omega, fidx, Ghat, u, out=None):
    precision = _precision(u)
    on_device = _fields(fidx, 3, grid.nz * grid.ny * grid.nx, complex_dtype(precision), u=u, out=out)
    _table("Ghat", Ghat, int(omega.numel()), 6, grid.lz * grid.ly * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, u)
    model = _model3(grid, ref, m, precision)
    batch = _batch(omega, fidx)
    out = torch.empty_like(u) if out is None else out
    work, n = _work3(grid, batch.B, precision, OP_APPLY, u.device)
    _check(load().ls_apply_3d(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(u), _ptr(out), precision,
                              _ptr(work), n, _stream(u.device)), "ls_apply_3d")
    return out


def ls_solve_3d(grid: Grid3, ref: Medium, m, omega, fidx, Ghat, rhs, u0=None, restart=30, tol=1e-6, max_iter=1000,
                check_every=8):
    """A u = rhs in 3D by GMRES(restart); returns (u, iters, relres, code)."""
    precision = _precision(rhs)
    on_device = _fields(fidx, 3, grid.nz * grid.ny * grid.nx, complex_dtype(precision), rhs=rhs, u0=u0)
    _table("Ghat", Ghat, int(omega.numel()), 6, grid.lz * grid.ly * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, rhs)
    model = _model3(grid, ref, m, precision)
    batch = _batch(omega, fidx)
    u = torch.empty_like(rhs) if u0 is None else u0.clone()
    work, n = _work3(grid, batch.B, precision, OP_SOLVE, rhs.device, restart)
    (iters, relres, code), st = _status(batch.B, rhs.device)
    opts = _kopts(tol, max_iter, check_every, zero_guess=u0 is None)
    _check(load().ls_solve_3d(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(rhs), _ptr(u),
                              ctypes.byref(opts), int(restart), ctypes.byref(st), precision, _ptr(work), n,
                              _stream(rhs.device)), "ls_solve_3d")
    return u, iters, relres, code


def _products3(name, grid, ref, m_b, omega, fidx, Ghat, u_b, rec_cells, x, out, tol, max_iter, restart,
               check_every):
    precision = _precision(u_b)
    on_device = _fields(fidx, 3, grid.nz * grid.ny * grid.nx, complex_dtype(precision), u_b=u_b)
    _table("Ghat", Ghat, int(omega.numel()), 6, grid.lz * grid.ly * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, u_b, rec_cells, x)
    if rec_cells.dtype != torch.int32 or rec_cells.dim() != 2 or rec_cells.shape[1] != 3:
        raise DBIError("rec_cells must be int32 [n_rec][3]")
    model = _model3(grid, ref, m_b, precision)
    batch = _batch(omega, fidx)
    n = int(load().dbi_products_workspace_bytes_3d(ctypes.byref(grid), batch.B, precision, int(restart)))
    if n == 0:
        raise DBIError("invalid 3D grid, precision or restart for the workspace query")
    work = torch.empty(n, dtype=torch.uint8, device=u_b.device)
    (iters, relres, code), st = _status(batch.B, u_b.device)
    opts = _kopts(tol, max_iter, check_every, zero_guess=True)
    _check(getattr(load(), name)(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(u_b), _ptr(rec_cells),
                                 int(rec_cells.shape[0]), _ptr(x), _ptr(out), ctypes.byref(opts), int(restart),
                                 ctypes.byref(st), precision, _ptr(work), n, _stream(u_b.device)), name)
    return out, (iters, relres, code)


def frechet_apply_3d(grid: Grid3, ref: Medium, m_b, omega, fidx, Ghat, u_b, rec_cells, dm, tol=1e-6,
                     max_iter=1000, restart=30, check_every=8):
    """J dm in 3D: [B][n_rec][3] complex data perturbations (and the solves' status)."""
    _real("dm", dm, 6 * grid.nz * grid.ny * grid.nx, real_dtype(_precision(u_b)))
    d = torch.empty((u_b.shape[0], rec_cells.shape[0], 3), dtype=u_b.dtype, device=u_b.device)
    return _products3("frechet_apply_3d", grid, ref, m_b, omega, fidx, Ghat, u_b, rec_cells, dm, d, tol, max_iter,
                      restart, check_every)


def adjoint_apply_3d(grid: Grid3, ref: Medium, m_b, omega, fidx, Ghat, u_b, rec_cells, r, tol=1e-6,
                     max_iter=1000, restart=30, check_every=8):
    """Re J^H r in 3D summed over the problems: [6][nz][ny][nx] real (and the solves' status)."""
    precision = _precision(u_b)
    on_device = _fields(fidx, int(rec_cells.shape[0]), 3, complex_dtype(precision), r=r)
    g = torch.empty((6, grid.nz, grid.ny, grid.nx), dtype=real_dtype(_precision(u_b)), device=u_b.device)
    return _products3("adjoint_apply_3d", grid, ref, m_b, omega, fidx, Ghat, u_b, rec_cells, r, g, tol, max_iter,
                      restart, check_every)


def sample_3d(grid: Grid3, rec_cells, u):
    """P u: [B][n_rec][3] complex."""
    precision = _precision(u)
    _need_cuda(rec_cells, u)
    d = torch.empty((u.shape[0], rec_cells.shape[0], 3), dtype=u.dtype, device=u.device)
    _check(load().sample_3d(ctypes.byref(grid), int(u.shape[0]), _ptr(rec_cells), int(rec_cells.shape[0]), _ptr(u),
                            _ptr(d), precision, _stream(u.device)), "sample_3d")
    return d


def normal_cg_3d(grid: Grid3, ref: Medium, m_b, omega, fidx, Ghat, u_b, rec_cells, dd, iters=30, lam=None,
                 lambda_rel=1e-3, power_iters=10, power_start=None, tol=1e-6, max_iter=1000, restart=30,
                 check_every=8):
    """Tikhonov normal-equation CG in 3D; returns (dm [6][nz][ny][nx], lambda, residual history)."""
    precision = _precision(u_b)
    on_device = _fields(fidx, 3, grid.nz * grid.ny * grid.nx, complex_dtype(precision), u_b=u_b)
    on_device += _fields(fidx, int(rec_cells.shape[0]), 3, complex_dtype(precision), dd=dd)
    _table("Ghat", Ghat, int(omega.numel()), 6, grid.lz * grid.ly * grid.lx, complex_dtype(precision))
    if power_start is not None:
        _real("power_start", power_start, 6 * grid.nz * grid.ny * grid.nx, real_dtype(precision))
    _need_cuda(*on_device, Ghat, u_b, dd, rec_cells, *([] if power_start is None else [power_start]))
    model = _model3(grid, ref, m_b, precision)
    batch = _batch(omega, fidx)
    n_rec = int(rec_cells.shape[0])
    n = int(load().dbi_normal_cg_workspace_bytes_3d(ctypes.byref(grid), batch.B, precision, int(restart), n_rec,
                                                    int(iters)))
    if n == 0:
        raise DBIError("invalid arguments for the 3D normal-equation workspace query")
    work = torch.empty(n, dtype=torch.uint8, device=u_b.device)
    dm = torch.empty((6, grid.nz, grid.ny, grid.nx), dtype=real_dtype(precision), device=u_b.device)
    (its, relres, code), st = _status(batch.B, u_b.device)
    opts = _kopts(tol, max_iter, check_every, zero_guess=True)
    cg = CGOpts(int(iters), float(lam) if lam is not None else 0.0, float(lambda_rel), int(power_iters))
    lam_out = c_double(0.0)
    hist = (c_double * (int(iters) + 1))()
    _check(load().normal_cg_3d(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(u_b), _ptr(rec_cells),
                               n_rec, _ptr(dd), ctypes.byref(cg), _ptr(power_start), _ptr(dm), ctypes.byref(lam_out),
                               hist, ctypes.byref(opts), int(restart), ctypes.byref(st), precision, _ptr(work), n,
                               _stream(u_b.device)), "normal_cg_3d")
    return dm, float(lam_out.value), list(hist)


def greens_tabulate_k(grid: Grid, ref: Medium, omega: torch.Tensor, precision: int = C64):
    """Dhat [nf][6][lx][lz]: h^2/(lz lx) FFT of the central differences of G_h combined per stress
    component (D1G11, D1G13, D3G11 + D1G13, D3G13 + D1G33, D3G13, D3G33), column-major (Eq. 9)."""
    _need_cuda(omega)
    dev = omega.device
    nf = int(omega.numel())
    Dhat = torch.empty((nf, 6, grid.lx, grid.lz), dtype=complex_dtype(precision), device=dev)
    work, n = _work(grid, nf, precision, OP_GREENS_K, dev)
    _check(load().greens_tabulate_k(ctypes.byref(grid), ctypes.byref(ref), _ptr(omega), nf, precision,
                                    _ptr(Dhat), _ptr(work), n, _stream(dev)), "greens_tabulate_k")
    return Dhat


def ls_apply_k(grid: Grid, ref: Medium, m, omega, fidx, Ghat, Dhat, u, out=None):
    """A u in the paper-literal form of Eq. 9 (the gradient on the Green's tensor)."""
    precision = _precision(u)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), u=u, out=out)
    _table("Ghat", Ghat, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    _table("Dhat", Dhat, int(omega.numel()), 6, grid.lz * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, Dhat, u)
    model = _model(grid, ref, m, precision)
    batch = _batch(omega, fidx)
    out = torch.empty_like(u) if out is None else out
    work, n = _work(grid, batch.B, precision, OP_APPLY_K, u.device)
    _check(load().ls_apply_k(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(Dhat), _ptr(u),
                             _ptr(out), precision, _ptr(work), n, _stream(u.device)), "ls_apply_k")
    return out


def ls_solve_k(grid: Grid, ref: Medium, m, omega, fidx, Ghat, Dhat, rhs, u0=None, tol=1e-6, max_iter=1000,
               check_every=8):
    """Solve A u = rhs with the operator of ls_apply_k; returns (u, iters, relres, code)."""
    precision = _precision(rhs)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), rhs=rhs, u0=u0)
    _table("Ghat", Ghat, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    _table("Dhat", Dhat, int(omega.numel()), 6, grid.lz * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, Dhat, rhs)
    model = _model(grid, ref, m, precision)
    batch = _batch(omega, fidx)
    u = torch.empty_like(rhs) if u0 is None else u0.clone()
    work, n = _work(grid, batch.B, precision, OP_SOLVE_K, rhs.device)
    (iters, relres, code), st = _status(batch.B, rhs.device)
    opts = _kopts(tol, max_iter, check_every, zero_guess=u0 is None)
    _check(load().ls_solve_k(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(Dhat), _ptr(rhs),
                             _ptr(u), ctypes.byref(opts), ctypes.byref(st), precision, _ptr(work), n,
                             _stream(rhs.device)), "ls_solve_k")
    return u, iters, relres, code


def frechet_apply(grid: Grid, ref: Medium, m_b, omega, fidx, Ghat, u_b, rec_cells, dm, tol=1e-6,
                  max_iter=1000, check_every=8, with_status=False):
    """J dm sampled at the receivers, [B][n_rec][2] (and the solve's (iters, relres, code))."""
    precision = _precision(u_b)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), u_b=u_b)
    _table("Ghat", Ghat, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    _real("dm", dm, 5 * grid.nz * grid.nx, real_dtype(precision))
    _need_cuda(*on_device, Ghat, u_b, dm)
    model = _model(grid, ref, m_b, precision)
    if dm.dtype != real_dtype(precision):
        raise DBIError("dm must have the model's real dtype")
    batch = _batch(omega, fidx)
    rec = _receivers(rec_cells)
    d = torch.empty((batch.B, rec.n, 2), dtype=u_b.dtype, device=u_b.device)
    work, n = _work(grid, batch.B, precision, OP_FRECHET, u_b.device)
    (iters, relres, code), st = _status(batch.B, u_b.device)
    opts = _kopts(tol, max_iter, check_every)
    _check(load().frechet_apply(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(u_b),
                                ctypes.byref(rec), _ptr(dm), _ptr(d), ctypes.byref(opts), ctypes.byref(st),
                                precision, _ptr(work), n, _stream(u_b.device)), "frechet_apply")
    return (d, (iters, relres, code)) if with_status else d


def adjoint_apply(grid: Grid, ref: Medium, m_b, omega, fidx, Ghat, u_b, rec_cells, r, tol=1e-6,
                  max_iter=1000, check_every=8, with_status=False):
    """Re J^H r summed over problems, [5][nz][nx] (and the solve's (iters, relres, code))."""
    precision = _precision(u_b)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), u_b=u_b)
    on_device += _fields(fidx, int(rec_cells.shape[0]), 2, complex_dtype(precision), r=r)
    _table("Ghat", Ghat, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    _need_cuda(*on_device, Ghat, u_b, r)
    model = _model(grid, ref, m_b, precision)
    batch = _batch(omega, fidx)
    rec = _receivers(rec_cells)
    g = torch.empty((5, grid.nz, grid.nx), dtype=real_dtype(precision), device=u_b.device)
    work, n = _work(grid, batch.B, precision, OP_ADJOINT, u_b.device)
    (iters, relres, code), st = _status(batch.B, u_b.device)
    opts = _kopts(tol, max_iter, check_every)
    _check(load().adjoint_apply(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(u_b),
                                ctypes.byref(rec), _ptr(r), _ptr(g), ctypes.byref(opts), ctypes.byref(st),
                                precision, _ptr(work), n, _stream(u_b.device)), "adjoint_apply")
    return (g, (iters, relres, code)) if with_status else g


def data_residual(grid: Grid, omega, fidx, rec_cells, u, d_obs):
    """(r = P u - d_obs, phi = 1/2 ||r||^2 as a device float64 scalar tensor)."""
    precision = _precision(u)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), u=u)
    on_device += _fields(fidx, int(rec_cells.shape[0]), 2, complex_dtype(precision), d_obs=d_obs)
    _need_cuda(*on_device, u, d_obs)
    batch = _batch(omega, fidx)
    rec = _receivers(rec_cells)
    r = torch.empty_like(d_obs)
    phi = torch.empty((), dtype=torch.float64, device=u.device)
    _check(load().data_residual(ctypes.byref(grid), ctypes.byref(batch), ctypes.byref(rec), _ptr(u),
                                _ptr(d_obs), _ptr(r), _ptr(phi), precision, _stream(u.device)), "data_residual")
    return r, phi


def normal_cg(grid: Grid, ref: Medium, m_b, omega, fidx, Ghat, u_b, rec_cells, dd, iters=30, lam=None,
              lambda_rel=1e-3, power_iters=10, power_start=None, tol=1e-6, max_iter=1000, check_every=8):
    """Tikhonov normal-equation CG; returns (dm [5][nz][nx], lambda, residual history)."""
    precision = _precision(u_b)
    on_device = _fields(fidx, 2, grid.nz * grid.nx, complex_dtype(precision), u_b=u_b)
    on_device += _fields(fidx, int(rec_cells.shape[0]), 2, complex_dtype(precision), dd=dd)
    _table("Ghat", Ghat, int(omega.numel()), 3, grid.lz * grid.lx, complex_dtype(precision))
    if power_start is not None:
        _real("power_start", power_start, 5 * grid.nz * grid.nx, real_dtype(precision))
    _need_cuda(*on_device, Ghat, u_b, dd, power_start)
    model = _model(grid, ref, m_b, precision)
    batch = _batch(omega, fidx)
    rec = _receivers(rec_cells)
    dm = torch.empty((5, grid.nz, grid.nx), dtype=real_dtype(precision), device=u_b.device)
    work, n = _work(grid, batch.B, precision, OP_NORMAL_CG, u_b.device)
    (its, relres, code), st = _status(batch.B, u_b.device)
    opts = _kopts(tol, max_iter, check_every)
    cg = CGOpts(int(iters), float(lam) if lam is not None else 0.0, float(lambda_rel), int(power_iters))
    lam_out = c_double(0.0)
    hist = (c_double * (int(iters) + 1))()
    _check(load().normal_cg(ctypes.byref(model), ctypes.byref(batch), _ptr(Ghat), _ptr(u_b), ctypes.byref(rec),
                            _ptr(dd), ctypes.byref(cg), _ptr(power_start), _ptr(dm), ctypes.byref(lam_out),
                            hist, ctypes.byref(opts), ctypes.byref(st), precision, _ptr(work), n,
                            _stream(u_b.device)), "normal_cg")
    return dm, float(lam_out.value), list(hist)
