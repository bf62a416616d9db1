"""The C-ABI library builds, loads and exports every entry point that include/dbi.h declares; its
host-side argument checks reject bad calls before any CUDA work. No GPU is needed."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2402_02116_gb300 import build, dbi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^(?:const\s+char\s*\*|unsigned\s+long\s+long|long\s+long|int|size_t|void)"
                                r"\s*\**\s*(\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dbi.load()


def test_header_declares_the_paper_entry_points():
    names = declared_functions()
    for want in ("greens_tabulate", "ls_apply", "ls_solve", "frechet_apply", "adjoint_apply", "normal_cg",
                 "incident_field", "green_convolve", "data_residual", "dbi_workspace_bytes", "dbi_last_error",
                 "dbi_kernel_launches", "ls_apply_group", "ls_solve_group", "dbi_group_create", "dbi_group_tune",
                 "dbi_group_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in dbi.SIGNATURES, name


def test_workspace_query_is_host_only(lib):
    g = dbi.make_grid(32, 32, 64, 64, 10.0)
    assert dbi.workspace_bytes(g, 4, dbi.C64, dbi.OP_APPLY) > 4 * 2 * 32 * 64 * 8
    assert dbi.workspace_bytes(g, 4, dbi.C128, dbi.OP_SOLVE) > dbi.workspace_bytes(g, 4, dbi.C64, dbi.OP_SOLVE)
    bad = dbi.make_grid(32, 32, 48, 64, 10.0)  # 48 is not a supported FFT length
    assert dbi.workspace_bytes(bad, 4, dbi.C64, dbi.OP_APPLY) == 0
    small = dbi.make_grid(40, 32, 64, 64, 10.0)  # 64 < 2 * 40 - 1
    assert dbi.workspace_bytes(small, 4, dbi.C64, dbi.OP_APPLY) == 0
    g768 = dbi.make_grid(384, 300, 768, 768, 5.0)  # 3 x 256: a complex64 length only
    spectra, sources = 4 * 2 * 768 * 384 * 8, 4 * 2 * 384 * 300 * 8
    assert dbi.workspace_bytes(g768, 4, dbi.C64, dbi.OP_APPLY) >= spectra + sources
    assert dbi.workspace_bytes(g768, 4, dbi.C128, dbi.OP_APPLY) == 0
    assert dbi.workspace_bytes(dbi.make_grid(384, 300, 768, 512, 5.0), 4, dbi.C64, dbi.OP_APPLY) == 0  # 512 < 599


def test_argument_errors_are_reported_without_a_gpu(lib):
    ref = dbi.make_medium(2000.0, 2000.0, 1155.0)
    rc = lib.greens_tabulate(None, ctypes.byref(ref), None, 1, 0, None, None, None, 0, None)
    assert rc == -1 and b"NULL" in lib.dbi_last_error()
    g = dbi.make_grid(32, 32, 48, 64, 10.0)
    rc = lib.greens_tabulate(ctypes.byref(g), ctypes.byref(ref), None, 1, 0, None, None, None, 0, None)
    assert rc == -2 and b"power of two" in lib.dbi_last_error()
    g = dbi.make_grid(32, 32, 64, 64, 10.0)
    rc = lib.greens_tabulate(ctypes.byref(g), ctypes.byref(ref), None, 1, 7, None, None, None, 0, None)
    assert rc == -2
    bad_ref = dbi.make_medium(2000.0, 1000.0, 1155.0)  # alpha0 < beta0
    rc = lib.greens_tabulate(ctypes.byref(g), ctypes.byref(bad_ref), None, 1, 0, None, None, None, 0, None)
    assert rc == -1
    unstable = dbi.make_medium_vti(2200.0, 1.0e10, 2.0e10, 1.0e10, 3.0e9)  # C11 C33 < C13^2
    rc = lib.greens_tabulate(ctypes.byref(g), ctypes.byref(unstable), None, 1, 0, None, None, None, 0, None)
    assert rc == -1 and b"VTI" in lib.dbi_last_error()
    vti = dbi.make_medium_vti(2200.0, 1.65e10, 5.6e9, 1.375e10, 4.58e9)
    rc = lib.greens_tabulate_k(ctypes.byref(g), ctypes.byref(vti), None, 1, 0, None, None, 0, None)
    assert rc == -1 and b"isotropic" in lib.dbi_last_error()
    g768 = dbi.make_grid(300, 300, 768, 768, 5.0)  # the paper-literal form K has no length-768 stages
    rc = lib.greens_tabulate_k(ctypes.byref(g768), ctypes.byref(ref), None, 1, 0, None, None, 0, None)
    assert rc == -2 and b"power of two" in lib.dbi_last_error()
    rc = lib.greens_tabulate(ctypes.byref(g768), ctypes.byref(ref), None, 1, 1, None, None, None, 0, None)
    assert rc == -2 and b"768 with complex64" in lib.dbi_last_error()  # complex128
    rc = lib.greens_tabulate(ctypes.byref(g768), ctypes.byref(ref), None, 1, 0, None, None, None, 0, None)
    assert rc == -1 and b"need nf" in lib.dbi_last_error()  # complex64: the grid passes
    rc = lib.dbi_gmres_workspace_bytes(ctypes.byref(g), 4, 0, 65)
    assert rc == 0
    model = dbi.Model(g, ref, None)
    batch = dbi.Batch(2, 1, None, None)
    rc = lib.ls_apply(ctypes.byref(model), ctypes.byref(batch), None, None, None, 0, None, 0, None)
    assert rc == -1
    opts = dbi.KrylovOpts(-1.0, 10, 1)
    batch = dbi.Batch(0, 1, 1, None)
    rc = lib.ls_solve(ctypes.byref(model), ctypes.byref(batch), None, None, None, ctypes.byref(opts), None, 0,
                      None, 0, None)
    assert rc == -1 and b"tol" in lib.dbi_last_error()
    assert lib.dbi_version() >= 100


def test_3d_argument_errors_are_reported_without_a_gpu(lib):
    g = dbi.make_grid3(4, 3, 5, 16, 16, 16, 10.0)
    assert dbi.workspace_bytes_3d(g, 2, dbi.C64, dbi.OP_APPLY) > 0
    assert dbi.workspace_bytes_3d(g, 2, dbi.C64, dbi.OP_SOLVE, restart=65) == 0
    small = dbi.make_grid3(9, 3, 5, 16, 16, 16, 10.0)  # lz = 16 < 2 * 9 - 1
    assert dbi.workspace_bytes_3d(small, 2, dbi.C64, dbi.OP_APPLY) == 0
    odd = dbi.make_grid3(4, 3, 5, 16, 24, 16, 10.0)  # 24 is not a supported FFT length
    assert dbi.workspace_bytes_3d(odd, 2, dbi.C64, dbi.OP_APPLY) == 0
    vti = dbi.make_medium_vti(2200.0, 1.65e10, 5.6e9, 1.375e10, 4.58e9)
    rc = lib.greens_tabulate_3d(ctypes.byref(g), ctypes.byref(vti), None, 1, 0, None, None, None, 0, None)
    assert rc == -1 and b"isotropic" in lib.dbi_last_error()
    ref = dbi.make_medium(2000.0, 2000.0, 1155.0)
    model = dbi.Model3(g, ref, None)
    batch = dbi.Batch(2, 1, 1, 1)  # non-NULL placeholders: validation fails before any device access
    rc = lib.ls_apply_3d(ctypes.byref(model), ctypes.byref(batch), None, None, None, 0, None, 0, None)
    assert rc == -1 and b"NULL" in lib.dbi_last_error()
    opts = dbi.KrylovOpts(1e-6, 10, 1, 1)
    rc = lib.ls_solve_3d(ctypes.byref(model), ctypes.byref(batch), None, None, None, ctypes.byref(opts), 0, None, 0,
                         None, 0, None)
    assert rc == -1 and b"restart" in lib.dbi_last_error()
    big = dbi.Batch(30000, 1, 1, 1)  # B * 3 * nz exceeds the launch limit of the y pass
    rc = lib.ls_apply_3d(ctypes.byref(model), ctypes.byref(big), None, None, None, 0, None, 0, None)
    assert rc == -2 and b"too large" in lib.dbi_last_error()
    cg = dbi.CGOpts(5, 0.0, 0.0, 0)  # neither lambda nor an estimate
    rc = lib.normal_cg_3d(ctypes.byref(model), ctypes.byref(batch), None, None, None, 1, None, ctypes.byref(cg), None,
                          None, None, None, ctypes.byref(opts), 30, None, 0, None, 0, None)
    assert rc == -1 and b"CG options" in lib.dbi_last_error()
    assert lib.sample_3d(ctypes.byref(g), -1, None, 1, None, None, 0, None) == -1


def test_empty_batches_are_no_ops_without_a_gpu(lib):
    """B = 0 returns 0 after validating the arguments and before any device work, in every entry
    point that takes a batch of wavefields (the problem arrays may then be NULL; omega is a
    placeholder that is never read)."""
    ref = dbi.make_medium(2000.0, 2000.0, 1155.0)
    g = dbi.make_grid(8, 8, 16, 16, 10.0)
    model = dbi.Model(g, ref, None)
    empty = dbi.Batch(0, 1, 1, None)
    opts = dbi.KrylovOpts(1e-6, 10, 1, 1)
    by = ctypes.byref
    assert lib.green_convolve(by(g), by(empty), None, None, None, 0, None, 0, None) == 0
    assert lib.incident_field(by(g), by(empty), None, None, None, None, 0, None) == 0
    assert lib.ls_apply(by(model), by(empty), None, None, None, 0, None, 0, None) == 0
    assert lib.ls_apply_noalloc(by(model), by(empty), None, None, None, 0, None) == 0
    assert lib.ls_solve(by(model), by(empty), None, None, None, by(opts), None, 0, None, 0, None) == 0
    assert lib.ls_solve_gmres(by(model), by(empty), None, None, None, by(opts), 30, None, 0, None, 0, None) == 0
    assert lib.ls_apply_k(by(model), by(empty), None, None, None, None, 0, None, 0, None) == 0
    assert lib.ls_solve_k(by(model), by(empty), None, None, None, None, by(opts), None, 0, None, 0, None) == 0
    g3 = dbi.make_grid3(4, 3, 5, 16, 16, 16, 10.0)
    model3 = dbi.Model3(g3, ref, None)
    assert lib.incident_field_3d(by(g3), by(empty), None, None, None, None, 0, None) == 0
    assert lib.ls_apply_3d(by(model3), by(empty), None, None, None, 0, None, 0, None) == 0
    assert lib.ls_solve_3d(by(model3), by(empty), None, None, None, by(opts), 30, None, 0, None, 0, None) == 0
    assert lib.sample_3d(by(g3), 0, None, 1, None, None, 0, None) == 0
    # the checks before the early return still apply to an empty batch
    bad_opts = dbi.KrylovOpts(-1.0, 10, 1, 1)
    assert lib.ls_solve(by(model), by(empty), None, None, None, by(bad_opts), None, 0, None, 0, None) == -1
    assert lib.ls_solve_3d(by(model3), by(empty), None, None, None, by(opts), 0, None, 0, None, 0, None) == -1


def test_the_abi_from_plain_c(lib, tmp_path):
    """`tests/native/abi_from_c.c` includes both headers as C11 (-pedantic, warnings as errors),
    links the library and calls its host-side entry points: version, workspace queries (2D, 3D,
    both precisions, an unsupported FFT length) and an argument error with its message."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(build.LIB)
    exe = str(tmp_path / "abi_from_c")
    res = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                          os.path.join(ROOT, "tests", "native", "abi_from_c.c"), "-L", libdir, "-ldbi",
                          f"-Wl,-rpath,{libdir}", "-o", exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stdout + run.stderr
    assert run.stdout.count("ok ") == 7


def test_the_product_path_fails_loudly_without_the_library_or_a_gpu():
    """No CPU fallback: loading a missing library raises with the build instruction, and on a
    machine without a GPU a device problem cannot be made (fresh interpreters, since the library
    handle is cached per process)."""
    import subprocess
    import sys
    import torch
    code = "from paper_2402_02116_gb300 import dbi; dbi.load('/nonexistent/libdbi.so')"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "CUDA library not built" in r.stderr
    if not torch.cuda.is_available():
        code = ("from paper_2402_02116_gb300 import dbi, inputs\n"
                "from paper_2402_02116_gb300.problem import DeviceProblem\n"
                "DeviceProblem(inputs.small_case(nz=4, nx=4), dbi.C64)\n"
                "print('no error')")
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
        assert r.returncode != 0 and "no error" not in r.stdout


def test_workspace_queries_grow_with_the_batch_and_never_wrap(lib):
    """Every workspace query, for seeded random grids and batches and the one-cell grid: the size grows
    with B, complex128 needs at least what complex64 does, and a batch far beyond any GPU (2^20
    problems) gives a size above the bytes of its own complex64 wavefields (no 32-bit products
    that would wrap)."""
    import numpy as np
    rng = np.random.default_rng(31)
    ops2d = [dbi.OP_CONVOLVE, dbi.OP_APPLY, dbi.OP_SOLVE, dbi.OP_FRECHET, dbi.OP_ADJOINT, dbi.OP_NORMAL_CG,
             dbi.OP_APPLY_K, dbi.OP_SOLVE_K]
    shapes = [(1, 1)] + [(int(rng.integers(1, 513)), int(rng.integers(1, 513))) for _ in range(60)]
    for nz, nx in shapes:
        g = dbi.make_grid(nz, nx, max(16, 1 << (2 * nz - 2).bit_length()), max(16, 1 << (2 * nx - 2).bit_length()), 5.0)
        B = int(rng.integers(1, 300))
        for op in ops2d:
            small = dbi.workspace_bytes(g, B, dbi.C64, op)
            assert small > 0 and dbi.workspace_bytes(g, B + 7, dbi.C64, op) >= small, (nz, nx, B, op)
            assert dbi.workspace_bytes(g, B, dbi.C128, op) >= small
            huge = dbi.workspace_bytes(g, 1 << 20, dbi.C64, op)
            # every 2D operation holds at least one complex64 field's worth per problem (its
            # spectral scratch has lx >= nx columns); Python's integers do not wrap
            assert huge >= (1 << 20) * 2 * nz * nx * 8 and huge >= small, (nz, nx, op, huge)
        gm = lib.dbi_gmres_workspace_bytes(ctypes.byref(g), B, dbi.C64, 30)
        assert gm >= 31 * B * 2 * nz * nx * 8 and lib.dbi_gmres_workspace_bytes(ctypes.byref(g), 1 << 20, dbi.C64, 30) > gm
    for _ in range(30):
        nz, ny, nx = (int(v) for v in rng.integers(1, 65, size=3))
        g3 = dbi.make_grid3(nz, ny, nx, *(max(16, 1 << (2 * n - 2).bit_length()) for n in (nz, ny, nx)), 25.0)
        B = int(rng.integers(1, 100))
        field = B * 3 * nz * ny * nx * 8
        for op, restart in ((dbi.OP_APPLY, 1), (dbi.OP_SOLVE, 30)):
            a = dbi.workspace_bytes_3d(g3, B, dbi.C64, op, restart)
            assert a > 0 and dbi.workspace_bytes_3d(g3, B + 3, dbi.C64, op, restart) >= a
            assert dbi.workspace_bytes_3d(g3, B, dbi.C128, op, restart) >= a
        assert dbi.workspace_bytes_3d(g3, B, dbi.C64, dbi.OP_SOLVE, 30) >= 31 * field
        p = lib.dbi_products_workspace_bytes_3d(ctypes.byref(g3), B, dbi.C64, 30)
        assert p >= 31 * field and lib.dbi_products_workspace_bytes_3d(ctypes.byref(g3), 1 << 20, dbi.C64, 30) > p


def test_work_buffer_arena_overflow_is_reported(tmp_path):
    """The library's work-buffer arena (the bump allocator every entry point carves its scratch
    from), compiled into a host program and linked against the library: carves are aligned and
    inside the buffer; a carve past the end, a missing buffer or a wrapping size returns NULL and
    sets a sticky overflow flag, which the entry points check before their first launch
    (DBI_ERR_WORKSPACE with the caller's name in dbi_last_error)."""
    cc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cc):
        pytest.skip("nvcc not available")
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "arena_host")
    res = subprocess.run([cc, "-std=c++20", "-O1", "--expt-relaxed-constexpr", "-gencode",
                          "arch=compute_103a,code=sm_103a", os.path.join(ROOT, "tests", "native", "arena_host.cu"),
                          "-o", exe, "-L", libdir, "-ldbi", "-Xlinker", "-rpath=" + libdir],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stderr
    assert "arena ok" in run.stdout


def test_bicgstab_decision_branches_on_the_host(tmp_path):
    """The library's BiCGSTAB end-of-iteration decision compiled for the CPU from its own header and
    run on crafted inner products: NaN or infinity stops a problem with DBI_NONFINITE before any
    other test, convergence (residual or half step), the iteration limit, both breakdowns (omega = 0,
    <rhat, r> negligible) restart from the iterate with rhat := r and report DBI_BREAKDOWN, and beta
    equals (rho_new / rho)(alpha / omega) in std::complex arithmetic."""
    cc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "krylov_decide_host")
    res = subprocess.run([cc, "-std=c++20", "-O1", "--expt-relaxed-constexpr", "-gencode",
                          "arch=compute_103a,code=sm_103a",
                          os.path.join(ROOT, "tests", "native", "krylov_decide_host.cu"), "-o", exe],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stderr
    assert "decide ok" in run.stdout
