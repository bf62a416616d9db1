"""ctypes binding of the C++17 FP64 oracle (oracle/cpp/dbi_oracle.cpp): the same discrete problem
as oracle/dbi_oracle.py, written apart from it (own radix-2 FFT, C++17 Bessel functions, OpenMP
over the problems of a batch).

TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline and
reference legs may load it. It shares no code with the CUDA library and imports nothing from it.
`build()` compiles it with the host's C++ compiler (g++ -std=c++17 -O2 -fopenmp).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from ctypes import POINTER, c_double, c_int, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpp", "dbi_oracle.cpp")
LIB = os.path.join(HERE, "cpp", "_build", "libdbi_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cxx = os.environ.get("CXX") or shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        raise RuntimeError("no C++ compiler found for the C++ oracle")
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    res = subprocess.run([cxx, "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp],
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"building the C++ oracle failed:\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_green_lattice.argtypes = [c_int, c_int, c_double, c_double, c_double, c_double, c_double, c_void_p]
        lib.orc_create.argtypes = [c_int, c_int, c_double, c_int, c_int, c_double, c_double, c_double, c_void_p,
                                   c_int, c_void_p, c_int]
        lib.orc_create.restype = c_void_p
        lib.orc_destroy.argtypes = [c_void_p]
        lib.orc_apply.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_int]
        lib.orc_gradient.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                     c_double, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        lib.orc_max_threads.restype = c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(load().orc_max_threads())


def _p(a):
    return a.ctypes.data_as(c_void_p) if a is not None else None


def green_lattice(nz, nx, h, omega, alpha, beta, rho) -> np.ndarray:
    """G_h on the (2nz-1) x (2nx-1) offsets, [3][dz + nz - 1][dx + nx - 1] (G11, G13, G33)."""
    out = np.zeros((3, 2 * nz - 1, 2 * nx - 1), dtype=np.complex128)
    rc = load().orc_green_lattice(nz, nx, h, omega, alpha, beta, rho, _p(out))
    if rc:
        raise ValueError("orc_green_lattice: bad grid")
    return out


class Oracle:
    """One grid, its model and the Green's tables of its frequencies (built once, in parallel)."""

    def __init__(self, nz, nx, h, lz, lx, rho0, alpha0, beta0, model, omegas, threads=0):
        self.nz, self.nx = int(nz), int(nx)
        self._model = np.ascontiguousarray(model, dtype=np.float64)
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        self.ctx = load().orc_create(self.nz, self.nx, float(h), int(lz), int(lx), float(rho0), float(alpha0),
                                     float(beta0), _p(self._model), len(om), _p(om), int(threads))
        if not self.ctx:
            raise ValueError("orc_create: bad grid (FFT lengths must be powers of two >= 2n - 1)")

    def __del__(self):
        if getattr(self, "ctx", None):
            load().orc_destroy(self.ctx)
            self.ctx = None

    def apply(self, fidx, u, direct=False, threads=0):
        """A u (Eq. 10) for every problem: u [B][2][nz][nx] complex; problem b at frequency fidx[b]."""
        fidx = np.ascontiguousarray(fidx, dtype=np.int32)
        u = np.ascontiguousarray(u, dtype=np.complex128)
        out = np.empty_like(u)
        load().orc_apply(self.ctx, len(fidx), _p(fidx), _p(u), _p(out), int(bool(direct)), int(threads))
        return out

    def gradient(self, fidx, src_cells, forces, rec_cells, d_obs, tol=1e-12, max_iter=3000, threads=0,
                 keep_fields=False):
        """Misfit gradient of a batch (Eq. 23, 25, 32-35), one problem per OpenMP thread. Returns
        (g [5][nz][nx], residuals [B][nrec][2], passes [B], relres [B][2], u or None)."""
        B = len(fidx)
        fidx = np.ascontiguousarray(fidx, dtype=np.int32)
        src = np.ascontiguousarray(src_cells, dtype=np.int32).reshape(B, 2)
        frc = np.ascontiguousarray(forces, dtype=np.float64).reshape(B, 2)
        rec = np.ascontiguousarray(rec_cells, dtype=np.int32)
        d_obs = np.ascontiguousarray(d_obs, dtype=np.complex128)
        g = np.zeros((5, self.nz, self.nx))
        r = np.zeros((B, len(rec), 2), dtype=np.complex128)
        passes = np.zeros(B, dtype=np.int32)
        relres = np.zeros((B, 2))
        u = np.zeros((B, 2, self.nz, self.nx), dtype=np.complex128) if keep_fields else None
        load().orc_gradient(self.ctx, B, _p(fidx), _p(src), _p(frc), len(rec), _p(rec), _p(d_obs), float(tol),
                            int(max_iter), int(threads), _p(g), _p(u), _p(r), _p(passes), _p(relres))
        return g, r, passes, relres, u


def for_workload(w, model=None, threads=0) -> Oracle:
    """The oracle of a seeded workload (grid, reference medium, model, frequencies)."""
    return Oracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.model if model is None else model,
                  w.omegas, threads)
