"""Uneven batches: many LS problems of different grid sizes run together (include/dbi_group.h).

`UnevenBatch` takes a list of `DeviceProblem`s (each with its own grid, model, Green's tables,
frequencies and sources) and builds one plan over all their wavefields ("slots"). Fields are flat
complex tensors holding every slot's [2][nz][nx] array in member order; `split` / `join` convert
between the flat form and per-member [B][2][nz][nx] views. Every call goes to the CUDA library
(argument marshalling only).
"""
from __future__ import annotations

import ctypes

import torch

from . import dbi


class UnevenBatch:
    def __init__(self, problems, precision: int = dbi.C64):
        if not problems:
            raise ValueError("need at least one problem")
        self.problems = list(problems)
        self.precision = precision
        self.device = self.problems[0].device
        self.cdt = dbi.complex_dtype(precision)
        n = len(self.problems)
        members = (dbi.GroupMember * n)()
        for k, P in enumerate(self.problems):
            if P.precision != precision:
                raise ValueError("every problem must use the batch's precision")
            members[k].model = dbi._model(P.grid, P.ref, P.m, precision)
            members[k].Ghat = P.Ghat.data_ptr()
            members[k].omega = P.omega.data_ptr()
            members[k].nf = int(P.omega.numel())
            members[k].B = P.B
            members[k].fidx = P.fidx.data_ptr()
        self._members = members
        h = ctypes.c_void_p()
        dbi._check(dbi.load().dbi_group_create(members, n, precision, ctypes.byref(h)), "dbi_group_create")
        self._h = h
        self.slots = int(dbi.load().dbi_group_slots(h))
        self.field_elems = int(dbi.load().dbi_group_field_elems(h))
        offs = (ctypes.c_longlong * (self.slots + 1))()
        dbi._check(dbi.load().dbi_group_offsets(h, offs), "dbi_group_offsets")
        self.offsets = list(offs)
        self._work = None
        self._bound = None

    def close(self):
        if getattr(self, "_h", None):
            dbi.load().dbi_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- fields ---------------------------------------------------------------------------------
    def empty_field(self):
        return torch.empty(self.field_elems, dtype=self.cdt, device=self.device)

    def member_range(self, k: int):
        s0 = sum(P.B for P in self.problems[:k])
        return self.offsets[s0], self.offsets[s0 + self.problems[k].B]

    def split(self, flat):
        out = []
        for k, P in enumerate(self.problems):
            a, b = self.member_range(k)
            out.append(flat[a:b].view(P.B, 2, P.grid.nz, P.grid.nx))
        return out

    def join(self, fields):
        return torch.cat([f.reshape(-1) for f in fields]).contiguous()

    def incident(self):
        return self.join([P.incident() for P in self.problems])

    # --- workspace ------------------------------------------------------------------------------
    def bind(self, op: int = dbi.OP_SOLVE):
        """Allocate the work buffer for `op` (OP_APPLY or OP_SOLVE) and attach it to the plan."""
        if self._bound is not None and (self._bound == op or self._bound == dbi.OP_SOLVE):
            return
        n = int(dbi.load().dbi_group_workspace_bytes(self._h, op))
        self._work = torch.empty(max(n, 1), dtype=torch.uint8, device=self.device)
        dbi._check(dbi.load().dbi_group_bind(self._h, dbi._ptr(self._work), n, op, dbi._stream(self.device)),
                   "dbi_group_bind")
        self._bound = op

    # --- entry points ---------------------------------------------------------------------------
    def _fields(self, **named):
        """Field arguments hold every slot's block (field_elems elements of the batch's dtype): the
        persistent kernels index them by the plan's offsets."""
        for name, t in named.items():
            if t is not None and (t.numel() != self.field_elems or t.dtype != self.cdt):
                raise dbi.DBIError(f"{name} holds {t.numel()} elements of {t.dtype}; the batch's fields hold "
                                   f"{self.field_elems} of {self.cdt}")
        dbi._need_cuda(*named.values())

    def apply(self, u, out=None):
        """A u for every slot (flat fields)."""
        self._fields(u=u, out=out)
        self.bind(dbi.OP_APPLY)
        out = torch.empty_like(u) if out is None else out
        dbi._check(dbi.load().ls_apply_group(self._h, dbi._ptr(u), dbi._ptr(out), dbi._stream(self.device)),
                   "ls_apply_group")
        return out

    def solve(self, rhs, tol=1e-6, max_iter=2000, check_every=8, graph=True, u0=None):
        """Solve A u = rhs for every slot; returns (u, iters, relres, code), status per slot."""
        self._fields(rhs=rhs, u0=u0)
        self.bind(dbi.OP_SOLVE)
        u = torch.empty_like(rhs) if u0 is None else u0.clone()
        (iters, relres, code), st = dbi._status(self.slots, self.device)
        opts = dbi._kopts(tol, max_iter, check_every, zero_guess=u0 is None)
        flags = dbi.GROUP_GRAPH if graph else 0
        dbi._check(dbi.load().ls_solve_group(self._h, dbi._ptr(rhs), dbi._ptr(u), ctypes.byref(opts),
                                             ctypes.byref(st), flags, dbi._stream(self.device)), "ls_solve_group")
        return u, iters, relres, code

    def tune(self, u):
        """Autotune radix plans and persistent grids on field u; returns the measurements."""
        self._fields(u=u)
        self.bind(dbi.OP_APPLY)
        out = torch.empty_like(u)
        rep = dbi.GroupTuning()
        dbi._check(dbi.load().dbi_group_tune(self._h, dbi._ptr(u), dbi._ptr(out), dbi._stream(self.device),
                                             ctypes.byref(rep)), "dbi_group_tune")
        lens = [(rep.lengths[i], rep.plan[i], (rep.plan_ms[i][0], rep.plan_ms[i][1]))
                for i in range(8) if rep.lengths[i]]
        return {"lengths": lens, "ctas_per_sm": list(rep.ctas_per_sm), "max_ctas": list(rep.max_ctas),
                "apply_ms": rep.apply_ms}
