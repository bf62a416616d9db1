"""Host-side plan of an uneven batch (include/dbi_group.h): slot and field offsets, workspace
sizes and argument checks. The plan is built on the host from member descriptors; the device
pointers are only stored, so placeholder addresses suffice and no GPU is needed."""
import ctypes

import pytest

from paper_2402_02116_gb300 import build, dbi

FAKE = 0x100000  # placeholder device address (never dereferenced by the planner)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dbi.load()


def member(nz, nx, lz, lx, B, nf=2, h=5.0):
    m = dbi.GroupMember()
    m.model.grid = dbi.make_grid(nz, nx, lz, lx, h)
    m.model.ref = dbi.make_medium(2000.0, 2000.0, 1155.0)
    m.model.m = FAKE
    m.Ghat, m.omega, m.fidx = FAKE, FAKE, FAKE
    m.nf, m.B = nf, B
    return m


def make(lib, specs, precision=dbi.C64):
    arr = (dbi.GroupMember * len(specs))(*[member(*s) for s in specs])
    h = ctypes.c_void_p()
    rc = lib.dbi_group_create(arr, len(specs), precision, ctypes.byref(h))
    return rc, h


def test_offsets_follow_the_members_in_order(lib):
    specs = [(64, 64, 128, 128, 3), (20, 12, 64, 32, 2), (256, 256, 512, 512, 1), (8, 8, 16, 16, 4)]
    rc, h = make(lib, specs)
    assert rc == 0
    try:
        slots = sum(s[4] for s in specs)
        assert lib.dbi_group_slots(h) == slots
        want = [0]
        for nz, nx, _, _, B in specs:
            for _ in range(B):
                want.append(want[-1] + 2 * nz * nx)
        assert lib.dbi_group_field_elems(h) == want[-1]
        offs = (ctypes.c_longlong * (slots + 1))()
        assert lib.dbi_group_offsets(h, offs) == 0
        assert list(offs) == want
        apply_b = lib.dbi_group_workspace_bytes(h, dbi.OP_APPLY)
        solve_b = lib.dbi_group_workspace_bytes(h, dbi.OP_SOLVE)
        spectra = sum(2 * B * lx * nz * 8 for nz, nx, lz, lx, B in specs)
        assert apply_b >= spectra and solve_b >= apply_b + 6 * want[-1] * 8
        assert lib.dbi_group_workspace_bytes(h, dbi.OP_FRECHET) == 0
    finally:
        lib.dbi_group_destroy(h)


def test_complex128_plan_needs_more_workspace(lib):
    specs = [(32, 32, 64, 64, 2), (16, 16, 32, 32, 1)]
    _, h64 = make(lib, specs, dbi.C64)
    _, h128 = make(lib, specs, dbi.C128)
    try:
        assert lib.dbi_group_workspace_bytes(h128, dbi.OP_SOLVE) > lib.dbi_group_workspace_bytes(h64, dbi.OP_SOLVE)
    finally:
        lib.dbi_group_destroy(h64)
        lib.dbi_group_destroy(h128)


def test_bad_members_are_rejected(lib):
    for specs, code, text in (([(32, 32, 48, 64, 1)], -2, b"power of two"),
                              ([(40, 32, 64, 64, 1)], -1, b"too small"),
                              ([(32, 32, 64, 64, 0)], -1, b"B >= 1")):
        rc, h = make(lib, specs)
        assert rc == code and not h.value, specs
        assert text in lib.dbi_last_error()
    h = ctypes.c_void_p()
    assert lib.dbi_group_create(None, 0, dbi.C64, ctypes.byref(h)) == -1
    m = (dbi.GroupMember * 1)(member(8, 8, 16, 16, 1))
    m[0].Ghat = None
    assert lib.dbi_group_create(m, 1, dbi.C64, ctypes.byref(h)) == -1


def test_length_768_members_are_complex64_only(lib):
    """FFT length 768 (3 x 256) is a complex64 length: a member with it is planned in complex64, and
    its row stages add a contrast-source scratch field per slot to the workspace; complex128 rejects
    it like any other length that is not a power of two."""
    specs = [(384, 384, 768, 768, 2), (40, 300, 128, 768, 1), (64, 64, 128, 128, 3)]
    rc, h = make(lib, specs, dbi.C64)
    assert rc == 0
    try:
        spectra = sum(2 * B * lx * nz * 8 for nz, nx, lz, lx, B in specs)
        sources = sum(2 * B * nz * nx * 8 for nz, nx, lz, lx, B in specs if lx == 768)
        assert lib.dbi_group_workspace_bytes(h, dbi.OP_APPLY) >= spectra + sources
    finally:
        lib.dbi_group_destroy(h)
    rc, h = make(lib, specs, dbi.C128)
    assert rc == -2 and not h.value and b"power of two" in lib.dbi_last_error()


def test_unbound_plan_refuses_work(lib):
    rc, h = make(lib, [(8, 8, 16, 16, 1)])
    try:
        assert lib.ls_apply_group(h, FAKE, FAKE * 2, None) == -3
        assert b"not bound" in lib.dbi_last_error()
        opts = dbi.KrylovOpts(1e-6, 10, 2, 1)
        assert lib.ls_solve_group(h, FAKE, FAKE * 2, ctypes.byref(opts), None, 1, None) == -3
        assert lib.dbi_set_radix_plan(dbi.C64, 48, 1) == -1
    finally:
        lib.dbi_group_destroy(h)


def _pow2_at_least(n):
    return 1 << max(4, (n - 1).bit_length())


def test_random_plans_keep_their_invariants(lib):
    """200 seeded random member lists (1-6 members, grids 1-300 cells per side, FFT grids from the
    smallest allowed up to twice that, 1-5 slots each, both precisions): the slot count, the field
    offsets (members and their slots in order, 2 nz nx elements each), the spectra held by the
    apply workspace, solve >= apply, and destroy."""
    import numpy as np
    rng = np.random.default_rng(23)
    for trial in range(200):
        specs = []
        for _ in range(int(rng.integers(1, 7))):
            nz, nx = int(rng.integers(1, 301)), int(rng.integers(1, 301))
            lz = min(1024, _pow2_at_least(2 * nz - 1) * int(rng.choice([1, 1, 2])))
            lx = min(1024, _pow2_at_least(2 * nx - 1) * int(rng.choice([1, 1, 2])))
            specs.append((nz, nx, lz, lx, int(rng.integers(1, 6))))
        prec = dbi.C64 if trial % 2 == 0 else dbi.C128
        rc, h = make(lib, specs, prec)
        assert rc == 0, (specs, lib.dbi_last_error())
        try:
            slots = sum(s[4] for s in specs)
            assert lib.dbi_group_slots(h) == slots
            offs = (ctypes.c_longlong * (slots + 1))()
            assert lib.dbi_group_offsets(h, offs) == 0
            want = [0]
            for nz, nx, _, _, B in specs:
                want += [want[-1] + 2 * nz * nx * (k + 1) for k in range(B)]
            assert list(offs) == want and lib.dbi_group_field_elems(h) == want[-1]
            csize = 8 if prec == dbi.C64 else 16
            spectra = sum(2 * B * lx * nz * csize for nz, nx, lz, lx, B in specs)
            apply_b = lib.dbi_group_workspace_bytes(h, dbi.OP_APPLY)
            assert apply_b >= spectra and lib.dbi_group_workspace_bytes(h, dbi.OP_SOLVE) >= apply_b
        finally:
            lib.dbi_group_destroy(h)


def test_random_invalid_members_are_rejected(lib):
    """A valid list with one member broken at random (FFT length not a power of two, FFT grid
    smaller than 2 n - 1, no slots) is rejected as a whole with no plan."""
    import numpy as np
    rng = np.random.default_rng(29)
    for trial in range(60):
        specs = [(16, 16, 32, 32, 1), (40, 24, 128, 64, 2)]
        kind = trial % 3
        nz, nx = int(rng.integers(2, 200)), int(rng.integers(2, 200))
        lz, lx = _pow2_at_least(2 * nz - 1), _pow2_at_least(2 * nx - 1)
        if kind == 0:  # not a power of two, and not 768 (3 x 256, a complex64 length)
            bl = 3 * lz // 2 if lz >= 32 else 48
            bad = (nz, nx, 640 if bl == 768 else bl, lx, 1)
        elif kind == 1:
            bad = (nz, nx, lz // 2 if lz > 16 and lz // 2 < 2 * nz - 1 else lz, lx // 2 if lx > 16 else 8, 1)
        else:
            bad = (nz, nx, lz, lx, 0)
        specs.insert(int(rng.integers(0, 3)), bad)
        rc, h = make(lib, specs)
        assert rc < 0 and not h.value, (bad, rc)
