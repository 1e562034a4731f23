"""The C-ABI library loads and exports every entry point declared in include/hsgn.h.

Runs on CPU: only host-side logic is exercised (symbol table, error strings,
argument validation that happens before any CUDA call, workspace sizing).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hsgn.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hsgn_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_07539_gb300 import build, solver
    build.build()
    return solver.load()


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for required in ("hsgn_create", "hsgn_step", "hsgn_run", "hsgn_adjoint", "hsgn_destroy",
                     "hsgn_set_state", "hsgn_get_state", "hsgn_tridiag_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_error_strings(lib):
    for code in range(0, 9):
        s = lib.hsgn_error_string(code)
        assert s and len(s) > 1
    assert b"unknown" in lib.hsgn_error_string(99)


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    from paper_2510_07539_gb300.solver import Grid
    h = ctypes.c_void_p()
    bad = [Grid(2, 0.0, 1.0, 0, 0), Grid(10, 1.0, 0.0, 0, 0), Grid(10, 0.0, 1.0, 7, 0),
           Grid(10, 0.0, 1.0, 0, 1)]
    for g in bad:
        assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, None, 0, ctypes.byref(h)) == 1
    g = Grid(10, 0.0, 1.0, 0, 0)
    assert lib.hsgn_create(ctypes.byref(g), -1.0, 1.0, None, 0, ctypes.byref(h)) == 1
    assert lib.hsgn_create(ctypes.byref(g), 9.81, -1.0, None, 0, ctypes.byref(h)) == 1
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, None, 0x4000, ctypes.byref(h)) == 6
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, None, 0, None) == 1
    # a bottom needs the well-balanced form; in mixed precision that form runs
    # on the windowed kernel only (not with the exact separator solve)
    bottom = (ctypes.c_double * 10)()
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, bottom, 0, ctypes.byref(h)) == 1
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, bottom, 0x1, ctypes.byref(h)) == 1
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, bottom, 0x7, ctypes.byref(h)) == 6
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, None, 0x7, ctypes.byref(h)) == 6
    assert not h.value
    # comparison schemes: FP64 flat bottom only; an unknown scheme is invalid
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, None, 0x300 | 0x1, ctypes.byref(h)) == 6
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, None, 0x100 | 0x2, ctypes.byref(h)) == 6
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, None, 0x500, ctypes.byref(h)) == 1
    # the double-float form: not with the exact solve, nor with both the FP32-flux
    # split and the bottom form
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, None, 0x8 | 0x4, ctypes.byref(h)) == 6
    assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, None, 0x8 | 0x2 | 0x1, ctypes.byref(h)) == 6
    assert not h.value
    lib.hsgn_destroy(None)


def test_workspace_sizing(lib):
    nb = ctypes.c_size_t()
    assert lib.hsgn_tridiag_workspace_bytes(0, ctypes.byref(nb)) == 1
    assert lib.hsgn_tridiag_workspace_bytes(1000, ctypes.byref(nb)) == 0
    small = nb.value
    assert lib.hsgn_tridiag_workspace_bytes(10_000_000, ctypes.byref(nb)) == 0
    assert nb.value > 24 * 10_000_000 > small


def test_null_handle_calls_are_rejected(lib):
    assert lib.hsgn_step(None, 0.1, None) == 1
    assert lib.hsgn_run(None, 0.1, 1, None) == 1
    assert lib.hsgn_check(None, None) == 1
    buf = (ctypes.c_double * 4)()
    ptr = ctypes.cast(buf, ctypes.c_void_p)
    assert lib.hsgn_set_state(None, ptr, ptr, ptr, ptr, None) == 1
    assert lib.hsgn_get_state(None, ptr, ptr, ptr, ptr, None) == 1
    assert lib.hsgn_copy_state_out(None, ptr, ptr, ptr, ptr, None) == 1
    assert lib.hsgn_enqueue(None, 0.1, 1, None) == 1
    dt = ctypes.c_double()
    assert lib.hsgn_suggest_dt(None, 2.0, 0.5, ctypes.byref(dt), None) == 1
    v = (ctypes.c_int32 * 2)()
    assert lib.hsgn_batched_set_tiles(None, ctypes.cast(v, ctypes.c_void_p)) == 1
    assert lib.hsgn_batched_get_tiles(None, ctypes.cast(v, ctypes.c_void_p)) == 1
    i1, i2 = ctypes.c_int32(), ctypes.c_int32()
    assert lib.hsgn_df_overlap(None, ctypes.byref(i1), ctypes.byref(i2), None) == 1
    ms = (ctypes.c_double * 3)()
    ch = ctypes.c_int32()
    assert lib.hsgn_batched_autotune(None, 2, ctypes.cast(ms, ctypes.c_void_p), ctypes.byref(ch),
                                     None) == 1
    assert lib.hsgn_batched_set_dt(None, ctypes.cast(ms, ctypes.c_void_p)) == 1
    assert lib.hsgn_profile(None, 1) == 1
    lib.hsgn_destroy(None)


def test_batched_create_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    ns = (ctypes.c_int64 * 2)(100, 2)  # 2 cells: below the minimum of 3
    xl = (ctypes.c_double * 2)(0.0, 0.0)
    xr = (ctypes.c_double * 2)(10.0, 10.0)
    lm = (ctypes.c_double * 2)(100.0, 100.0)
    args = [ctypes.cast(a, ctypes.c_void_p) for a in (ns, xl, xr, lm)]
    assert lib.hsgn_create_batched(2, *args, 9.81, 0, 1, ctypes.byref(h)) == 1
    ns[1] = 100
    xr[1] = -1.0  # empty interval
    assert lib.hsgn_create_batched(2, *args, 9.81, 0, 1, ctypes.byref(h)) == 1
    xr[1] = 10.0
    lm[0] = -1.0  # negative lambda
    assert lib.hsgn_create_batched(2, *args, 9.81, 0, 1, ctypes.byref(h)) == 1
    lm[0] = 100.0
    assert lib.hsgn_create_batched(0, *args, 9.81, 0, 1, ctypes.byref(h)) == 1
    assert lib.hsgn_create_batched(2, *args, 9.81, 7, 1, ctypes.byref(h)) == 1  # unknown BC
    assert not h.value


def test_degenerate_grids_are_rejected(lib):
    # fewer than 3 cells (the stencil of a stage spans 5) is an invalid grid;
    # nothing is allocated
    from paper_2510_07539_gb300.solver import Grid
    h = ctypes.c_void_p()
    for n in (0, 1, 2, -5):
        g = Grid(n, 0.0, 1.0, 0, 0)
        for flags in (0, 0x1):
            assert lib.hsgn_create(ctypes.byref(g), 9.81, 1.0, None, flags, ctypes.byref(h)) == 1
    assert not h.value


@pytest.mark.parametrize("noalloc", [False, True])
def test_tridiag_wrappers_reject_bad_arrays_before_any_launch(noalloc):
    # A short array, or one that is not on the current CUDA device, would hand
    # the kernels a pointer they index past its end; the binding refuses both
    # before it touches the library or the device (this runs without a GPU).
    torch = pytest.importorskip("torch")
    from paper_2510_07539_gb300 import solver
    f = solver.tridiag_solve_noalloc if noalloc else solver.tridiag_solve
    n = 16
    ok = [torch.ones(n, dtype=torch.float64) for _ in range(4)]
    for k in range(4):
        bad = list(ok)
        bad[k] = torch.ones(n - 1, dtype=torch.float64)
        with pytest.raises(ValueError, match="entries"):
            f(*bad, periodic=False)
    with pytest.raises(ValueError, match="entries"):
        f(*ok, periodic=True, out=torch.empty(n + 1, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA"):
        f(*ok, periodic=False)
