"""Python binding of the C ABI in include/hsgn.h (argument marshalling only).

Every step of the numerical method runs in the CUDA library libhsgn.so; this
module passes torch tensor pointers and the current CUDA stream through ctypes.
Importing it loads the library and raises if it is missing: there is no CPU or
eager fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhsgn.so")

HSGN_OK = 0
BC_PERIODIC = 0
BC_TRANSMISSIVE = 1
FLAG_FP64 = 0x0
FLAG_MIXED = 0x1
FLAG_RUSANOV_LOCAL = 0x10
FLAG_WELL_BALANCED = 0x2
FLAG_EXACT_SOLVE = 0x4
FLAG_DOUBLE_FLOAT = 0x8
# time-stepping schemes (flags & SCHEME_MASK)
SCHEME_PRINTED, SCHEME_ARS222, SCHEME_SI1, SCHEME_EX_HEUN, SCHEME_EX_EULER = (
    0x000, 0x100, 0x200, 0x300, 0x400)
SCHEME_MASK = 0x700

ERROR_NAMES = {
    1: "HSGN_ERR_INVALID_ARG", 2: "HSGN_ERR_CUDA", 3: "HSGN_ERR_NONPOSITIVE_DEPTH",
    4: "HSGN_ERR_NOT_COERCIVE", 5: "HSGN_ERR_NONFINITE", 6: "HSGN_ERR_UNIMPLEMENTED",
    7: "HSGN_ERR_OUT_OF_MEMORY", 8: "HSGN_ERR_TRUNCATION",
}


class HsgnError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.hsgn_error_string(code).decode() if _lib is not None else "?"
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)} ({msg})")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x_left", ctypes.c_double), ("x_right", ctypes.c_double),
                ("bc", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I64 = ctypes.c_int64


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "hsgn_create": [ctypes.POINTER(Grid), _D, _D, _P, ctypes.c_int32, ctypes.POINTER(_P)],
        "hsgn_set_state": [_P, _P, _P, _P, _P, _P],
        "hsgn_get_state": [_P, _P, _P, _P, _P, _P],
        "hsgn_copy_state_out": [_P, _P, _P, _P, _P, _P],
        "hsgn_step": [_P, _D, _P],
        "hsgn_run": [_P, _D, _I64, _P],
        "hsgn_enqueue": [_P, _D, _I64, _P],
        "hsgn_profile": [_P, ctypes.c_int32],
        "hsgn_profile_read": [_P, _P, _P, ctypes.c_int32],
        "hsgn_check": [_P, _P],
        "hsgn_df_overlap": [_P, _P, _P, _P],
        "hsgn_suggest_dt": [_P, _D, _D, ctypes.POINTER(_D), _P],
        "hsgn_stage": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _D, ctypes.POINTER(_P), _P],
        "hsgn_adjoint": [_P, _D, _I64, _I64, _P, _P, _I64, _P, _P, _P, _P],
        "hsgn_tridiag_workspace_bytes": [_I64, ctypes.POINTER(ctypes.c_size_t)],
        "hsgn_create_batched": [ctypes.c_int32, _P, _P, _P, _P, _D, ctypes.c_int32, ctypes.c_int32,
                                ctypes.POINTER(_P)],
        "hsgn_batched_set_dt": [_P, _P],
        "hsgn_batched_suggest_dt": [_P, _D, _D, _P, _P],
        "hsgn_batched_set_tiles": [_P, _P],
        "hsgn_batched_get_tiles": [_P, _P],
        "hsgn_batched_autotune": [_P, ctypes.c_int32, _P, _P, _P],
        "hsgn_tridiag_solve": [_I64, ctypes.c_int32, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.hsgn_destroy.argtypes = [_P]
    lib.hsgn_destroy.restype = None
    lib.hsgn_error_string.argtypes = [ctypes.c_int]
    lib.hsgn_error_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != HSGN_OK:
        raise HsgnError(rc, where)


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor):
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("arrays must be contiguous float64 tensors")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One hSGN instance on the current CUDA device (owns its state on the device)."""

    def __init__(self, n: int, x_left: float, x_right: float, bc: int = BC_PERIODIC,
                 g: float = 9.81, lam: float = 100.0, flags: int = FLAG_FP64, bathymetry=None):
        """bathymetry: None (flat) or n bottom elevations (needs FLAG_WELL_BALANCED)."""
        load()
        self.n, self.bc, self.g, self.lam, self.flags = int(n), int(bc), float(g), float(lam), flags
        self.dx = (x_right - x_left) / n
        grid = Grid(int(n), float(x_left), float(x_right), int(bc), 0)
        bptr = None
        if bathymetry is not None:
            bt = bathymetry if isinstance(bathymetry, torch.Tensor) else \
                torch.as_tensor(bathymetry, dtype=torch.float64)
            if bt.numel() != self.n:
                raise ValueError(f"expected {self.n} bottom values")
            bt = bt.to(torch.float64).contiguous()
            bptr = _ptr(bt)  # copied synchronously by hsgn_create
        h = _P()
        _check(_lib.hsgn_create(ctypes.byref(grid), float(g), float(lam), bptr, int(flags),
                                ctypes.byref(h)), "hsgn_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.hsgn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, h, q, m, r, stream=None):
        ts = [t if isinstance(t, torch.Tensor) else torch.as_tensor(t, dtype=torch.float64)
              for t in (h, q, m, r)]
        for t in ts:
            if t.numel() != self.n:
                raise ValueError(f"expected {self.n} values")
        self._keep = ts  # the copy is asynchronous: keep the sources alive
        _check(_lib.hsgn_set_state(self._h, *(_ptr(t) for t in ts), _stream(stream)),
               "hsgn_set_state")

    def get_state(self, out=None, device="cuda", stream=None):
        if out is None:
            out = [torch.empty(self.n, dtype=torch.float64, device=device) for _ in range(4)]
        _check(_lib.hsgn_get_state(self._h, *(_ptr(t) for t in out), _stream(stream)),
               "hsgn_get_state")
        return tuple(out)

    def copy_state_out(self, out, stream=None):
        """Enqueue the copy of the state into `out` (four float64 tensors,
        device or pinned host) without waiting; errors surface at the next
        synchronising call (check, run, get_state)."""
        _check(_lib.hsgn_copy_state_out(self._h, *(_ptr(t) for t in out), _stream(stream)),
               "hsgn_copy_state_out")
        return tuple(out)

    def step(self, dt: float, stream=None):
        _check(_lib.hsgn_step(self._h, float(dt), _stream(stream)), "hsgn_step")

    def run(self, dt: float, n_steps: int, stream=None):
        _check(_lib.hsgn_run(self._h, float(dt), int(n_steps), _stream(stream)), "hsgn_run")

    def run_cfl(self, cfl: float, mcfl: float, n_steps: int, stream=None) -> float:
        """n_steps steps, each with dt from the CFL rule of its own state
        (hsgn_run_cfl, double-float forms); returns the time advanced."""
        f = _lib.hsgn_run_cfl
        f.argtypes = [_P, _D, _D, _I64, ctypes.POINTER(_D), _P]
        f.restype = ctypes.c_int
        t = _D()
        _check(f(self._h, float(cfl), float(mcfl), int(n_steps), ctypes.byref(t),
                 _stream(stream)), "hsgn_run_cfl")
        return t.value

    def enqueue(self, dt: float, n_steps: int, stream=None):
        _check(_lib.hsgn_enqueue(self._h, float(dt), int(n_steps), _stream(stream)), "hsgn_enqueue")

    def df_overlap(self, stream=None):
        """(rows the last step's coupling needed, overlap rows of the next
        step) of a double-float form (hsgn_df_overlap)."""
        need, ov = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(_lib.hsgn_df_overlap(self._h, ctypes.byref(need), ctypes.byref(ov),
                                    _stream(stream)), "hsgn_df_overlap")
        return int(need.value), int(ov.value)

    def profile(self, enable: bool):
        _check(_lib.hsgn_profile(self._h, int(bool(enable))), "hsgn_profile")

    def profile_read(self, reset: bool = True):
        """Returns {kind: (total_ms, launches)} for assemble / reduced / backsub."""
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_int64 * 3)()
        _check(_lib.hsgn_profile_read(self._h, ctypes.cast(ms, _P), ctypes.cast(cnt, _P),
                                      int(bool(reset))), "hsgn_profile_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(("assemble", "reduced", "backsub"))}

    def check(self, stream=None):
        _check(_lib.hsgn_check(self._h, _stream(stream)), "hsgn_check")

    def suggest_dt(self, cfl: float, mcfl: float, stream=None) -> float:
        dt = _D()
        _check(_lib.hsgn_suggest_dt(self._h, float(cfl), float(mcfl), ctypes.byref(dt),
                                    _stream(stream)), "hsgn_suggest_dt")
        return dt.value

    def stage(self, base, lin, tau: float, speed: float = 0.0, out=None, stream=None):
        if out is None:
            out = [torch.empty(self.n, dtype=torch.float64, device=base[0].device)
                   for _ in range(4)]
        arr = _P * 4
        b = arr(*(_ptr(t) for t in base))
        l_ = arr(*(_ptr(t) for t in lin))
        o = arr(*(_ptr(t) for t in out))
        _check(_lib.hsgn_stage(self._h, b, l_, float(tau), float(speed), o, _stream(stream)),
               "hsgn_stage")
        return tuple(out)

    def adjoint(self, dt: float, n_steps: int, gauge_cells, gauge_data, checkpoint_every: int = 100,
                stream=None):
        """Gauge misfit J of n_steps steps from the current state and its gradient
        (hsgn_adjoint): returns (J, [dJ/dh0, dJ/dq0, dJ/dm0, dJ/dr0], dJ/db); the
        state is left after the last step."""
        import numpy as np
        cells = np.ascontiguousarray(np.asarray(gauge_cells, dtype=np.int64))
        data = gauge_data if isinstance(gauge_data, torch.Tensor) else torch.as_tensor(
            np.asarray(gauge_data, dtype=np.float64))
        data = data.to(torch.float64).contiguous()
        if data.numel() != n_steps * cells.size:
            raise ValueError("gauge_data must hold n_steps x n_gauges values")
        dev = torch.device("cuda", torch.cuda.current_device())
        grads = [torch.empty(self.n, dtype=torch.float64, device=dev) for _ in range(4)]
        gb = torch.empty(self.n, dtype=torch.float64, device=dev)
        arr = _P * 4
        g4 = arr(*(_ptr(t) for t in grads))
        J = ctypes.c_double()
        self._keep = (cells, data)
        _check(_lib.hsgn_adjoint(self._h, float(dt), int(n_steps), int(cells.size),
                                 cells.ctypes.data_as(ctypes.c_void_p), _ptr(data),
                                 int(checkpoint_every), g4, _ptr(gb), ctypes.byref(J),
                                 _stream(stream)), "hsgn_adjoint")
        return J.value, grads, gb


class GaugeMisfit(torch.autograd.Function):
    """J(h0, q0, m0, r0, b) = 1/2 sum_s sum_g (h_g^s - d_{s,g})^2 dt over n_steps
    steps of the paper's scheme in the well-balanced FP64 form, with its exact
    discrete gradient (hsgn_adjoint) for backward. Inputs are float64 CUDA
    tensors of n cells; b is the bottom."""

    @staticmethod
    def forward(ctx, h0, q0, m0, r0, b, x_left, x_right, bc, lam, dt, n_steps, gauge_cells,
                gauge_data, checkpoint_every=100):
        n = h0.numel()
        with Solver(n, x_left, x_right, bc, lam=lam, flags=FLAG_WELL_BALANCED,
                    bathymetry=b.detach()) as s:
            s.set_state(*(t.detach().contiguous() for t in (h0, q0, m0, r0)))
            J, grads, gb = s.adjoint(dt, n_steps, gauge_cells, gauge_data, checkpoint_every)
        ctx.save_for_backward(*grads, gb)
        return torch.tensor(J, dtype=torch.float64, device=h0.device)

    @staticmethod
    def backward(ctx, gJ):
        gh, gq, gm, gr, gb = ctx.saved_tensors
        return (gJ * gh, gJ * gq, gJ * gm, gJ * gr, gJ * gb) + (None,) * 9


def fma_peak(bits: int, stream=None) -> float:
    """Measured fused multiply-add throughput of the current device in
    TFLOP/s, single (32) or double (64) precision (hsgn_fma_peak)."""
    lib = load()
    f = lib.hsgn_fma_peak
    f.argtypes = [ctypes.c_int32, ctypes.POINTER(_D), _P]
    f.restype = ctypes.c_int
    out = _D()
    _check(f(int(bits), ctypes.byref(out), _stream(stream)), "hsgn_fma_peak")
    return out.value


def tridiag_workspace_bytes(n: int) -> int:
    load()
    nb = ctypes.c_size_t()
    _check(_lib.hsgn_tridiag_workspace_bytes(int(n), ctypes.byref(nb)), "hsgn_tridiag_workspace_bytes")
    return nb.value


def _check_rows(a, b, c, d, out):
    """Every array of a tridiagonal call has b's length and lives on the current
    CUDA device (the kernels index all of them up to n - 1)."""
    n = b.numel()
    arrays = (a, b, c, d) + (() if out is None else (out,))
    for t in arrays:
        if t.numel() != n:
            raise ValueError(f"tridiagonal arrays must all have {n} entries, got {t.numel()}")
    for t in arrays:
        if t.device.type != "cuda" or t.device.index != torch.cuda.current_device():
            raise ValueError("tridiagonal arrays must be CUDA tensors on the current device")
    return n


def tridiag_solve(a, b, c, d, periodic: bool, stream=None, out=None, workspace=None):
    """Solve the (cyclic) tridiagonal system on the GPU; returns x (a new
    tensor, or `out`). `workspace`: a uint8 device tensor of at least
    tridiag_workspace_bytes(n) + 256 bytes, allocated here when None."""
    n = _check_rows(a, b, c, d, out)
    load()
    x = torch.empty_like(d) if out is None else out
    nbytes = tridiag_workspace_bytes(n)
    ws = workspace
    if ws is not None and (ws.device.type != "cuda"
                           or ws.device.index != torch.cuda.current_device()):
        raise ValueError("the workspace must be a CUDA tensor on the current device")
    if ws is None or ws.numel() < max(nbytes, 256) + 256:
        ws = torch.empty(max(nbytes, 256) + 256, dtype=torch.uint8, device=d.device)
    base = ws.data_ptr()
    aligned = (base + 255) // 256 * 256
    _check(_lib.hsgn_tridiag_solve(int(n), int(bool(periodic)), _ptr(a), _ptr(b), _ptr(c), _ptr(d),
                                   _ptr(x), ctypes.c_void_p(aligned), ctypes.c_size_t(nbytes),
                                   _stream(stream)), "hsgn_tridiag_solve")
    return x


NOALLOC_MAX_N = 262144


def tridiag_solve_noalloc(a, b, c, d, periodic: bool, out=None, stream=None):
    """Same solve as tridiag_solve through the entry point that allocates
    nothing (fixed device scratch inside the library, n <= NOALLOC_MAX_N)."""
    _check_rows(a, b, c, d, out)
    lib = load()
    f = lib.hsgn_tridiag_solve_noalloc
    f.argtypes = [_I64, ctypes.c_int32, _P, _P, _P, _P, _P, _P]
    f.restype = ctypes.c_int
    x = torch.empty_like(d) if out is None else out
    _check(f(int(b.numel()), int(bool(periodic)), _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x),
             _stream(stream)), "hsgn_tridiag_solve_noalloc")
    return x


class BatchedSolver(Solver):
    """A batch of independent instances (packed state, mixed precision).

    ns, x_left, x_right, lams: one entry per instance. The state arrays passed
    to set_state / returned by get_state are the instances' arrays
    concatenated in order; `offsets` gives each instance's first cell."""

    def __init__(self, ns, x_left, x_right, lams, bc: int = BC_PERIODIC, g: float = 9.81,
                 flags: int = FLAG_MIXED):
        import numpy as np
        load()
        ns = np.ascontiguousarray(ns, dtype=np.int64)
        xl = np.ascontiguousarray(x_left, dtype=np.float64)
        xr = np.ascontiguousarray(x_right, dtype=np.float64)
        lm = np.ascontiguousarray(lams, dtype=np.float64)
        self.count = int(len(ns))
        self.ns = ns
        self.offsets = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        self.n = int(self.offsets[-1])
        self.bc, self.g, self.flags = int(bc), float(g), flags
        h = _P()
        _check(_lib.hsgn_create_batched(self.count, ns.ctypes.data, xl.ctypes.data, xr.ctypes.data,
                                        lm.ctypes.data, float(g), int(bc), int(flags),
                                        ctypes.byref(h)), "hsgn_create_batched")
        self._h = h

    def set_dt(self, dts):
        import numpy as np
        d = np.ascontiguousarray(dts, dtype=np.float64)
        if d.shape != (self.count,):
            raise ValueError(f"expected {self.count} time steps")
        _check(_lib.hsgn_batched_set_dt(self._h, d.ctypes.data), "hsgn_batched_set_dt")

    def suggest_dt(self, cfl: float, mcfl: float, stream=None):
        import numpy as np
        out = np.empty(self.count)
        _check(_lib.hsgn_batched_suggest_dt(self._h, float(cfl), float(mcfl), out.ctypes.data,
                                            _stream(stream)), "hsgn_batched_suggest_dt")
        return out

    def set_tiles(self, variant):
        """Per instance the batch variant 0 .. 3 (hsgn_batched_set_tiles)."""
        import numpy as np
        v = np.ascontiguousarray(variant, dtype=np.int32)
        if v.shape != (self.count,):
            raise ValueError(f"expected {self.count} variants")
        _check(_lib.hsgn_batched_set_tiles(self._h, v.ctypes.data), "hsgn_batched_set_tiles")

    def get_tiles(self):
        """Per instance the batch variant in use (hsgn_batched_get_tiles)."""
        import numpy as np
        v = np.empty(self.count, dtype=np.int32)
        _check(_lib.hsgn_batched_get_tiles(self._h, v.ctypes.data), "hsgn_batched_get_tiles")
        return v

    def autotune(self, steps: int = 4, stream=None):
        """Pick the tiles of the batch by timing (the state is kept); returns
        the ms per step with every instance on variant 0, 1, 2, 3 and of the
        cost-model assignment (NaN if not timed or ruled out) and the choice
        kept (0 .. 3 for one variant everywhere, 4 for the assignment)."""
        import numpy as np
        ms = np.empty(5)
        ch = ctypes.c_int32(-1)
        _check(_lib.hsgn_batched_autotune(self._h, int(steps), ms.ctypes.data, ctypes.byref(ch),
                                          _stream(stream)), "hsgn_batched_autotune")
        return {"ms_per_step": [float(x) for x in ms], "choice": int(ch.value)}

    def step(self, dt: float = 0.0, stream=None):
        super().step(0.0, stream)

    def run(self, dt: float = 0.0, n_steps: int = 1, stream=None):
        super().run(0.0, n_steps, stream)

    def enqueue(self, dt: float = 0.0, n_steps: int = 1, stream=None):
        super().enqueue(0.0, n_steps, stream)
