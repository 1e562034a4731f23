"""FP64 CPU oracle of the semi-implicit IMEX hSGN step (test infrastructure).

This package is the plain, serial reference that the CUDA library is checked
against. Only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product path never does. It shares no code with
the CUDA library: the arithmetic lives in ``hsgn_oracle.c`` (plain C, compiled
with ``-O2 -ffp-contract=off`` so that no multiply-add is fused), and this file
only marshals numpy arrays through ctypes.

Paper: Macca, Boscheri, Ricchiuto, "Semi-implicit strategies for the
Serre-Green-Naghdi equations in hyperbolic form" (arXiv 2510.07539); the C file
cites the section and equation of every step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsgn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libhsgn_oracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC = 0
BC_TRANSMISSIVE = 1

# time-stepping schemes of run/step (see hsgn_oracle.c)
SCHEME_PRINTED, SCHEME_ARS222, SCHEME_SI1, SCHEME_EX_HEUN, SCHEME_EX_EULER = 0, 1, 2, 3, 4

ERRORS = {
    0: "ok",
    1: "invalid argument",
    2: "non-positive depth",
    3: "not coercive (beta <= 0 or zero pivot)",
    4: "non-finite value",
    5: "out of memory",
}


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: oracle error {code} ({ERRORS.get(code, '?')})")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("dx", ctypes.c_double),
        ("bc", ctypes.c_int32),
        ("delta_half", ctypes.c_int32),
        ("g", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("rusanov", ctypes.c_int32),
        ("form", ctypes.c_int32),
        ("speed", ctypes.c_double),
        ("bathy", ctypes.POINTER(ctypes.c_double)),
        ("recon", ctypes.c_int32),
        ("scheme", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(ctypes.c_double)
        lib.oracle_tridiag_solve.argtypes = [ctypes.c_int64, ctypes.c_int32] + [P] * 5
        lib.oracle_stage.argtypes = [ctypes.POINTER(_Params)] + [P] * 8 + [ctypes.c_double] + [P] * 4
        lib.oracle_assemble.argtypes = ([ctypes.POINTER(_Params)] + [P] * 8 + [ctypes.c_double]
                                        + [P] * 9)
        lib.oracle_run.argtypes = [ctypes.POINTER(_Params)] + [P] * 4 + [ctypes.c_double,
                                                                         ctypes.c_int64]
        lib.oracle_imex_scalar.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int64, P]
        lib.oracle_imex_scalar_scheme.argtypes = ([ctypes.c_int32] + [ctypes.c_double] * 4
                                                  + [ctypes.c_int64, P])
        lib.oracle_explicit_rhs.argtypes = [ctypes.POINTER(_Params)] + [P] * 8
        lib.oracle_stage_adjoint.argtypes = ([ctypes.POINTER(_Params)] + [P] * 8 + [ctypes.c_double]
                                             + [P] * 14)
        I64P = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_adjoint.argtypes = ([ctypes.POINTER(_Params)] + [P] * 4
                                       + [ctypes.c_double, ctypes.c_int64, ctypes.c_int64, I64P, P,
                                          P] + [P] * 5)
        lib.oracle_suggest_dt.argtypes = ([ctypes.POINTER(_Params)] + [P] * 3
                                          + [ctypes.c_double] * 2 + [P] * 3)
        for f in ("oracle_tridiag_solve", "oracle_stage", "oracle_assemble", "oracle_run",
                  "oracle_imex_scalar", "oracle_imex_scalar_scheme", "oracle_explicit_rhs",
                  "oracle_stage_adjoint", "oracle_adjoint",
                  "oracle_suggest_dt"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _f64(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None and a.shape != (n,):
        raise ValueError(f"expected shape ({n},), got {a.shape}")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, where: str):
    if rc != 0:
        raise OracleError(rc, where)


class Params:
    """Grid and physics of one hSGN instance (uniform 1D grid of n cells)."""

    def __init__(self, n, dx, bc=BC_PERIODIC, g=9.81, lam=100.0, delta_half=False,
                 rusanov=1, speed=0.0, form=0, bathy=None, recon=1, scheme=0):
        self.n, self.dx, self.bc, self.g, self.lam = int(n), float(dx), int(bc), float(g), float(lam)
        self.delta_half = bool(delta_half)
        self.rusanov, self.speed = int(rusanov), float(speed)
        self.form = int(form)
        self.bathy = None if bathy is None else _f64(bathy, self.n)
        self.recon, self.scheme = int(recon), int(scheme)

    def _c(self) -> _Params:
        bp = _ptr(self.bathy) if self.bathy is not None else None
        return _Params(self.n, self.dx, self.bc, int(self.delta_half), self.g, self.lam,
                       self.rusanov, self.form, self.speed, bp, self.recon, self.scheme)


def tridiag_solve(a, b, c, d, periodic: bool) -> np.ndarray:
    """Solve a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i] (cyclic if periodic)."""
    n = len(b)
    a, b, c, d = (_f64(v, n) for v in (a, b, c, d))
    x = np.empty(n)
    _check(_load().oracle_tridiag_solve(n, int(periodic), _ptr(a), _ptr(b), _ptr(c), _ptr(d),
                                        _ptr(x)), "tridiag_solve")
    return x


def stage(p: Params, Ub, Ul, tau: float):
    """One implicit stage: returns (h, q, m, r) from base Ub and linearisation Ul."""
    n = p.n
    ub = [_f64(v, n) for v in Ub]
    ul = [_f64(v, n) for v in Ul]
    out = [np.empty(n) for _ in range(4)]
    pc = p._c()
    _check(_load().oracle_stage(ctypes.byref(pc), *map(_ptr, ub), *map(_ptr, ul), float(tau),
                                *map(_ptr, out)), "stage")
    return tuple(out)


def assemble(p: Params, Ub, Ul, tau: float) -> dict:
    """Per-cell assembled quantities of one stage (starred values, coefficients, rows)."""
    n = p.n
    ub = [_f64(v, n) for v in Ub]
    ul = [_f64(v, n) for v in Ul]
    names = ("qs", "ms", "rs", "beta", "delta", "a", "b", "c", "d")
    out = {k: np.empty(n) for k in names}
    pc = p._c()
    _check(_load().oracle_assemble(ctypes.byref(pc), *map(_ptr, ub), *map(_ptr, ul), float(tau),
                                   *(_ptr(out[k]) for k in names)), "assemble")
    return out


def run(p: Params, U, dt: float, n_steps: int):
    """n_steps IMEX steps of size dt; returns a new (h, q, m, r) tuple."""
    n = p.n
    st = [np.array(_f64(v, n), copy=True) for v in U]
    pc = p._c()
    _check(_load().oracle_run(ctypes.byref(pc), *map(_ptr, st), float(dt), int(n_steps)), "run")
    return tuple(st)


def step(p: Params, U, dt: float):
    return run(p, U, dt, 1)


def imex_scalar(aE: float, aI: float, y: float, dt: float, n_steps: int = 1,
                scheme: int = 0) -> float:
    """Steps of y' = aE y + aI y (aE explicit, aI implicit) with scheme `scheme`."""
    out = ctypes.c_double()
    _check(_load().oracle_imex_scalar_scheme(int(scheme), float(aE), float(aI), float(y),
                                             float(dt), int(n_steps), ctypes.byref(out)),
           "imex_scalar")
    return out.value


def explicit_rhs(p: Params, U):
    """Right-hand side L(U) of the explicit hSGN scheme (Sec. 4.4), 4 arrays."""
    n = p.n
    u = [_f64(v, n) for v in U]
    out = [np.empty(n) for _ in range(4)]
    pc = p._c()
    _check(_load().oracle_explicit_rhs(ctypes.byref(pc), *map(_ptr, u), *map(_ptr, out)),
           "explicit_rhs")
    return out


def suggest_dt(p: Params, U, cfl: float, mcfl: float):
    """Returns (dt, nu_max, u_max) from the time-step rule."""
    n = p.n
    h, q, m = (_f64(v, n) for v in U[:3])
    dt, nu, um = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    pc = p._c()
    _check(_load().oracle_suggest_dt(ctypes.byref(pc), _ptr(h), _ptr(q), _ptr(m), float(cfl),
                                     float(mcfl), ctypes.byref(dt), ctypes.byref(nu),
                                     ctypes.byref(um)), "suggest_dt")
    return dt.value, nu.value, um.value


def stage_adjoint(p: Params, Ub, Ul, tau: float, Ao):
    """Adjoint of one stage (form 1, global speed): given dJ/dU_out (4 arrays)
    returns (dJ/dU_b, dJ/dU_l, dJ/db, dJ/ds)."""
    n = p.n
    ub = [_f64(v, n) for v in Ub]
    ul = [_f64(v, n) for v in Ul]
    ao = [_f64(v, n) for v in Ao]
    ab = [np.zeros(n) for _ in range(4)]
    al = [np.zeros(n) for _ in range(4)]
    gb = np.zeros(n)
    sa = np.zeros(1)
    pc = p._c()
    _check(_load().oracle_stage_adjoint(ctypes.byref(pc), *map(_ptr, ub), *map(_ptr, ul),
                                        float(tau), *map(_ptr, ao), *map(_ptr, ab),
                                        *map(_ptr, al), _ptr(gb), _ptr(sa)), "stage_adjoint")
    return ab, al, gb, float(sa[0])


def misfit(states_h, gauge_cells, gauge_data, dt):
    """J = 1/2 sum_s sum_g (h_g^s - d_{s,g})^2 dt for the depths after each step."""
    e = np.asarray(states_h)[:, np.asarray(gauge_cells)] - np.asarray(gauge_data)
    return 0.5 * float(np.sum(e * e)) * dt


def adjoint(p: Params, U, dt: float, n_steps: int, gauge_cells, gauge_data):
    """(J, [dJ/dh0, dJ/dq0, dJ/dm0, dJ/dr0], dJ/db, final state) of the gauge
    misfit over n_steps steps of the paper's scheme (form 1, global speed)."""
    n = p.n
    u = [_f64(v, n).copy() for v in U]
    cells = np.ascontiguousarray(gauge_cells, dtype=np.int64)
    data = np.ascontiguousarray(gauge_data, dtype=np.float64).reshape(n_steps, len(cells))
    g = [np.zeros(n) for _ in range(4)]
    gb = np.zeros(n)
    J = np.zeros(1)
    pc = p._c()
    _check(_load().oracle_adjoint(ctypes.byref(pc), *map(_ptr, u), float(dt), int(n_steps),
                                  len(cells), cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  _ptr(data), _ptr(J), *map(_ptr, g), _ptr(gb)), "adjoint")
    return float(J[0]), g, gb, u
