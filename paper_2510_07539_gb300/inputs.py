"""Seeded synthetic inputs for the hSGN workloads (shared by tests and benchmark).

This module holds initial conditions and random test data only: no step of the
numerical method. Every generator is deterministic for a given seed
(``numpy.random.default_rng``). The default seed of a configuration is
``SEED_BASE + id`` with id 1..5 for the five workloads below.

Workloads (cell-centred point values on a uniform grid of n cells):
  1 solitary wave, flat bottom, periodic (Sec. 6.3 closed form)
  2 smoothed dam break / undular bore, transmissive (tanh smoothing, Sec. 6.4)
  3 batch of independent periodic solitary waves of uneven length
  4 wave over a random smooth bathymetry (sum of Gaussians)
  5 solitary wave towards a 1:20 shelf (Sec. 6.4.3 geometry)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

G = 9.81
SEED_BASE = 20251007


def cell_centres(n: int, x_left: float, x_right: float):
    dx = (x_right - x_left) / n
    return x_left + (np.arange(n) + 0.5) * dx, dx


# --------------------------------------------------------------------------
# SGN solitary wave (Sec. 6.3): h = h0 (1 + eps sech^2(k (x - x0 - C t))),
# u = C (1 - h0/h), C = sqrt(g h0 (1 + eps)), k = sqrt(3 eps / (4 h0^2 (1 + eps))).
# Auxiliary hSGN variables as in Sec. 6.3.1: eta = h, w = -h u_x.
# --------------------------------------------------------------------------
def solitary_params(h0: float, amp: float, g: float = G):
    eps = amp / h0
    speed = math.sqrt(g * h0 * (1.0 + eps))
    kappa = math.sqrt(3.0 * eps / (4.0 * h0 * h0 * (1.0 + eps)))
    return eps, speed, kappa


def solitary(x, h0: float, amp: float, x0: float = 0.0, t: float = 0.0, g: float = G,
             period: float | None = None):
    """(h, q, m, r) of the solitary wave; `period` wraps the distance to the crest."""
    eps, speed, kappa = solitary_params(h0, amp, g)
    xi = np.asarray(x, dtype=np.float64) - x0 - speed * t
    if period is not None:
        xi = (xi + 0.5 * period) % period - 0.5 * period
    th = np.tanh(kappa * xi)
    sech2 = 1.0 - th * th
    h = h0 * (1.0 + eps * sech2)
    u = speed * (1.0 - h0 / h)
    hx = -2.0 * h0 * eps * kappa * sech2 * th
    ux = speed * h0 * hx / (h * h)
    return h, h * u, h * h, -h * h * ux


def gaussian_bell(n: int = 5000, x_left: float = -200.0, x_right: float = 200.0,
                  h_inf: float = 1.0, amp: float = 1.0):
    """The breakdown of a Gaussian bell (Sec. 6.1): h = h_inf + amp exp(-x^2/20),
    u = 0, eta = h, w = 0 on [x_left, x_right]: x, dx, (h, q, m, r)."""
    x, dx = cell_centres(n, x_left, x_right)
    h = h_inf + amp * np.exp(-x * x / 20.0)
    z = np.zeros(n)
    return x, dx, (h, z.copy(), h * h, z.copy())


# --------------------------------------------------------------------------
# Smoothed dam break: h = (hl + hr)/2 - (hl - hr)/2 tanh(x / (w dx)), u = 0,
# eta = h, w = 0 (the tanh smoothing of the Favre-wave set-up, Sec. 6.4).
# --------------------------------------------------------------------------
def dam_break(n: int, dx: float, h_left: float = 1.2, h_right: float = 1.0,
              width_cells: float = 5.0):
    x = (np.arange(n) + 0.5 - 0.5 * n) * dx
    h = 0.5 * (h_left + h_right) - 0.5 * (h_left - h_right) * np.tanh(x / (width_cells * dx))
    z = np.zeros(n)
    return x, (h, z.copy(), h * h, z.copy())


# --------------------------------------------------------------------------
# Random smooth positive states and random hSGN-like tridiagonal systems for
# parity tests. Smoothness: a few random Fourier modes per field.
# --------------------------------------------------------------------------
def _smooth_field(rng, x, length, modes=6, amp=1.0):
    f = np.zeros_like(x)
    for k in range(1, modes + 1):
        a, b = rng.normal(size=2) * amp / k
        f += a * np.cos(2 * np.pi * k * x / length) + b * np.sin(2 * np.pi * k * x / length)
    return f


def random_state(seed: int, n: int, dx: float = 0.1, h_mean: float = 1.0, h_var: float = 0.15,
                 u_amp: float = 0.3, eta_rel: float = 0.02, w_amp: float = 0.05):
    """A smooth periodic state with h in about h_mean +- h_var and eta close to h."""
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) * dx
    length = n * dx

    def unit(f):
        return f / max(1e-300, np.max(np.abs(f)))

    h = h_mean + h_var * unit(_smooth_field(rng, x, length))
    u = u_amp * unit(_smooth_field(rng, x, length))
    eta = h * (1.0 + eta_rel * unit(_smooth_field(rng, x, length)))
    w = w_amp * unit(_smooth_field(rng, x, length))
    return h, h * u, h * eta, h * w


def random_tridiag(seed: int, n: int, periodic: bool, coupling: float = 3.0):
    """Rows a, b, c, d of an SPD, strictly diagonally dominant system with the
    structure of the hSGN depth matrix: off-diagonals -k_{i+1/2} < 0, diagonal
    1 + k_{i-1/2} + k_{i+1/2}. Non-periodic systems have a[0] = c[n-1] = 0."""
    rng = np.random.default_rng(seed)
    k = coupling * rng.uniform(0.2, 1.0, size=n)  # k[i] couples i and i+1 (cyclic)
    km = np.roll(k, 1)
    a, c = -km.copy(), -k.copy()
    b = 1.0 + km + k
    if not periodic:
        a[0] = 0.0
        c[-1] = 0.0
        b[0] = 1.0 + k[0]
        b[-1] = 1.0 + km[-1]
    d = rng.normal(size=n)
    return a, b, c, d


# --------------------------------------------------------------------------
# Batched workload: independent periodic instances of uneven length.
# --------------------------------------------------------------------------
@dataclass
class Instance:
    n: int
    dx: float
    lam: float
    amp: float
    state: tuple


def batched_instances(seed: int, count: int, n_min: int = 256, n_max: int = 8192,
                      dx: float = 0.1, h0: float = 1.0, lams=(10.0, 100.0, 1000.0),
                      amp_range=(0.05, 0.4)):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_min, n_max + 1))
        amp = float(rng.uniform(*amp_range))
        lam = float(lams[int(rng.integers(0, len(lams)))])
        length = n * dx
        x, _ = cell_centres(n, -0.5 * length, 0.5 * length)
        out.append(Instance(n, dx, lam, amp, solitary(x, h0, amp, 0.0, period=length)))
    return out


# --------------------------------------------------------------------------
# Bathymetries.
# --------------------------------------------------------------------------
def gaussian_bathymetry(seed: int, x, count: int = 8, amp_max: float = 0.3,
                        width=(2.0, 10.0), clip: float = 0.6):
    rng = np.random.default_rng(seed)
    lo, hi = float(np.min(x)), float(np.max(x))
    b = np.zeros_like(x)
    for _ in range(count):
        a = rng.uniform(0.0, amp_max)
        w = rng.uniform(*width)
        xc = rng.uniform(lo, hi)
        b += a * np.exp(-((x - xc) ** 2) / (2.0 * w * w))
    return np.minimum(b, clip)


def shelf_bathymetry(x, x_toe: float, slope: float = 1.0 / 20.0, rise: float = 0.5):
    return np.clip((x - x_toe) * slope, 0.0, rise)


def wave_over_bottom(x, b, h0: float, amp: float, x0: float, period: float | None = None):
    """Still water at level h0 over the bottom b plus a solitary wave of
    amplitude amp centred at x0: h = h_sol - b, u = u_sol, eta = h, w = -h u_x
    (the flat-bottom wave's velocity field; not an exact solution over b)."""
    hs, qs, _, rs = solitary(x, h0, amp, x0, period=period)
    u = qs / hs
    ux = -rs / (hs * hs)
    h = hs - b
    return h, h * u, h * h, -h * h * ux


def gauss_bottom_wave(seed: int, n: int = 4096, dx: float = 0.1, amp: float = 0.1):
    """Periodic wave over a sum of 8 Gaussians (amplitudes up to 0.3, widths
    2-10, clipped at 0.6) on [0, n dx]: x, dx, b, U."""
    x, dx = cell_centres(n, 0.0, n * dx)
    b = gaussian_bathymetry(seed, x)
    L = n * dx
    return x, dx, b, wave_over_bottom(x, b, 1.0, amp, 0.5 * L, period=L)


def shelf_wave(n: int = 1 << 24, dx: float = 0.005, amp: float = 0.1):
    """Solitary wave of amplitude amp at L/2 - 80 running towards a 1:20 ramp
    that starts at L/2 and lifts the bottom by 0.5 (depth 1 -> 0.5), on
    [0, L], L = n dx: x, dx, b, U."""
    x, dx = cell_centres(n, 0.0, n * dx)
    L = n * dx
    b = shelf_bathymetry(x, 0.5 * L)
    return x, dx, b, wave_over_bottom(x, b, 1.0, amp, 0.5 * L - 80.0)
