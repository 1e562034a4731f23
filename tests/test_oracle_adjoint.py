"""Pins of the oracle's discrete adjoint (CPU, no GPU): the adjoint of one
stage and the gradient of a gauge misfit over a run, both against central
finite differences of the forward oracle along random smooth directions
(the derivative the adjoint must reproduce is fixed by the forward scheme
alone). Form 1 (well-balanced) with the global Rusanov speed."""
import math

import numpy as np
import pytest

import oracle
from paper_2510_07539_gb300 import inputs


def smooth(rng, n, modes=5):
    x = np.arange(n) / n
    f = np.zeros(n)
    for k in range(1, modes + 1):
        a, b = rng.normal(size=2) / k
        f += a * np.cos(2 * np.pi * k * x) + b * np.sin(2 * np.pi * k * x)
    return f / np.max(np.abs(f))


def bottom(n, dx, seed=3):
    x, _ = inputs.cell_centres(n, 0.0, n * dx)
    b = inputs.gaussian_bathymetry(seed, x, amp_max=0.1)
    return b - b.min()


@pytest.mark.parametrize("bc", [oracle.BC_PERIODIC, oracle.BC_TRANSMISSIVE])
def test_stage_adjoint_matches_finite_differences(bc):
    n, dx, lam, tau = 64, 0.1, 300.0, 0.004
    rng = np.random.default_rng(11 + bc)
    b = bottom(n, dx)
    Ub = inputs.random_state(101, n, dx)
    Ul = inputs.random_state(102, n, dx, h_var=0.1)
    Ub = (Ub[0] - 0.5 * b, Ub[1], Ub[2], Ub[3])
    Ul = (Ul[0] - 0.5 * b, Ul[1], Ul[2], Ul[3])
    s0 = 0.37
    W = [rng.normal(size=n) for _ in range(4)]  # J = sum_k W_k . S_k

    def J(ub, ul, bb, s):
        p = oracle.Params(n, dx, bc, lam=lam, form=1, bathy=bb, speed=s)
        out = oracle.stage(p, ub, ul, tau)
        return sum(float(np.dot(W[k], out[k])) for k in range(4))

    p = oracle.Params(n, dx, bc, lam=lam, form=1, bathy=b, speed=s0)
    Ab, Al, gb, gs = oracle.stage_adjoint(p, Ub, Ul, tau, W)
    eps = 1e-6
    for trial in range(3):
        vb = [0.05 * smooth(rng, n) for _ in range(4)]
        vl = [0.05 * smooth(rng, n) for _ in range(4)]
        vbb = 0.05 * smooth(rng, n)
        # base state
        fd = (J([Ub[k] + eps * vb[k] for k in range(4)], Ul, b, s0)
              - J([Ub[k] - eps * vb[k] for k in range(4)], Ul, b, s0)) / (2 * eps)
        ad = sum(float(np.dot(Ab[k], vb[k])) for k in range(4))
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), ("base", fd, ad)
        # linearisation state
        fd = (J(Ub, [Ul[k] + eps * vl[k] for k in range(4)], b, s0)
              - J(Ub, [Ul[k] - eps * vl[k] for k in range(4)], b, s0)) / (2 * eps)
        ad = sum(float(np.dot(Al[k], vl[k])) for k in range(4))
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), ("lin", fd, ad)
        # bottom
        fd = (J(Ub, Ul, b + eps * vbb, s0) - J(Ub, Ul, b - eps * vbb, s0)) / (2 * eps)
        ad = float(np.dot(gb, vbb))
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), ("bottom", fd, ad)
    fd = (J(Ub, Ul, b, s0 + eps) - J(Ub, Ul, b, s0 - eps)) / (2 * eps)
    assert abs(fd - gs) <= 1e-6 * max(1.0, abs(gs)), ("speed", fd, gs)


def gauge_case(n=64, steps=25, lam=100.0, seed=5):
    # a short periodic domain (6.4): bottoms of low bumps that stay below the clip
    dx = 0.1
    x, _ = inputs.cell_centres(n, 0.0, n * dx)
    b = 0.5 * bottom(n, dx, seed)
    # crest off the cell symmetry: max |u| (the Rusanov speed) has one argmax,
    # where the speed is differentiable
    U = inputs.wave_over_bottom(x, b, 1.0, 0.1, 0.5 * n * dx + 0.037, period=n * dx)
    p = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 2.0, 0.5)
    cells = [5, 20, 33, 47, 60]
    # data: the same run over a different bottom
    b2 = 0.5 * bottom(n, dx, seed + 1)
    assert np.max(np.abs(b - b2)) > 1e-3
    p2 = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=lam, form=1, bathy=b2)
    V, data = U, []
    for _ in range(steps):
        V = oracle.step(p2, V, dt)
        data.append(V[0][cells])
    return p, U, b, dt, steps, cells, np.array(data)


def run_misfit(p, U, dt, steps, cells, data):
    V, hs = U, []
    for _ in range(steps):
        V = oracle.step(p, V, dt)
        hs.append(V[0])
    return oracle.misfit(hs, cells, data, dt)


def test_run_adjoint_matches_finite_differences():
    p, U, b, dt, steps, cells, data = gauge_case()
    J, g, gb, _ = oracle.adjoint(p, U, dt, steps, cells, data)
    assert J > 0
    assert abs(J - run_misfit(p, U, dt, steps, cells, data)) <= 1e-13 * J
    rng = np.random.default_rng(2)
    eps = 1e-6  # with unit directions: truncation ~eps^2, rounding ~1e-16/eps
    n = p.n
    for trial in range(3):
        # initial state, all four variables
        v = [smooth(rng, n) for _ in range(4)]
        Jp = run_misfit(p, [U[k] + eps * v[k] for k in range(4)], dt, steps, cells, data)
        Jm = run_misfit(p, [U[k] - eps * v[k] for k in range(4)], dt, steps, cells, data)
        ad = sum(float(np.dot(g[k], v[k])) for k in range(4))
        assert abs((Jp - Jm) / (2 * eps) - ad) <= 1e-6 * abs(ad), ((Jp - Jm) / (2 * eps), ad)
        # bottom
        vb = smooth(rng, n)
        pp = oracle.Params(n, p.dx, p.bc, lam=p.lam, form=1, bathy=b + eps * vb)
        pm = oracle.Params(n, p.dx, p.bc, lam=p.lam, form=1, bathy=b - eps * vb)
        fd = (run_misfit(pp, U, dt, steps, cells, data) - run_misfit(pm, U, dt, steps, cells, data)) / (2 * eps)
        ad = float(np.dot(gb, vb))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_adjoint_of_a_lake_at_rest_with_matching_data_is_zero():
    # data equal to the forward run's own gauge depths: J = 0 and the gradient vanishes
    n, dx = 48, 0.1
    b = bottom(n, dx)
    h = 1.0 - b
    U = (h, 0 * h, h * h, 0 * h)
    p = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=100.0, form=1, bathy=b)
    cells = [3, 17, 30]
    data = np.tile(h[cells], (6, 1))
    J, g, gb, _ = oracle.adjoint(p, U, 0.02, 6, cells, data)
    assert J < 1e-26
    assert max(np.max(np.abs(x)) for x in g) < 1e-12 and np.max(np.abs(gb)) < 1e-12
