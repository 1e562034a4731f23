"""GPU parity of the discrete adjoint (hsgn_adjoint) with the oracle's
adjoint, its independence of the checkpoint interval, finite differences of
the GPU misfit on the adjoint workload (N = 4096, 2000 steps, 5 gauges), and
the torch.autograd.Function built on it."""
import math

import numpy as np
import pytest

import oracle
from paper_2510_07539_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_07539_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def S():
    from paper_2510_07539_gb300 import solver
    return solver


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def small_bottom(n, dx, seed):
    x, _ = inputs.cell_centres(n, 0.0, n * dx)
    b = inputs.gaussian_bathymetry(seed, x, amp_max=0.1)
    return 0.5 * (b - b.min())


def small_case(bc, n=64, steps=25, lam=100.0):
    dx = 0.1
    x, _ = inputs.cell_centres(n, 0.0, n * dx)
    b = small_bottom(n, dx, 5)
    U = inputs.wave_over_bottom(x, b, 1.0, 0.1, 0.5 * n * dx + 0.037, period=n * dx)
    p = oracle.Params(n, dx, bc, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 2.0, 0.5)
    cells = [5, 20, 33, 47, 60]
    p2 = oracle.Params(n, dx, bc, lam=lam, form=1, bathy=small_bottom(n, dx, 6))
    V, data = U, []
    for _ in range(steps):
        V = oracle.step(p2, V, dt)
        data.append(V[0][cells])
    return p, U, b, dt, steps, cells, np.array(data)


def gpu_adjoint(p, U, b, dt, steps, cells, data, K=100):
    with S().Solver(p.n, 0.0, p.n * p.dx, p.bc, lam=p.lam, flags=S().FLAG_WELL_BALANCED,
                    bathymetry=b) as s:
        s.set_state(*(dev(u) for u in U))
        J, g, gb = s.adjoint(dt, steps, cells, data, checkpoint_every=K)
        final = [t.cpu().numpy() for t in s.get_state()]
    return J, [t.cpu().numpy() for t in g], gb.cpu().numpy(), final


@pytest.mark.parametrize("bc", [oracle.BC_PERIODIC, oracle.BC_TRANSMISSIVE])
def test_adjoint_matches_oracle(bc):
    p, U, b, dt, steps, cells, data = small_case(bc)
    J, g, gb, final = gpu_adjoint(p, U, b, dt, steps, cells, data, K=7)
    Jr, gr, gbr, Ur = oracle.adjoint(p, U, dt, steps, cells, data)
    assert abs(J - Jr) <= 1e-11 * Jr
    for k in range(4):
        assert rel_l2(g[k], gr[k]) < 1e-9, (k, rel_l2(g[k], gr[k]))
    assert rel_l2(gb, gbr) < 1e-9, rel_l2(gb, gbr)
    for k in range(4):
        assert rel_l2(final[k], Ur[k]) < 1e-12 or np.max(np.abs(final[k] - Ur[k])) < 1e-13


def test_adjoint_independent_of_checkpoint_interval():
    p, U, b, dt, steps, cells, data = small_case(oracle.BC_PERIODIC)
    ref = gpu_adjoint(p, U, b, dt, steps, cells, data, K=steps)
    for K in (1, 4, 11):
        got = gpu_adjoint(p, U, b, dt, steps, cells, data, K=K)
        assert abs(got[0] - ref[0]) <= 1e-13 * ref[0]
        for k in range(4):
            assert rel_l2(got[1][k], ref[1][k]) < 1e-12
        assert rel_l2(got[2], ref[2]) < 1e-12


def test_adjoint_workload_finite_differences():
    # the adjoint workload: N = 4096, dx = 0.1, periodic, lambda = 100, a wave
    # a = 0.1 over 8 Gaussian bumps; 2000 steps at CFL_IMEX 2, 5 equispaced
    # gauges, data from the same run over a bottom of another seed;
    # checkpoints every 100 steps
    n, steps, lam = 4096, 2000, 100.0
    x, dx, b, U = inputs.gauss_bottom_wave(inputs.SEED_BASE + 4, n)
    U = inputs.wave_over_bottom(x, b, 1.0, 0.1, 0.5 * n * dx + 0.037, period=n * dx)
    b2 = inputs.gauss_bottom_wave(inputs.SEED_BASE + 5, n)[2]
    p = oracle.Params(n, dx, 0, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 2.0, 0.5)
    cells = [int(n * (k + 0.5) / 5) for k in range(5)]
    with S().Solver(n, 0.0, n * dx, 0, lam=lam, flags=S().FLAG_WELL_BALANCED,
                    bathymetry=b2) as s:
        s.set_state(*(dev(u) for u in U))
        hs = []
        for _ in range(steps):
            s.step(dt)
            hs.append(s.get_state()[0][cells].cpu().numpy())
    data = np.array(hs)
    J, g, gb, _ = gpu_adjoint(p, U, b, dt, steps, cells, data, K=100)
    assert J > 0
    rng = np.random.default_rng(3)
    eps = 1e-6
    zero = np.zeros((steps, len(cells)))

    def misfit(bb, UU):
        with S().Solver(n, 0.0, n * dx, 0, lam=lam, flags=S().FLAG_WELL_BALANCED,
                        bathymetry=bb) as s:
            s.set_state(*(dev(u) for u in UU))
            Jv, _, _ = s.adjoint(dt, steps, cells, data, checkpoint_every=steps)
        return Jv

    def smooth():
        f = np.zeros(n)
        for k in range(1, 6):
            a_, b_ = rng.normal(size=2) / k
            f += a_ * np.cos(2 * np.pi * k * x / (n * dx)) + b_ * np.sin(2 * np.pi * k * x / (n * dx))
        return f / np.max(np.abs(f))

    vb = smooth()
    fd = (misfit(b + eps * vb, U) - misfit(b - eps * vb, U)) / (2 * eps)
    ad = float(np.dot(gb, vb))
    assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
    vh = smooth()
    fd = (misfit(b, (U[0] + eps * vh, U[1], U[2], U[3])) -
          misfit(b, (U[0] - eps * vh, U[1], U[2], U[3]))) / (2 * eps)
    ad = float(np.dot(g[0], vh))
    assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
    del zero


def test_autograd_function_and_gradcheck():
    n, dx, lam, steps = 24, 0.1, 100.0, 3
    x, _ = inputs.cell_centres(n, 0.0, n * dx)
    b0 = small_bottom(n, dx, 7)
    U = inputs.wave_over_bottom(x, b0, 1.0, 0.1, 0.5 * n * dx + 0.037, period=n * dx)
    cells = [3, 11, 19]
    data = np.full((steps, 3), 0.95)
    dt = 0.01
    args = [dev(u).requires_grad_(True) for u in U] + [dev(b0).requires_grad_(True)]
    J = S().GaugeMisfit.apply(*args, 0.0, n * dx, 0, lam, dt, steps, cells, data, 2)
    J.backward()
    with S().Solver(n, 0.0, n * dx, 0, lam=lam, flags=S().FLAG_WELL_BALANCED, bathymetry=b0) as s:
        s.set_state(*(dev(u) for u in U))
        Jd, g, gb = s.adjoint(dt, steps, cells, data, checkpoint_every=2)
    assert abs(float(J.detach()) - Jd) <= 1e-14 * Jd
    for k in range(4):
        assert torch.equal(args[k].grad, g[k])
    assert torch.equal(args[4].grad, gb)

    def f(h, q, m, r, b):
        return S().GaugeMisfit.apply(h, q, m, r, b, 0.0, n * dx, 0, lam, dt, steps, cells, data, 2)

    inp = tuple(dev(u).requires_grad_(True) for u in U) + (dev(b0).requires_grad_(True),)
    assert torch.autograd.gradcheck(f, inp, eps=1e-6, atol=1e-7, rtol=1e-5)
