"""GPU parity of the comparison schemes (FP64 form) with the oracle: the
textbook ARS(2,2,2) tableau, the first-order semi-implicit step and the
explicit hSGN scheme with forward Euler or Heun's method (HSGN_SCHEME_*).
Tolerances as for the paper's scheme: 1e-12 relative L2 per step, 1e-9 over
trajectories, mass to 1e-13."""
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


# GPU scheme flag -> (oracle scheme, oracle reconstruction, CFL used in the tests)
SCHEMES = {
    "ars222": (0x100, oracle.SCHEME_ARS222, 1, 2.0),
    "si1": (0x200, oracle.SCHEME_SI1, 0, 2.0),
    "heun": (0x300, oracle.SCHEME_EX_HEUN, 1, 0.4),
    "euler": (0x400, oracle.SCHEME_EX_EULER, 0, 0.2),
}


def gpu_run(name, n, dx, bc, lam, U, dt, steps, use_graph=True, extra=0):
    flag = SCHEMES[name][0] | extra
    with S().Solver(n, 0.0, n * dx, bc, lam=lam, flags=flag) as s:
        s.set_state(*(dev(u) for u in U))
        if use_graph:
            s.run(dt, steps)
        else:
            for _ in range(steps):
                s.step(dt)
            s.check()
        return [t.cpu().numpy() for t in s.get_state()]


def params(name, n, dx, bc, lam, **kw):
    _, sch, recon, _ = SCHEMES[name]
    return oracle.Params(n, dx, bc, lam=lam, scheme=sch, recon=recon, **kw)


@pytest.mark.parametrize("name", list(SCHEMES))
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [5, 100, 1000, 1537])
def test_scheme_one_step_matches_oracle(name, n, bc):
    dx, lam = 0.1, 500.0
    U = inputs.random_state(3100 + n, n, dx)
    p = params(name, n, dx, bc, lam)
    dt, _, _ = oracle.suggest_dt(p, U, SCHEMES[name][3], 0.5)
    got = gpu_run(name, n, dx, bc, lam, U, dt, 1)
    ref = oracle.step(p, U, dt)
    for k in range(4):
        assert rel_l2(got[k], ref[k]) < 1e-12, (name, k, rel_l2(got[k], ref[k]))


@pytest.mark.parametrize("name", list(SCHEMES))
def test_scheme_solitary_trajectory(name):
    n, lam = 1000, 100.0
    x, dx = inputs.cell_centres(n, -50.0, 50.0)
    U = inputs.solitary(x, 1.0, 0.2, 0.0, period=100.0)
    p = params(name, n, dx, 0, lam)
    dt, _, _ = oracle.suggest_dt(p, U, SCHEMES[name][3], 0.5)
    got = gpu_run(name, n, dx, 0, lam, U, dt, 100)
    ref = oracle.run(p, U, dt, 100)
    for k in range(4):
        assert rel_l2(got[k], ref[k]) < 1e-9, (name, k, rel_l2(got[k], ref[k]))
    assert abs(math.fsum(got[0]) - math.fsum(U[0])) <= 1e-13 * math.fsum(U[0])


def test_heun_local_speed_and_graph_replay():
    n, dx, lam = 2049, 0.1, 300.0
    U = inputs.random_state(77, n, dx)
    p = params("heun", n, dx, 1, lam, rusanov=0)
    dt, _, _ = oracle.suggest_dt(p, U, 0.4, 0.5)
    a = gpu_run("heun", n, dx, 1, lam, U, dt, 7, use_graph=True, extra=S().FLAG_RUSANOV_LOCAL)
    b = gpu_run("heun", n, dx, 1, lam, U, dt, 7, use_graph=False, extra=S().FLAG_RUSANOV_LOCAL)
    for k in range(4):
        np.testing.assert_array_equal(a[k], b[k])
    ref = oracle.run(p, U, dt, 7)
    for k in range(4):
        assert rel_l2(a[k], ref[k]) < 1e-11, (k, rel_l2(a[k], ref[k]))


def test_ars222_dam_break_full_size_one_step():
    n, dx, lam = 1 << 20, 0.05, 1000.0
    x, U = inputs.dam_break(n, dx, 1.2, 1.0, 5.0 / dx)
    p = params("ars222", n, dx, 1, lam)
    dt, _, _ = oracle.suggest_dt(p, U, 4.0, 0.5)
    got = gpu_run("ars222", n, dx, 1, lam, U, dt, 1)
    ref = oracle.step(p, U, dt)
    assert rel_l2(got[0], ref[0]) < 1e-12 and rel_l2(got[2], ref[2]) < 1e-12
    # q and h w are roundoff-sized at rest: compare against the state's scale
    assert np.linalg.norm(got[1] - ref[1]) < 1e-12 * np.linalg.norm(U[0])
    assert np.linalg.norm(got[3] - ref[3]) < 1e-12 * lam * dt * np.linalg.norm(U[0])
