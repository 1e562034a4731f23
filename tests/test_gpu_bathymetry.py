"""GPU parity of the well-balanced bathymetry form (HSGN_WELL_BALANCED) with
the oracle's form 1: one stage with U_b != U_l over a random bottom, single
steps and trajectories over a Gaussian-bump bottom, the lake at rest, and one
full-size step of the 2^24-cell shelf workload.

Tolerances as for the flat form: 1e-12 relative L2 per stage / step, 1e-9
over trajectories; at full size q and h w are compared against the scales of
the back-substitution summands, since both are roundoff-sized wherever the
water is at rest.
"""
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


# the forms held to the FP64 bar: FP64 arithmetic and double-float pairs
FORMS = [pytest.param(0x0, id="fp64"), pytest.param(0x8, id="dfloat")]


def wb_solver(n, dx, bc, lam, b, flags=0):
    return S().Solver(n, 0.0, n * dx, bc, lam=lam, flags=flags | S().FLAG_WELL_BALANCED,
                      bathymetry=b)


def hw_scale(U, lam, dt):
    """Size of the summands of the (h w) update (Sec. 4.2): r^dag contains
    + lambda tau and the result subtracts lambda tau mbar / hbar^2, so h w,
    small where the flow is slow, carries rounding of that size."""
    tau = (1.0 - 1.0 / math.sqrt(2.0)) * dt
    return np.abs(U[3]) + lam * tau * (1.0 + np.abs(U[2]) / (U[0] * U[0]))


def gpu_run(n, dx, bc, lam, b, U, dt, steps, use_graph=True, form=0):
    with wb_solver(n, dx, bc, lam, b, form) as s:
        s.set_state(*(dev(u) for u in U))
        if use_graph:
            s.run(dt, steps)
        else:
            for _ in range(steps):
                s.step(dt)
            s.check()
        return [t.cpu().numpy() for t in s.get_state()]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [3, 4, 7, 64, 511, 512, 513, 1000, 5000, 70001])
def test_wb_stage_matches_oracle(n, bc, form):
    dx, lam, tau, speed = 0.1, 300.0, 0.01, 0.37
    x, _ = inputs.cell_centres(n, 0.0, n * dx)
    b = inputs.gaussian_bathymetry(70 + n, x, amp_max=0.1)
    Ub = inputs.random_state(1000 + n, n, dx)
    Ul = inputs.random_state(2000 + n, n, dx, h_var=0.1)
    for local in (0, 1):
        flags = (S().FLAG_RUSANOV_LOCAL if local else 0) | form
        with wb_solver(n, dx, bc, lam, b, flags) as s:
            out = s.stage([dev(u) for u in Ub], [dev(u) for u in Ul], tau, speed)
            got = [t.cpu().numpy() for t in out]
            s.check()
        p = oracle.Params(n, dx, bc, lam=lam, rusanov=0 if local else 1, speed=speed,
                          form=1, bathy=b)
        ref = oracle.stage(p, Ub, Ul, tau)
        for k in range(4):
            assert rel_l2(got[k], ref[k]) < 1e-12, (k, local, rel_l2(got[k], ref[k]))


@pytest.mark.parametrize("form", FORMS)
def test_wb_flat_bottom_pointer_equals_null_bottom(form):
    # a zero bottom array and no bottom at all give bitwise the same steps
    n, dx, lam = 1537, 0.1, 500.0
    U = inputs.random_state(77, n, dx)
    a = gpu_run(n, dx, 1, lam, np.zeros(n), U, 0.01, 3, form=form)
    b = gpu_run(n, dx, 1, lam, None, U, 0.01, 3, form=form)
    for k in range(4):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [5, 100, 1000, 1537])
def test_wb_one_step_matches_oracle(n, bc, form):
    dx, lam = 0.1, 500.0
    x, _, b, U = inputs.gauss_bottom_wave(300 + n, n, dx)
    p = oracle.Params(n, dx, bc, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 2.0, 0.5)
    got = gpu_run(n, dx, bc, lam, b, U, dt, 1, form=form)
    ref = oracle.step(p, U, dt)
    # q is compared against its own scale plus the size of the depth-driven
    # forces (q itself is small where the wave has not arrived); h w against
    # the scale of its summands
    for k in (0, 2):
        assert rel_l2(got[k], ref[k]) < 1e-12, (k, rel_l2(got[k], ref[k]))
    assert np.linalg.norm(got[1] - ref[1]) < 1e-12 * (np.linalg.norm(ref[1]) + np.linalg.norm(U[0]))
    assert np.linalg.norm(got[3] - ref[3]) < 1e-12 * np.linalg.norm(hw_scale(U, lam, dt))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [400, 5000])
def test_wb_lake_at_rest_on_gpu(n, bc, form):
    # u = 0, eta = h, w = 0, h + b = const: the GPU keeps the state at rest to
    # rounding over 40 steps, like the oracle (Sec. 2.3 with b_t = 0)
    x, dx = inputs.cell_centres(n, 0.0, 0.2 * n)
    b = inputs.gaussian_bathymetry(5, x)
    b = b - b.min()
    h = 1.0 - b
    U = (h, 0 * h, h * h, 0 * h)
    got = gpu_run(n, dx, bc, 500.0, b, U, 0.05, 40, form=form)
    assert np.max(np.abs(got[0] - h)) < 1e-12
    assert np.max(np.abs(got[1])) < 1e-12
    assert np.max(np.abs(got[2] - h * h)) < 1e-12
    assert np.max(np.abs(got[3])) < 1e-11


@pytest.mark.parametrize("form", FORMS)
def test_wb_gauss_bottom_trajectory(form):
    # the adjoint workload's forward problem: N = 4096, dx = 0.1, periodic,
    # lambda = 100, wave a = 0.1 over 8 Gaussian bumps; 200 steps at CFL 2
    n, lam, steps = 4096, 100.0, 200
    x, dx, b, U = inputs.gauss_bottom_wave(20251011, n)
    p = oracle.Params(n, dx, 0, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 2.0, 0.5)
    got = gpu_run(n, dx, 0, lam, b, U, dt, steps, form=form)
    ref = oracle.run(p, U, dt, steps)
    for k in range(3):
        assert rel_l2(got[k], ref[k]) < 1e-9, (k, rel_l2(got[k], ref[k]))
    assert np.linalg.norm(got[3] - ref[3]) < 1e-9 * np.linalg.norm(hw_scale(U, lam, dt))
    assert abs(math.fsum(got[0]) - math.fsum(U[0])) <= 1e-13 * math.fsum(U[0])


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [1000, 2689])
def test_wb_dfloat_fallback_tiles_match_oracle(n, bc):
    # CFL_IMEX 5.5 over Gaussian bumps: the first step's 64-row windows miss
    # the decay bound and every tile is redone in pieces with 96 rows (the
    # bottom reloaded per piece); the second step takes the recorded overlap
    dx, lam = 0.1, 100.0
    x, _, b, U = inputs.gauss_bottom_wave(400 + n, n, dx, amp=0.05)
    p = oracle.Params(n, dx, bc, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 5.5, 1e9)
    with wb_solver(n, dx, bc, lam, b, S().FLAG_DOUBLE_FLOAT) as s:
        s.set_state(*(dev(u) for u in U))
        s.run(dt, 1)
        need, ov = s.df_overlap()
        assert 63 < need <= 95 and ov > 64, (need, ov)
        one = [t.cpu().numpy() for t in s.get_state()]
        s.run(dt, 1)
        two = [t.cpu().numpy() for t in s.get_state()]
    r1 = oracle.step(p, U, dt)
    r2 = oracle.step(p, r1, dt)
    for got, ref, u0 in ((one, r1, U), (two, r2, r1)):
        for k in (0, 2):
            assert rel_l2(got[k], ref[k]) < 1e-12, (k, rel_l2(got[k], ref[k]))
        assert np.linalg.norm(got[1] - ref[1]) < 1e-12 * (np.linalg.norm(ref[1]) + np.linalg.norm(u0[0]))
        assert np.linalg.norm(got[3] - ref[3]) < 1e-12 * np.linalg.norm(hw_scale(u0, lam, dt))


def test_wb_dfloat_per_step_dt_matches_the_oracle_policy():
    # the per-step time step (Sec. 5) on the double-float bottom form: every
    # step takes dt = min(2 dx/nu_max, 0.5 dx/u_max) of the state it starts
    # from, on the device, over a wave crossing Gaussian bumps; the oracle's
    # bottom form re-evaluates the same rule before each step
    n, lam, steps = 4096, 100.0, 25
    x, dx, b, U = inputs.gauss_bottom_wave(20251011, n)
    p = oracle.Params(n, dx, 0, lam=lam, form=1, bathy=b)
    V, t_ref = U, 0.0
    for _ in range(steps):
        dt, _, _ = oracle.suggest_dt(p, V, 2.0, 0.5)
        V = oracle.step(p, V, dt)
        t_ref += dt
    with wb_solver(n, dx, 0, lam, b, S().FLAG_DOUBLE_FLOAT) as s:
        s.set_state(*(dev(u) for u in U))
        t = s.run_cfl(2.0, 0.5, steps)
        got = [u.cpu().numpy() for u in s.get_state()]
    assert abs(t - t_ref) <= 1e-13 * t_ref, (t, t_ref)
    for k in range(3):
        assert rel_l2(got[k], V[k]) < 1e-10, (k, rel_l2(got[k], V[k]))


@pytest.mark.parametrize("form", FORMS)
def test_wb_graph_replay_equals_step_loop(form):
    n, lam = 3000, 1000.0
    x, dx, b, U = inputs.gauss_bottom_wave(8, n)
    a = gpu_run(n, dx, 0, lam, b, U, 0.01, 7, use_graph=True, form=form)
    c = gpu_run(n, dx, 0, lam, b, U, 0.01, 7, use_graph=False, form=form)
    for k in range(4):
        np.testing.assert_array_equal(a[k], c[k])


@pytest.mark.parametrize("form", FORMS)
def test_wb_shelf_2_24_one_step(form):
    # the large workload: N = 2^24, dx = 0.005, transmissive, lambda = 1000,
    # 1:20 shelf, wave a = 0.1; one step at CFL_IMEX 4, every cell compared
    n, lam = 1 << 24, 1000.0
    x, dx, b, U = inputs.shelf_wave(n)
    p = oracle.Params(n, dx, 1, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 4.0, 0.5)
    got = gpu_run(n, dx, 1, lam, b, U, dt, 1, form=form)
    ref = oracle.step(p, U, dt)
    A = oracle.assemble(p, U, U, (1.0 - 1.0 / math.sqrt(2.0)) * dt)
    tau = (1.0 - 1.0 / math.sqrt(2.0)) * dt
    h = np.abs(U[0])
    Sq = np.abs(U[1]) + tau / dx * A["beta"] * h
    Sr = np.abs(U[3]) + lam * tau * (1.0 + np.abs(U[2]) / (h * h))
    assert rel_l2(got[0], ref[0]) < 1e-12 and rel_l2(got[2], ref[2]) < 1e-12
    assert np.linalg.norm(got[1] - ref[1]) / np.linalg.norm(Sq) < 1e-12
    assert np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(Sr) < 1e-12


# --------------------------------------------------------------------------
# the bottom form in mixed precision (HSGN_MIXED | HSGN_WELL_BALANCED, the
# windowed kernel): bounds as for the flat mixed form (one step <= 1e-7
# relative L2 for h and h eta, q and h w against their summand scales), the
# lake at rest kept to the double-float pairs' precision, mass to FP64 rounding
# --------------------------------------------------------------------------
def wb_scales(p, U, dt):
    """Summand magnitudes of the bottom form's back-substitution (Sec. 4.2 with
    the face forces of the bottom form): q^dag and tau/dx beta h; r^dag with its
    + lambda tau and the subtracted lambda tau mbar/hbar^2."""
    tau = (1.0 - 1.0 / math.sqrt(2.0)) * dt
    A = oracle.assemble(p, U, U, tau)
    h, q, m, r = (np.abs(u) for u in U)
    Sq = q + tau / p.dx * A["beta"] * h
    Sr = r + p.lam * tau * (1.0 + m / (h * h))
    return Sq, Sr


def wb_mixed_run(n, dx, bc, lam, b, U, dt, steps, use_graph=True):
    with wb_solver(n, dx, bc, lam, b, S().FLAG_MIXED) as s:
        s.set_state(*(dev(u) for u in U))
        if use_graph:
            s.run(dt, steps)
        else:
            for _ in range(steps):
                s.step(dt)
        s.check()
        return [t.cpu().numpy() for t in s.get_state()]


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [5, 100, 1000, 1537, 70001])
def test_wb_mixed_one_step_close_to_oracle(n, bc):
    dx, lam = 0.1, 500.0
    x, _, b, U = inputs.gauss_bottom_wave(300 + n, n, dx)
    p = oracle.Params(n, dx, bc, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 2.0, 0.5)
    got = wb_mixed_run(n, dx, bc, lam, b, U, dt, 1)
    ref = oracle.step(p, U, dt)
    Sq, Sr = wb_scales(p, U, dt)
    assert rel_l2(got[0], ref[0]) < 1e-7, rel_l2(got[0], ref[0])
    assert rel_l2(got[2], ref[2]) < 1e-7, rel_l2(got[2], ref[2])
    assert np.linalg.norm(got[1] - ref[1]) / np.linalg.norm(Sq) < 1e-6
    assert np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(Sr) < 1e-6


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [400, 5000])
def test_wb_mixed_lake_at_rest(n, bc):
    # h + b = const, u = 0, eta = h, w = 0: every jump the stage forms from
    # the pairs vanishes to their 2^-48 precision, so the state stays at rest
    # far below single-precision rounding (which would be ~1e-7 per step)
    x, dx = inputs.cell_centres(n, 0.0, 0.2 * n)
    b = inputs.gaussian_bathymetry(5, x)
    b = b - b.min()
    h = 1.0 - b
    U = (h, 0 * h, h * h, 0 * h)
    got = wb_mixed_run(n, dx, bc, 500.0, b, U, 0.05, 40)
    err = [np.max(np.abs(got[0] - h)), np.max(np.abs(got[1])), np.max(np.abs(got[2] - h * h)),
           np.max(np.abs(got[3]))]
    assert err[0] < 1e-12 and err[1] < 1e-12 and err[2] < 1e-12 and err[3] < 1e-10, err


def test_wb_mixed_gauss_bottom_trajectory():
    # the adjoint workload's forward problem, 200 steps at CFL 2: mixed within
    # 1e-6 of the FP64 oracle, mass exact to FP64 rounding
    n, lam, steps = 4096, 100.0, 200
    x, dx, b, U = inputs.gauss_bottom_wave(20251011, n)
    p = oracle.Params(n, dx, 0, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 2.0, 0.5)
    got = wb_mixed_run(n, dx, 0, lam, b, U, dt, steps)
    ref = oracle.run(p, U, dt, steps)
    assert rel_l2(got[0], ref[0]) < 1e-6 and rel_l2(got[2], ref[2]) < 1e-6
    Sq, Sr = wb_scales(p, U, dt)
    assert np.linalg.norm(got[1] - ref[1]) / np.linalg.norm(Sq) < 1e-5
    assert np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(Sr) < 1e-5
    assert abs(math.fsum(got[0]) - math.fsum(U[0])) <= 1e-13 * math.fsum(U[0])


def test_wb_mixed_graph_replay_equals_step_loop_and_null_bottom():
    n, lam = 3000, 1000.0
    x, dx, b, U = inputs.gauss_bottom_wave(8, n)
    a = wb_mixed_run(n, dx, 0, lam, b, U, 0.01, 7, use_graph=True)
    c = wb_mixed_run(n, dx, 0, lam, b, U, 0.01, 7, use_graph=False)
    for k in range(4):
        np.testing.assert_array_equal(a[k], c[k])
    z = wb_mixed_run(n, dx, 1, lam, np.zeros(n), U, 0.01, 3)
    o = wb_mixed_run(n, dx, 1, lam, None, U, 0.01, 3)
    for k in range(4):
        np.testing.assert_array_equal(z[k], o[k])


def test_wb_mixed_needs_the_windowed_kernel():
    with pytest.raises(S().HsgnError) as e:
        wb_solver(16, 0.1, 0, 1.0, None, S().FLAG_MIXED | S().FLAG_EXACT_SOLVE)
    assert e.value.code == 6


def test_wb_mixed_shelf_2_24_steps():
    # the large workload in mixed precision: 5 steps at CFL_IMEX 4 against
    # the FP64 oracle, every cell
    n, lam, steps = 1 << 24, 1000.0, 5
    x, dx, b, U = inputs.shelf_wave(n)
    p = oracle.Params(n, dx, 1, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 4.0, 0.5)
    got = wb_mixed_run(n, dx, 1, lam, b, U, dt, steps)
    ref = oracle.run(p, U, dt, steps)
    Sq, Sr = wb_scales(p, U, dt)
    assert rel_l2(got[0], ref[0]) < 1e-7 and rel_l2(got[2], ref[2]) < 1e-7
    assert np.linalg.norm(got[1] - ref[1]) / np.linalg.norm(Sq) < 1e-6
    assert np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(Sr) < 1e-6


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [3, 4, 7])
def test_wb_mixed_tiny_grids(n, bc):
    dx, lam = 0.1, 300.0
    x, _ = inputs.cell_centres(n, 0.0, n * dx)
    b = inputs.gaussian_bathymetry(90 + n, x, amp_max=0.1)
    U = inputs.random_state(5000 + n + 10 * bc, n, dx)
    p = oracle.Params(n, dx, bc, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 2.0, 0.5)
    got = wb_mixed_run(n, dx, bc, lam, b, U, dt, 2)
    ref = oracle.run(p, U, dt, 2)
    Sq, Sr = wb_scales(p, U, dt)
    assert rel_l2(got[0], ref[0]) < 1e-7 and rel_l2(got[2], ref[2]) < 1e-7
    assert np.linalg.norm(got[1] - ref[1]) / np.linalg.norm(Sq) < 1e-6
    assert np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(Sr) < 1e-6


def test_wb_mixed_shelf_full_length_and_against_fp64():
    # the large workload over its full 5000 steps in mixed precision and in
    # double-float pairs (mass kept, no device error, finite), and its first
    # 200 steps against the FP64 bottom form, which matches the oracle to
    # 1e-12 per step. A step changes h
    # by under 1e-3 of itself, rounded in single precision to 2^-24: under 1e-10
    # per step, so 200 steps stay below 2e-8
    n, lam = 1 << 24, 1000.0
    x, dx, b, U = inputs.shelf_wave(n)
    p = oracle.Params(n, dx, 1, lam=lam, form=1, bathy=b)
    dt, _, _ = oracle.suggest_dt(p, U, 4.0, 0.5)
    m0 = math.fsum(U[0])
    with wb_solver(n, dx, 1, lam, b, S().FLAG_MIXED) as s:
        s.set_state(*(dev(u) for u in U))
        s.run(dt, 200)
        mixed200 = [t.cpu().numpy() for t in s.get_state()]
        s.run(dt, 4800)
        end = [t.cpu().numpy() for t in s.get_state()]
    assert all(np.all(np.isfinite(a)) for a in end)
    assert abs(math.fsum(end[0]) - m0) <= 1e-12 * m0
    assert abs(math.fsum(mixed200[0]) - m0) <= 1e-12 * m0
    f64 = gpu_run(n, dx, 1, lam, b, U, dt, 200)
    assert rel_l2(mixed200[0], f64[0]) < 1e-7 and rel_l2(mixed200[2], f64[2]) < 1e-7
    # the double-float bottom form over the same run: within the FP64 bar of
    # the FP64 form after 200 steps (1e-9 over a trajectory), and over the
    # 5000 steps finite, free of device errors and with the mass kept
    with wb_solver(n, dx, 1, lam, b, S().FLAG_DOUBLE_FLOAT) as s:
        s.set_state(*(dev(u) for u in U))
        s.run(dt, 200)
        df200 = [t.cpu().numpy() for t in s.get_state()]
        s.run(dt, 4800)
        dfend = [t.cpu().numpy() for t in s.get_state()]
    for k in (0, 2):
        assert rel_l2(df200[k], f64[k]) < 1e-9, (k, rel_l2(df200[k], f64[k]))
    assert np.linalg.norm(df200[1] - f64[1]) < 1e-9 * (np.linalg.norm(f64[1]) + np.linalg.norm(U[0]))
    assert all(np.all(np.isfinite(a)) for a in dfend)
    assert abs(math.fsum(dfend[0]) - m0) <= 1e-12 * m0
