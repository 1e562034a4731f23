"""Pins of the oracle's comparison schemes (CPU, no GPU).

The schemes next to the paper's IMEX tableau: the textbook three-stage
ARS(2,2,2) double tableau, the first-order semi-implicit step (one stage of
eq. (GN_hyp_eq_semi_fully_discrete) with tau = dt), and the explicit hSGN
scheme of Sec. 4.4, eq. (GN_hyp_eq_explicit), with forward Euler or Heun's
method. Pinned against:
  * the scalar split test equation, evaluated from each double Butcher
    tableau by the generic stage list of Sec. 3.2 written out here;
  * the continuous hSGN right-hand side, differentiated spectrally for a
    smooth periodic state (consistency order of the explicit operator);
  * temporal order at a fixed grid, the linear hSGN dispersion relation,
    exact mass conservation, constant states, and the SGN solitary wave.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2510_07539_gb300 import inputs

G = 9.81
GAM = 1.0 - 1.0 / math.sqrt(2.0)
DEL = 1.0 - 1.0 / (2.0 * GAM)

# double Butcher tableaux (explicit A, implicit A); U^{n+1} = last implicit stage
TABLEAUX = {
    oracle.SCHEME_PRINTED: (np.array([[0.0, 0.0], [1.0 / (2.0 * GAM), 0.0]]),
                            np.array([[GAM, 0.0], [1.0 - GAM, GAM]])),
    oracle.SCHEME_ARS222: (np.array([[0.0, 0.0, 0.0], [GAM, 0.0, 0.0], [DEL, 1.0 - DEL, 0.0]]),
                           np.array([[0.0, 0.0, 0.0], [0.0, GAM, 0.0], [0.0, 1.0 - GAM, GAM]])),
}


def stage_list_step(AE, AI, zE, zI):
    """One step of size 1 from y = 1 of y' = zE y + zI y by the generic stage
    list: Y_E^(i) = 1 + sum_{j<i} AE_ij K_j, Y_I^(i) = 1 + sum_{j<i} AI_ij K_j
    + AI_ii K_i, K_i = zE Y_E^(i) + zI Y_I^(i)."""
    s = AE.shape[0]
    K = np.zeros(s)
    YI = 1.0
    for i in range(s):
        YE = 1.0 + AE[i, :i] @ K[:i]
        rest = 1.0 + AI[i, :i] @ K[:i]
        K[i] = (zE * YE + zI * rest) / (1.0 - zI * AI[i, i])
        YI = rest + AI[i, i] * K[i]
    return YI


@pytest.mark.parametrize("scheme", [oracle.SCHEME_PRINTED, oracle.SCHEME_ARS222])
@pytest.mark.parametrize("zE,zI", [(0.3, -2.0), (-0.1, -50.0), (0.0, -1.0), (1.0, 0.0),
                                   (0.25, -0.25), (-0.7, -1e3)])
def test_imex_schemes_match_their_tableaux(scheme, zE, zI):
    AE, AI = TABLEAUX[scheme]
    r = oracle.imex_scalar(zE, zI, 1.0, 1.0, 1, scheme=scheme)
    assert abs(r - stage_list_step(AE, AI, zE, zI)) <= 1e-13 * max(1.0, abs(r))


@pytest.mark.parametrize("zE,zI", [(0.3, -2.0), (-0.1, -50.0), (1.0, 0.0), (0.25, -0.25)])
def test_one_step_schemes_match_their_definitions(zE, zI):
    z = zE + zI
    assert abs(oracle.imex_scalar(zE, zI, 1.0, 1.0, 1, scheme=oracle.SCHEME_SI1)
               - (1.0 + zE) / (1.0 - zI)) <= 1e-14 * max(1.0, abs(z))
    assert abs(oracle.imex_scalar(zE, zI, 1.0, 1.0, 1, scheme=oracle.SCHEME_EX_EULER)
               - (1.0 + z)) <= 1e-14 * max(1.0, abs(z))
    assert abs(oracle.imex_scalar(zE, zI, 1.0, 1.0, 1, scheme=oracle.SCHEME_EX_HEUN)
               - (1.0 + z + 0.5 * z * z)) <= 1e-14 * max(1.0, z * z)


@pytest.mark.parametrize("split", [0.0, 0.5, 1.0])
def test_ars222_second_order_and_stiff_decay(split):
    for z in (1e-1, 5e-2, 2.5e-2):
        r = oracle.imex_scalar(split * z, (1 - split) * z, 1.0, 1.0, 1, scheme=oracle.SCHEME_ARS222)
        assert abs(r - math.exp(z)) <= 0.5 * z ** 3
    assert abs(oracle.imex_scalar(0.0, -1e8, 1.0, 1.0, 1, scheme=oracle.SCHEME_ARS222)) < 1e-7


# --------------------------------------------------------------------------
# explicit operator against the continuous right-hand side
# --------------------------------------------------------------------------
def spectral_dx(f, length):
    k = 2 * math.pi * np.fft.rfftfreq(len(f), d=length / len(f))
    return np.fft.irfft(1j * k * np.fft.rfft(f), n=len(f))


def continuous_rhs(U, length, lam):
    """hSGN right-hand side (Sec. 2.2, eq. (hSGN_eq)) with p_x = a^2 h_x +
    lambda alpha (h eta)_x (eq. (eq:hSGN_px)), exact for a band-limited state."""
    h, q, m, r = U
    u, eta = q / h, m / h
    alpha = -(2 * eta / h - 1) / (3 * h)
    a2 = G * h + (lam / 3) * eta ** 2 / h ** 2 - lam * eta * alpha
    d = lambda f: spectral_dx(f, length)
    return (-d(q), -d(q * u) - a2 * d(h) - lam * alpha * d(m), -d(m * u) + r,
            -d(r * u) - lam * (m / h ** 2 - 1))


@pytest.mark.parametrize("recon,order,ns", [(1, 2.0, (64, 128, 256)), (0, 1.0, (256, 512, 1024))])
def test_explicit_rhs_converges_to_the_pde(recon, order, ns):
    # without reconstruction the O(dx) Rusanov term dominates only on finer grids
    length, lam = 40.0, 100.0
    errs = []
    for n in ns:
        dx = length / n
        U = inputs.random_state(31, n, dx, h_var=0.1, u_amp=0.3)
        umax = float(np.max(np.abs(U[1] / U[0])))
        p = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=lam, recon=recon, speed=umax)
        L = oracle.explicit_rhs(p, U)
        E = continuous_rhs(U, length, lam)
        errs.append(max(np.max(np.abs(L[k] - E[k])) for k in range(4)))
    rates = [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]
    assert all(order - 0.3 < r < order + 0.6 for r in rates), (errs, rates)


def test_explicit_rhs_is_zero_at_rest_and_conserves_mass():
    n, dx = 200, 0.1
    h = np.full(n, 1.3)
    U = (h, 0 * h, h * h, 0 * h)
    L = oracle.explicit_rhs(oracle.Params(n, dx, oracle.BC_TRANSMISSIVE, lam=500.0), U)
    for k in range(4):
        assert np.max(np.abs(L[k])) < 1e-13
    V = inputs.random_state(5, n, dx)
    L = oracle.explicit_rhs(oracle.Params(n, dx, oracle.BC_PERIODIC, lam=500.0, speed=0.4), V)
    assert abs(math.fsum(L[0])) < 1e-12


# --------------------------------------------------------------------------
# the schemes on hSGN
# --------------------------------------------------------------------------
@pytest.mark.parametrize("scheme,order,steps", [
    (oracle.SCHEME_ARS222, 2, (8, 16, 32)),
    (oracle.SCHEME_SI1, 1, (64, 128, 256)),
    (oracle.SCHEME_EX_HEUN, 2, (64, 128, 256)),
    (oracle.SCHEME_EX_EULER, 1, (64, 128, 256)),
])
def test_temporal_order(scheme, order, steps):
    n, dx = 128, 0.2
    U = inputs.random_state(21, n, dx, h_var=0.05, u_amp=0.1)
    p = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=100.0, scheme=scheme)
    T = 0.4
    ref = oracle.run(p, U, T / 8192, 8192)
    errs = []
    for s in steps:
        V = oracle.run(p, U, T / s, s)
        errs.append(max(np.max(np.abs(V[k] - ref[k])) for k in range(4)))
    rates = [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]
    assert all(order - 0.3 < r < order + 0.4 for r in rates), (errs, rates)


@pytest.mark.parametrize("scheme", [oracle.SCHEME_ARS222, oracle.SCHEME_SI1,
                                    oracle.SCHEME_EX_HEUN, oracle.SCHEME_EX_EULER])
def test_schemes_conserve_mass_and_constant_states(scheme):
    n, dx = 301, 0.1
    U = inputs.random_state(9, n, dx)
    p = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=300.0, scheme=scheme)
    V = oracle.run(p, U, 0.002, 20)
    assert abs(math.fsum(V[0]) - math.fsum(U[0])) <= 1e-13 * math.fsum(U[0])
    c = np.full(n, 0.8)
    C = (c, 0.3 * c, c * c, 0 * c)
    W = oracle.run(oracle.Params(n, dx, oracle.BC_TRANSMISSIVE, lam=300.0, scheme=scheme), C,
                   0.002, 5)
    for k in range(4):
        np.testing.assert_allclose(W[k], C[k], rtol=0, atol=1e-13)


def slow_branch(k, h0, lam):
    A = h0 * h0
    B = -(lam + G * h0 ** 3 * k * k + (lam / 3.0) * k * k * h0 * h0)
    C = G * h0 * lam * k * k
    return math.sqrt((-B - math.sqrt(B * B - 4 * A * C)) / (2 * A))


def measured_omega(n, lam, scheme, cfl, h0=1.0, length=20.0, periods=0.5, eps=1e-6):
    """Phase speed of a small linear wave (small root of the hSGN dispersion
    relation, derived from eq. (hSGN_eq)) measured from the first Fourier mode."""
    dx = length / n
    x = (np.arange(n) + 0.5) * dx
    k = 2 * math.pi / length
    wp = slow_branch(k, h0, lam)
    eta_hat = lam * eps / (lam - wp * wp * h0 * h0)
    th = k * x
    h = h0 + eps * np.cos(th)
    u = (wp * eps / (k * h0)) * np.cos(th)
    eta = h0 + eta_hat * np.cos(th)
    w = eta_hat * wp * np.sin(th)
    U = (h, h * u, h * eta, h * w)
    p = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=lam, scheme=scheme)
    nu = math.sqrt(G * h0 + lam / 3.0)
    T = periods * 2 * math.pi / wp
    steps = max(4, int(math.ceil(T / (cfl * dx / nu))))
    dt = T / steps
    phase, prev, V = 0.0, 0.0, U
    for _ in range(steps):
        V = oracle.step(p, V, dt)
        z = np.sum((V[0] - h0) * np.exp(-1j * th))
        ang = -np.angle(z)
        phase += (ang - prev + math.pi) % (2 * math.pi) - math.pi
        prev = ang
    return phase / T, wp


@pytest.mark.parametrize("scheme,cfl", [(oracle.SCHEME_ARS222, 1.0), (oracle.SCHEME_EX_HEUN, 0.4)])
def test_second_order_schemes_converge_to_the_dispersion_relation(scheme, cfl):
    errs = []
    for n in (32, 64, 128):
        om, exact = measured_omega(n, 100.0, scheme, cfl)
        errs.append(abs(om - exact) / exact)
    assert errs[-1] < 3e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


@pytest.mark.parametrize("scheme,cfl,order", [(oracle.SCHEME_ARS222, 1.0, 2),
                                              (oracle.SCHEME_EX_HEUN, 0.4, 2)])
def test_solitary_wave_convergence(scheme, cfl, order):
    errs = []
    for n in (200, 400, 800):
        x, dx = inputs.cell_centres(n, -50.0, 50.0)
        U = inputs.solitary(x, 1.0, 0.2, 0.0, period=100.0)
        p = oracle.Params(n, dx, 0, lam=1000.0, scheme=scheme)
        dt, _, _ = oracle.suggest_dt(p, U, cfl, 0.5)
        steps = int(math.ceil(1.0 / dt))
        V = oracle.run(p, U, 1.0 / steps, steps)
        E = inputs.solitary(x, 1.0, 0.2, 0.0, t=1.0, period=100.0)
        errs.append(np.sum(np.abs(V[0] - E[0])) / np.sum(np.abs(V[0])))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 1.8, errs


def spectral_radius(U, g, lam):
    """max over cells of |u| + c, c^2 = g h + (lambda/3) eta^2/h^2 (Sec. 2.2,
    the eigenvalues of the hSGN system), from its definition."""
    h, q, m, _ = U
    eta = m / h
    return float(np.max(np.abs(q / h) + np.sqrt(g * h + (lam / 3.0) * eta * eta / (h * h))))


def test_explicit_steps_use_the_spectral_radius_as_rusanov_speed():
    # every wave of the explicit schemes is explicit: their Rusanov speed is
    # the spectral radius of the state (reading R12). One Euler step is
    # U + dt L(U); one Heun step is (U + U* + dt L(U*))/2 with U* the Euler
    # step, each L with the spectral radius of its own state
    n, dx, lam, g = 400, 0.1, 300.0, 9.81
    U = inputs.random_state(31, n, dx)
    dt = 0.004

    def L(V):
        p = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=lam,
                          speed=spectral_radius(V, g, lam))
        return oracle.explicit_rhs(p, V)

    def L0(V):  # forward Euler runs without reconstruction (first order)
        p = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=lam, recon=0,
                          speed=spectral_radius(V, g, lam))
        return oracle.explicit_rhs(p, V)

    LU0 = L0(U)
    euler = [U[k] + dt * LU0[k] for k in range(4)]
    got = oracle.run(oracle.Params(n, dx, oracle.BC_PERIODIC, lam=lam, recon=0,
                                   scheme=oracle.SCHEME_EX_EULER), U, dt, 1)
    for k in range(4):
        np.testing.assert_allclose(got[k], euler[k], rtol=1e-13, atol=1e-13)
    p_heun = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=lam, scheme=oracle.SCHEME_EX_HEUN)
    got = oracle.run(p_heun, U, dt, 1)
    # Heun's two evaluations share the step's speed, that of U^n
    LU = L(U)
    sp = spectral_radius(U, g, lam)
    p = oracle.Params(n, dx, oracle.BC_PERIODIC, lam=lam, speed=sp)
    Us = [U[k] + dt * LU[k] for k in range(4)]
    LUs = oracle.explicit_rhs(p, Us)
    heun = [0.5 * (U[k] + Us[k] + dt * LUs[k]) for k in range(4)]
    for k in range(4):
        np.testing.assert_allclose(got[k], heun[k], rtol=1e-13, atol=1e-13)


def test_explicit_heun_gaussian_bell_stays_bounded():
    # the breakdown of the Gaussian bell (Sec. 6.1, lambda = 100) to t = 35 with
    # Heun at CFL 0.4, on 1000 cells of [-200, 200]: with a Rusanov speed of
    # |u| only, the centred acoustic terms of the explicit scheme are undamped
    # and the depth goes negative long before t = 35
    x, dx, U = inputs.gaussian_bell(n=1000)
    p = oracle.Params(1000, dx, oracle.BC_TRANSMISSIVE, lam=100.0, scheme=oracle.SCHEME_EX_HEUN)
    dt0, _, _ = oracle.suggest_dt(p, U, 0.4, 0.0)
    steps = int(np.ceil(35.0 / dt0))
    got = oracle.run(p, U, 35.0 / steps, steps)
    assert np.all(got[0] > 0.5) and np.all(got[0] < 2.0)
