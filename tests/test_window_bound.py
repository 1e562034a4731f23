"""The decay bound behind the windowed depth solve (no GPU needed).

The windowed mixed-precision stage drops the coupling of the depth system
beyond a window and bounds the effect at a row i rows inside the window by
rho*^(i+1) |x_outside| with rho* = 2K / (B + sqrt(B^2 - 4 kappa K)),
B = 1 + K + kappa, where kappa and K bound the face couplings
tau^2 beta / dx^2 from below and above. This checks the bound against direct
solves of random windows with the structure of the depth matrix (diagonal
1 + l_i + r_i, off-diagonals -l_i, -r_i, l_i = r_{i-1}).
"""
import numpy as np


def rho_star(K, kap):
    B = 1.0 + K + kap
    return 2.0 * K / (B + np.sqrt(B * B - 4.0 * kap * K))


def window_response(kf):
    """Response of a window to a unit value just outside its left edge."""
    l, r = kf[:-1], kf[1:]
    W = len(l)
    A = np.diag(1 + l + r) - np.diag(r[:-1], 1) - np.diag(l[1:], -1)
    f = np.zeros(W)
    f[0] = l[0]
    return np.linalg.solve(A, f)


def test_bound_holds_on_random_windows():
    rng = np.random.default_rng(20251007)
    for _ in range(2000):
        W = int(rng.integers(10, 160))
        K = rng.uniform(0.01, 40.0)
        kap = K * rng.uniform(0.0, 1.0)
        kf = rng.uniform(kap, K, size=W + 1)
        e = window_response(kf)
        rho = rho_star(K, kap)
        assert np.all(np.abs(e) <= rho ** (np.arange(W) + 1) * (1 + 1e-9))


def test_bound_is_the_decay_rate_for_uniform_coefficients():
    # constant coupling k: the response decays like the smaller root of
    # k z^2 - (1 + 2k) z + k = 0, which rho*(k, k) equals
    for k in (0.1, 1.35, 5.0):
        e = window_response(np.full(201, k))
        rate = e[60] / e[59]
        assert abs(rate - rho_star(k, k)) < 1e-9
        z = ((1 + 2 * k) - np.sqrt((1 + 2 * k) ** 2 - 4 * k * k)) / (2 * k)
        assert abs(rho_star(k, k) - z) < 1e-12


def test_loose_limit_without_lower_bound():
    # kappa = 0 gives K / (1 + K), the bound when nothing is known below
    for K in (0.5, 3.0):
        assert abs(rho_star(K, 0.0) - K / (1 + K)) < 1e-15
