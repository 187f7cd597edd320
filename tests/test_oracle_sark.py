"""Pins for the SARK coefficients and scheme (Sec. 4)."""
import math

import mpmath as mp
import numpy as np
import pytest

from oracle import sark


def test_rk4_limit():
    E, A, B = sark.sark_coefficients(-1e-9)
    for i in range(4):
        for j in range(4):
            assert abs(A[i][j] - sark.RK4_A[i][j]) < 1e-8
    np.testing.assert_allclose(B, sark.RK4_B, atol=1e-8)
    np.testing.assert_allclose(E, 1.0, atol=1e-8)


@pytest.mark.parametrize('gamma', [-1e-6, -1e-3, -0.3, -1.0, -5.0, -40.0])
def test_sum_identities(gamma):
    E, A, B = sark.sark_coefficients(gamma)
    phi1 = lambda z: float(mp.expm1(mp.mpf(z)) / mp.mpf(z))
    assert abs(sum(B) - phi1(gamma)) < 1e-15 * max(1.0, abs(phi1(gamma)))
    for i in range(1, 4):
        ci = sark.RK4_C[i]
        # corrected stage constraint: sum_j atilde_ij = gamma^-1 (exp(c_i gamma) - 1)
        assert abs(sum(A[i]) - ci * phi1(ci * gamma)) < 1e-15
        assert abs(E[i] - math.exp(ci * gamma)) < 1e-15
    assert abs(E[4] - math.exp(gamma)) < 1e-15


def test_printed_stage_constraint_is_garbled():
    # the printed stage constraint carries an extra 1/c_i; the printed coefficients do not satisfy it
    gamma = -1.0
    E, A, B = sark.sark_coefficients(gamma)
    printed = (1 / 0.5) * (math.exp(0.5 * gamma) - 1) / gamma
    assert abs(sum(A[1]) - printed) > 0.1


def _phi(k, z):
    z = mp.mpf(z)
    return mp.nsum(lambda m: z ** m / mp.factorial(m + k), [0, mp.inf])


@pytest.mark.parametrize('gamma', [-1e-4, -0.5, -3.0, -20.0])
def test_matches_etdrk4_phi_functions(gamma):
    # the printed coefficients equal the Cox-Matthews ETDRK4 phi-combinations
    with mp.workdps(40):
        h = gamma / 2
        p1h, p2h = _phi(1, h), _phi(2, h)
        p1, p2, p3 = _phi(1, gamma), _phi(2, gamma), _phi(3, gamma)
        want_A = [float(p1h / 2), float(p1h / 2 - p2h), float(p2h), float(p1 - 2 * p2), 0.0, float(2 * p2)]
        want_B = [float(p1 - 3 * p2 + 4 * p3), float(2 * p2 - 4 * p3), float(2 * p2 - 4 * p3), float(4 * p3 - p2)]
    E, A, B = sark.sark_coefficients(gamma)
    got_A = [A[1][0], A[2][0], A[2][1], A[3][0], A[3][1], A[3][2]]
    np.testing.assert_allclose(got_A, want_A, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(B, want_B, rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize('tau', [1e-4, 1e-2, 1.0])
def test_constant_forcing_is_exact(tau):
    # y' = -y/tau + g, g constant: y(t) = g tau + (y0 - g tau) exp(-t/tau), for any dt
    g, y0, dt = 3.0, -0.7, 0.013
    y, t = y0, 0.0
    for _ in range(25):
        y = sark.sark_scalar_step(y, t, dt, tau, lambda yy, tt: g)
        t += dt
    exact = g * tau + (y0 - g * tau) * math.exp(-t / tau)
    assert abs(y - exact) < 1e-13 * max(1.0, abs(exact))


def test_fourth_order_convergence():
    tau = 0.7
    def run(n):
        dt, y, t = 1.0 / n, 0.3, 0.0
        for _ in range(n):
            y = sark.sark_scalar_step(y, t, dt, tau, lambda yy, tt: math.sin(3 * tt))
            t += dt
        a = 3.0
        # exact: particular (tau (sin a t - a tau cos a t)) / (1 + a^2 tau^2) plus homogeneous part
        yp = lambda tt: tau * (math.sin(a * tt) - a * tau * math.cos(a * tt)) / (1 + a * a * tau * tau)
        exact = yp(1.0) + (0.3 - yp(0.0)) * math.exp(-1.0 / tau)
        return abs(y - exact)
    e1, e2, e3 = run(10), run(20), run(40)
    assert 3.7 < math.log2(e1 / e2) < 4.4
    assert 3.7 < math.log2(e2 / e3) < 4.4


def test_nonlinear_rk4_limit_order():
    # tau = inf: plain RK4 on y' = -y^2 (nonlinear), fourth order
    def run(n):
        dt, y, t = 1.0 / n, 1.0, 0.0
        for _ in range(n):
            y = sark.sark_scalar_step(y, t, dt, float('inf'), lambda yy, tt: -yy * yy)
            t += dt
        return abs(y - 0.5)
    assert 3.7 < math.log2(run(8) / run(16)) < 4.4
