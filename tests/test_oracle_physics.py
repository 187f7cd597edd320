"""Pins for the oracle's physics (Sec. 2: flux matrices, collision term, macroscopic maps)."""
import math

import numpy as np
import pytest

from oracle import physics


def test_flux_matrices_symmetric_hermite_spectrum():
    # a Hermite moment system is symmetric hyperbolic; for this truncation the
    # characteristic speeds in any direction are the roots of He_1, He_2, He_3:
    # {0} U {-1, 1} U {0, -sqrt3, sqrt3}
    for th in np.linspace(0, 2 * math.pi, 13):
        An = math.cos(th) * physics.ATX + math.sin(th) * physics.ATY
        assert np.allclose(An, An.T)
        lam = np.sort(np.linalg.eigvalsh(An))
        np.testing.assert_allclose(lam, [-math.sqrt(3), -1, 0, 0, 1, math.sqrt(3)], atol=1e-14)


def test_equilibrium_flux_is_euler_flux():
    # At equilibrium the moment flux -A q must reproduce the Euler fluxes:
    # (rho u, p + rho u^2, rho u v) in x and (rho v, rho u v, p + rho v^2) in y,
    # with p = rho c^2 (Sec. 2: p = rho RT, rho u = sqrt(RT) q2).
    rng = np.random.default_rng(0)
    c = 7.0
    Ax, Ay = physics.flux_matrices(c)
    for _ in range(10):
        rho, u, v = rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1)
        q = physics.equilibrium_state(rho, u, v, c)
        fx = -Ax @ q
        fy = -Ay @ q
        p = rho * c * c
        np.testing.assert_allclose([fx[0], c * fx[1], c * fx[2]], [rho * u, p + rho * u * u, rho * u * v], rtol=1e-13)
        np.testing.assert_allclose([fy[0], c * fy[1], c * fy[2]], [rho * v, rho * u * v, p + rho * v * v], rtol=1e-13)


def test_abs_normal_matrix_closed_form():
    # |At_n| = alpha At_n^2 + beta At_n^4 interpolates |x| on the spectrum {0, 1, sqrt3}
    al = (9 - math.sqrt(3)) / 6
    be = (math.sqrt(3) - 3) / 6
    th = np.linspace(0, 2 * math.pi, 17)
    absA = physics.abs_normal_matrix(np.cos(th), np.sin(th))
    for k, t in enumerate(th):
        An = math.cos(t) * physics.ATX + math.sin(t) * physics.ATY
        A2 = An @ An
        np.testing.assert_allclose(absA[k], al * A2 + be * A2 @ A2, atol=1e-14)


def test_collision_vanishes_at_equilibrium_and_split():
    rng = np.random.default_rng(1)
    tau = 3e-4
    q = physics.equilibrium_state(rng.uniform(0.5, 2, 8), rng.uniform(-1, 1, 8), rng.uniform(-1, 1, 8), 10.0)
    assert np.abs(physics.collision(q, tau)).max() < 1e-9
    # N(q) = -Lambda q + Ntilde(q) for any q
    qq = q + rng.normal(0, 0.01, q.shape)
    n4, n5, n6 = physics.ntilde(qq[:, 0], qq[:, 1], qq[:, 2], tau)
    Nfull = physics.collision(qq, tau)
    np.testing.assert_allclose(Nfull[:, 3], -qq[:, 3] / tau + n4, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(Nfull[:, 4], -qq[:, 4] / tau + n5, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(Nfull[:, 5], -qq[:, 5] / tau + n6, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize('Ma,Re', [(0.1, 100), (0.1, 1000), (0.05, 1600)])
def test_viscosity_reading(Ma, Re):
    c, tau = physics.sound_speed_and_tau(Ma, Re)
    # nu = tau RT (Sec. 2) equals 1/Re in units U = L = 1, and c = U/Ma
    assert abs(tau * c * c - 1.0 / Re) < 1e-15
    assert abs(c - 1.0 / Ma) < 1e-15


def test_macroscopic_round_trip():
    q = physics.equilibrium_state(1.2, 0.3, -0.4, 10.0)
    rho, ru, rv = physics.macroscopic(q, 10.0)
    np.testing.assert_allclose([rho, ru, rv], [1.2, 1.2 * 0.3, -1.2 * 0.4], rtol=1e-15)
