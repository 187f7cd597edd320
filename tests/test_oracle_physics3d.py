"""Pins for the oracle's 3D Galerkin-Boltzmann physics (Sec. 2: the 10-moment system)."""
import math

import numpy as np
import pytest

from oracle import physics, physics3d


def test_z_free_moments_reduce_to_the_printed_2d_matrices():
    sub = list(physics3d.SUBSET_2D)
    np.testing.assert_array_equal(physics3d.ATX[np.ix_(sub, sub)], physics.ATX)
    np.testing.assert_array_equal(physics3d.ATY[np.ix_(sub, sub)], physics.ATY)
    # z-derivative never touches the z-free moments among themselves
    assert not physics3d.ATZ[np.ix_(sub, sub)].any()


def test_y_and_z_are_interchangeable():
    """Swapping the y and z axes maps Atilde_y onto Atilde_z (isotropy of the expansion)."""
    swap = {a: i for i, a in enumerate(physics3d.MULTI_INDEX)}
    perm = [swap[(a[0], a[2], a[1])] for a in physics3d.MULTI_INDEX]
    np.testing.assert_array_equal(physics3d.ATY[np.ix_(perm, perm)], physics3d.ATZ)


def test_symmetric_with_the_hermite_spectrum():
    rng = np.random.default_rng(7)
    want = np.array([-math.sqrt(3), -1, -1, 0, 0, 0, 0, 1, 1, math.sqrt(3)])
    for A in (physics3d.ATX, physics3d.ATY, physics3d.ATZ):
        np.testing.assert_array_equal(A, A.T)
    for _ in range(20):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        An = n[0] * physics3d.ATX + n[1] * physics3d.ATY + n[2] * physics3d.ATZ
        np.testing.assert_allclose(np.linalg.eigvalsh(An), want, atol=1e-13)
        # the closed form used by the kernels: |A| = alpha A^2 + beta A^4 on that spectrum
        al, be = (9 - math.sqrt(3)) / 6, (math.sqrt(3) - 3) / 6
        A2 = An @ An
        np.testing.assert_allclose(al * A2 + be * A2 @ A2, physics3d.abs_normal_matrix(n), atol=1e-13)


def test_equilibrium_moment_flux_is_the_euler_flux():
    """c Atilde_d q at equilibrium: mass flux rho u_d, momentum flux (p delta + rho u u_d) / c."""
    c = 10.0
    rho, u, v, w = 1.3, 0.7, -0.4, 0.25
    q = physics3d.equilibrium_state(rho, u, v, w, c)
    vel = (u, v, w)
    p = rho * c * c
    for d, A in enumerate((physics3d.ATX, physics3d.ATY, physics3d.ATZ)):
        flux = c * (A @ q)
        assert abs(flux[0] - rho * vel[d]) < 1e-13
        for i in range(3):
            want = (p * (i == d) + rho * vel[i] * vel[d]) / c
            assert abs(flux[1 + i] - want) < 1e-12


def test_collision_term():
    tau = 1e-3
    q = physics3d.equilibrium_state(1.1, 0.3, -0.2, 0.5, 10.0)
    np.testing.assert_allclose(physics3d.collision(q, tau), 0.0, atol=1e-12)
    rng = np.random.default_rng(3)
    q = q + 0.01 * rng.normal(size=10)
    lam = np.array([0] * 4 + [1] * 6) / tau
    nt = np.zeros(10)
    nt[4:] = physics3d.ntilde(q[0], q[1], q[2], q[3], tau)
    np.testing.assert_allclose(physics3d.collision(q, tau), -lam * q + nt, rtol=1e-13, atol=1e-10)


@pytest.mark.parametrize('d', [0, 1, 2])
def test_two_dimensional_states_stay_two_dimensional(d):
    """A state with no velocity along axis d and moments even in it has zero coupling
    into the odd moments of axis d (the 3D system contains the 2D ones)."""
    vel = [0.4, -0.3, 0.2]
    vel[d] = 0.0
    q = physics3d.equilibrium_state(1.0, *vel, c=5.0)
    A = (physics3d.ATX, physics3d.ATY, physics3d.ATZ)[(d + 1) % 3]
    odd = [i for i, a in enumerate(physics3d.MULTI_INDEX) if a[d] % 2 == 1]
    np.testing.assert_allclose((A @ q)[odd], 0.0, atol=1e-15)
