"""Pins for the oracle's boundary conditions (walls and far field; readings, the paper gives
neither) and the plunging-airfoil case: ghost-state identities, rest and free stream
preserved, mass conserved at walls, and an exact standing acoustic wave between walls
converging at the rate N+1."""
import math

import numpy as np
import pytest

from oracle import physics
from oracle.solver import Motion, OracleSolver
from paper_2607_00199_b300 import inputs


def _state(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v = flow(xn[..., 0], xn[..., 1])
    return np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))


def test_wall_ghost_identities():
    rng = np.random.default_rng(5)
    q = rng.normal(size=(40, 6))
    q[:, 0] = 1.0 + 0.1 * np.abs(q[:, 0])
    wx, wy = rng.normal(size=40) * 0.3, rng.normal(size=40) * 0.3
    # a reflection: applying it twice is the identity
    np.testing.assert_allclose(physics.wall_ghost(physics.wall_ghost(q, wx, wy), wx, wy), q, atol=1e-14)
    # a wall at rest flips the odd (first-order) moments and keeps the even ones
    g = physics.wall_ghost(q, 0.0, 0.0)
    np.testing.assert_array_equal(g[:, [1, 2]], -q[:, [1, 2]])
    np.testing.assert_array_equal(g[:, [0, 3, 4, 5]], q[:, [0, 3, 4, 5]])
    # the Maxwellian at velocity u reflects to the Maxwellian at 2 u_w - u
    c = 10.0
    rho, u, v = 1.2, 0.7, -0.4
    uw, vw = 0.3, 0.1
    qe = physics.equilibrium_state(rho, u, v, c)
    np.testing.assert_allclose(physics.wall_ghost(qe, uw / c, vw / c),
                               physics.equilibrium_state(rho, 2 * uw - u, 2 * vw - v, c), atol=1e-15)


def test_rest_state_is_steady_with_walls_and_far_field():
    mesh = inputs.naca_ogrid_mesh(24, 8, R=5.0)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=100, far_state=(1.0, 0.0, 0.0))
    q = _state(o, o.X, lambda x, y: (np.ones_like(x), 0 * x, 0 * x))
    F = o.rhs(q, o.X, o.motion.velocity(o.X, 0.0))
    # round-off of the derivative operators on the thinnest cells: ~ eps c / h_min
    assert np.abs(F).max() < 1e-13 * o.c / inputs.min_altitude(mesh)


def test_free_stream_preserved_with_far_field_on_a_plunging_mesh():
    """GCL with moving boundaries: the uniform free stream is the far-field state, so with
    the whole mesh plunging rigidly it stays uniform to round-off."""
    mesh = inputs.wall_channel_mesh(6, 4, 2.0, 1.0)
    mesh['bc'] = np.where(mesh['bc'] > 0, inputs.BC_FARFIELD, 0).astype(np.int8)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=100, motion=Motion(0.25, 2.0, kind='plunge'), far_state=(1.0, 1.0, 0.3))
    q0 = _state(o, o.X, lambda x, y: (np.ones_like(x), 1.0 + 0 * x, 0.3 + 0 * x))
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    q, xv, _ = o.run(q0, o.X.copy(), 0.0, dt, 10)
    assert np.abs(q - q0).max() < 1e-13
    assert np.abs(xv[:, 1] - o.X[:, 1]).max() > 1e-4 and np.abs(xv[:, 0] - o.X[:, 0]).max() == 0


def test_mass_conserved_between_walls():
    mesh = inputs.wall_channel_mesh(5, 4, 2.0, 1.0)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=100)
    q0 = _state(o, o.X, lambda x, y: inputs.random_flow(x, 2 * math.pi * y, 9))
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    m0 = o.integral(q0[:, 0], o.X)
    q, xv, _ = o.run(q0, o.X.copy(), 0.0, dt, 8)
    assert abs(o.integral(q[:, 0], xv) - m0) < 1e-13 * abs(m0)
    assert np.abs(q - q0).max() > 1e-6


def _standing_wave_error(nx, N):
    """q = rest + eps [r cos(k(x - s t)) + R r cos(k(x + s t))] on the x-chain (q1, q2, q5) of
    At_x, r = (1, sqrt3, sqrt2), R the reflection of the first moments, s = sqrt3 c, k = pi/L:
    an exact solution with zero velocity on the walls x = 0, L (collision off)."""
    L = 1.0
    mesh = inputs.wall_channel_mesh(nx, 3, L, 0.5)
    o = OracleSolver(mesh, N, c=1.0, tau=float('inf'))
    r = np.array([1.0, math.sqrt(3.0), 0.0, 0.0, math.sqrt(2.0), 0.0])
    Rr = r * np.array([1.0, -1.0, -1.0, 1.0, 1.0, 1.0])
    k, s, eps = math.pi / L, math.sqrt(3.0), 0.01
    rest = np.array([1.0, 0, 0, 0, 0, 0])

    def exact(t):
        x = o.node_coords(o.X)[..., 0]
        return (rest[None, :, None] + eps * (r[None, :, None] * np.cos(k * (x - s * t))[:, None, :]
                                             + Rr[None, :, None] * np.cos(k * (x + s * t))[:, None, :]))

    T = 0.2
    dt = 0.5 * inputs.min_altitude(mesh) / (math.sqrt(3.0) * (N + 1) ** 2)
    steps = int(math.ceil(T / dt))
    q, xv, _ = o.run(exact(0.0), o.X.copy(), 0.0, T / steps, steps)
    err = q - exact(T)
    _, J, _, _ = o.geometry(xv)
    return math.sqrt(np.einsum('e,ij,efi,efj->', J, o.ref.M, err, err))


@pytest.mark.parametrize('N', [1, 2, 3])
def test_standing_wave_between_walls_converges(N):
    e1, e2 = _standing_wave_error(4, N), _standing_wave_error(8, N)
    assert math.log2(e1 / e2) > N + 1 - 0.4, (e1, e2)


def test_ogrid_mesh_and_plunge_motion():
    mesh = inputs.naca_ogrid_mesh(32, 12, R=20.0)
    o = OracleSolver(mesh, 2, Ma=0.1, Re=1000, motion=Motion(0.25, 2.0, kind='plunge'))
    _, J, _, _ = o.geometry(o.X)
    assert J.min() > 0
    assert (o.bc == inputs.BC_WALL).sum() == 32 and (o.bc == inputs.BC_FARFIELD).sum() == 32
    # the airfoil surface is the closed-trailing-edge NACA 0012 section, chord 1
    surf = mesh['X'][:32]
    np.testing.assert_allclose(np.abs(surf[:, 1]), inputs.naca4_thickness(surf[:, 0]), atol=1e-15)
    assert abs(surf[:, 0].max() - 1.0) < 1e-15 and abs(surf[:, 0].min()) < 1e-15
    # rigid plunge h(t) = 0.25 sin(2 pi 0.5 t): uniform vertical grid velocity
    v = o.motion.velocity(o.X, 0.3)
    np.testing.assert_allclose(v[:, 1], 0.25 * math.pi * math.cos(math.pi * 0.3))
    assert np.abs(v[:, 0]).max() == 0
