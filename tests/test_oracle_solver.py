"""Pins for the oracle's ALE right-hand side and SARK step (Secs. 2-5, Sec. 7.1)."""
import math
import os

import numpy as np
import pytest

from oracle import physics
from oracle.solver import Motion, OracleSolver
from paper_2607_00199_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')


def _state(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v = flow(xn[..., 0], xn[..., 1])
    return np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))


def test_connectivity_is_an_involution():
    mesh = inputs.periodic_square_mesh(5, jitter=0.1)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=100)
    K = o.K
    for e in range(K):
        for f in range(3):
            e2, f2 = o.nbr_elem[e, f], o.nbr_face[e, f]
            assert o.nbr_elem[e2, f2] == e and o.nbr_face[e2, f2] == f
            # node pairing is a bijection between the two faces, and an involution
            back = {int(o.nbr_node[e2, f2, k]) for k in range(o.ref.Nfp)}
            assert back == set(int(i) for i in o.ref.fmask[f])


def _free_stream_error(n, N, L, A, T, u0, v0, nsteps, cfl=0.5):
    mesh = inputs.periodic_square_mesh(n, L=L, jitter=0.0)
    o = OracleSolver(mesh, N, Ma=0.1, Re=100, motion=Motion(A, T, L, L))
    q0 = _state(o, o.X, lambda x, y: inputs.free_stream(x, y, u0, v0))
    dt = inputs.cfl_dt(mesh, N, o.c, cfl)
    # the right-hand side balances the stiff decay exactly: F(q0) = Lambda q0 (Sec. 5)
    lam = np.array([0, 0, 0, 1, 1, 1]) / o.tau
    F = o.rhs(q0, o.X, o.motion.velocity(o.X, 0.3 * T))
    assert np.abs(F - lam[None, :, None] * q0).max() < 1e-12 * np.abs(F).max()
    q, xv, t = o.run(q0, o.X.copy(), 0.0, dt, nsteps)
    moved = np.abs(xv - o.X).max()
    rho, ru, rv = physics.macroscopic(q.transpose(0, 2, 1), o.c)
    area = L * L
    err_u = math.sqrt(o.integral((ru - u0) ** 2, xv) / area)
    err_v = math.sqrt(o.integral((rv - v0) ** 2, xv) / area)
    return err_u, err_v, moved


def test_free_stream_preserved_paper_setup():
    # Sec. 7.1: L = 20, X0 = Y0 = 0.5, n = 1, rho = 1, u = v = 1, Ma = 0.1, Re = 100,
    # 20 x 20 cells (K = 20^2 read as 20 x 20 quads, split into triangles).
    rows = [l.split() for l in open(os.path.join(GOLDEN, 'gcl_free_stream_table.txt')) if l.strip() and l[0] != '#']
    paper_scale = max(float(r[1]) for r in rows)
    eu, ev, moved = _free_stream_error(20, 3, 20.0, 0.5, 1.0, 1.0, 1.0, 60)
    assert moved > 0.05                       # the mesh really deformed
    # round-off level, the scale of the paper's Table 2
    assert eu < 20 * paper_scale and ev < 20 * paper_scale, (eu, ev)


@pytest.mark.parametrize('N', [2, 4])
def test_free_stream_preserved_fast_motion(N):
    eu, ev, moved = _free_stream_error(6, N, 2 * math.pi, 0.15, 0.05, 1.0, 0.0, 40)
    assert moved > 0.04
    assert eu < 1e-13 and ev < 1e-13, (eu, ev)


def _plane_wave_error(n, N, A, t_end=0.5, cfl=0.4):
    """Collision off (tau = inf): q = qbar + r cos(x - lam c t) with At_x r = lam r is exact."""
    L = 2 * math.pi
    mesh = inputs.periodic_square_mesh(n, L=L, jitter=0.0)
    o = OracleSolver(mesh, N, c=1.0, tau=float('inf'), motion=Motion(A, 0.7, L, L))
    lam, R = np.linalg.eigh(physics.ATX)
    k = int(np.argmax(lam))           # fastest wave, lam = sqrt(3)
    rvec = R[:, k]
    qbar = np.array([1.0, 0.1, -0.2, 0.0, 0.05, 0.0])

    def exact(xn, t):
        ph = np.cos(xn[..., 0] - lam[k] * t)
        return (qbar[None, None, :] + ph[..., None] * rvec[None, None, :]).transpose(0, 2, 1)

    dt0 = inputs.cfl_dt(mesh, N, 1.0, cfl)
    nsteps = int(math.ceil(t_end / dt0))
    dt = t_end / nsteps
    q0 = exact(o.node_coords(o.X), 0.0)
    q, xv, t = o.run(q0, o.X.copy(), 0.0, dt, nsteps)
    err = q - exact(o.node_coords(xv), t)
    return math.sqrt(sum(o.integral(err[:, f] ** 2, xv) for f in range(6)))


@pytest.mark.parametrize('N,A', [(2, 0.0), (2, 0.1), (3, 0.0), (3, 0.1)])
def test_plane_wave_convergence_rate(N, A):
    ns = (4, 8, 16) if N == 2 else (4, 8)
    errs = [_plane_wave_error(n, N, A) for n in ns]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert rates[-1] > N + 0.6, (errs, rates)


def test_planted_anti_upwind_flux_is_caught(monkeypatch):
    # a sign mistake in the upwinding (|An| -> -|An|) must break the convergence pin
    good = _plane_wave_error(8, 2, 0.0)
    orig = physics.abs_normal_matrix
    monkeypatch.setattr(physics, 'abs_normal_matrix', lambda nx, ny: -orig(nx, ny))
    bad = _plane_wave_error(8, 2, 0.0)
    assert not (bad < 3 * good)


def _kinetic_energy(o, q, xv):
    return o.diagnostics(q, xv)['kinetic_energy']


@pytest.mark.parametrize('A', [0.0, 0.05])
def test_taylor_green_decay(A):
    # incompressible limit: E_K(t) = E_K(0) exp(-4 nu t) with nu = 1/Re
    Ma, Re, N, n = 0.1, 10.0, 4, 8
    mesh = inputs.periodic_square_mesh(n)
    o = OracleSolver(mesh, N, Ma=Ma, Re=Re, motion=Motion(A, 1.0))
    q = _state(o, o.X, lambda x, y: inputs.taylor_green(x, y, Ma))
    t_end = 0.4
    dt0 = inputs.cfl_dt(mesh, N, o.c, 0.5)
    nsteps = int(math.ceil(t_end / dt0))
    dt = t_end / nsteps
    e0 = _kinetic_energy(o, q, o.X)
    q, xv, t = o.run(q, o.X.copy(), 0.0, dt, nsteps)
    rate = -math.log(_kinetic_energy(o, q, xv) / e0) / t
    assert abs(rate - 4.0 / Re) < 0.03 * 4.0 / Re, rate


def test_mass_conserved_on_static_mesh():
    mesh = inputs.periodic_square_mesh(6, jitter=0.1)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=100)
    q = _state(o, o.X, lambda x, y: inputs.random_flow(x, y, 7))
    m0 = o.integral(q[:, 0], o.X)
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    q, xv, t = o.run(q, o.X.copy(), 0.0, dt, 30)
    assert abs(o.integral(q[:, 0], xv) - m0) < 1e-13 * abs(m0)


def test_diagnostics_closed_forms_taylor_green():
    # Sec. 7.2 E_K for the 2D vortex u = sin x cos y, v = -cos x sin y with
    # rho = 1 + Ma^2/4 (cos 2x + cos 2y) on [0, 2 pi]^2: the rho perturbation
    # integrates to zero against |u|^2, so int rho = 4 pi^2 and E_K = 1/4 exactly;
    # both momenta vanish.  The nodal-interpolant integrals converge as h^(N+1).
    errs = []
    for n in (8, 16):
        mesh = inputs.periodic_square_mesh(n, jitter=0.1)
        o = OracleSolver(mesh, 4, Ma=0.1, Re=1000.0)
        d = o.diagnostics(_state(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1)), o.X)
        assert abs(d['area'] - 4 * math.pi ** 2) < 1e-12
        errs.append(max(abs(d['mass'] - 4 * math.pi ** 2), abs(d['kinetic_energy'] - 0.25),
                        abs(d['momentum_x']), abs(d['momentum_y'])))
    assert errs[1] < 1e-7 and errs[1] < errs[0] / 16, errs


def test_diagnostics_uniform_flow_exact():
    # constant integrands are integrated exactly on any affine mesh
    mesh = inputs.periodic_square_mesh(5, L=3.0, jitter=0.2)
    o = OracleSolver(mesh, 3, Ma=0.2, Re=50.0)
    d = o.diagnostics(_state(o, o.X, lambda x, y: inputs.free_stream(x, y, 0.6, -0.8)), o.X)
    assert abs(d['area'] - 9.0) < 1e-13
    assert abs(d['mass'] - 9.0) < 1e-13
    assert abs(d['kinetic_energy'] - 0.5) < 1e-13          # |u|^2 / 2 = (0.36 + 0.64) / 2
    assert abs(d['momentum_x'] - 9.0 * 0.6) < 1e-13 and abs(d['momentum_y'] + 9.0 * 0.8) < 1e-13


def test_mass_and_momentum_conserved_on_moving_mesh():
    # d/dt int q J = int (-div F + v_G . grad q + q div v_G) = 0 on the periodic
    # domain and the collision leaves the conserved moments q1..q3 unchanged
    # (Sec. 2): the semi-discrete scheme conserves them, the SARK step with
    # stage geometry (Sec. 6) up to its own O(dt^4) error, so the drift over a
    # fixed time falls at least 8x when dt halves; the torus area is exact.
    mesh = inputs.periodic_square_mesh(6, jitter=0.1)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=100, motion=Motion(0.1, 0.1))
    q0 = _state(o, o.X, lambda x, y: inputs.random_flow(x, y, 3))
    d0 = o.diagnostics(q0, o.X)
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    drift = []
    for k in (1, 2):
        q, xv, t = o.run(q0, o.X.copy(), 0.0, dt / k, 20 * k)
        assert np.abs(xv - o.X).max() > 0.01
        d1 = o.diagnostics(q, xv)
        assert abs(d1['area'] - d0['area']) < 1e-12 * d0['area']
        drift.append(max(abs(d1[k] - d0[k]) for k in ('mass', 'momentum_x', 'momentum_y')))
    assert drift[0] < 1e-7 * d0['mass'] and drift[1] < drift[0] / 8, drift


# ---- the prescribed mesh motion (Sec. 5, Sec. 7.1) and its RK4 vertex integration --------

def test_sinxy_motion_velocity_is_the_time_derivative_of_the_displacement():
    """The free-stream motion of Sec. 7.1: d(X, t) = A sin(2 pi t / T) S(X) with
    S = sin(2 pi X / Lx) sin(2 pi Y / Ly) on both components.  The velocity equals a central
    difference of the displacement; closed-form values at points where S is 1, 1/2 or -1
    (Lx != Ly, so a swapped period fails); periodic in X and Y; zero displacement at t = 0."""
    A, T, Lx, Ly = 0.05, 1.3, 2.0 * math.pi, 4.0
    m = Motion(A, T, Lx, Ly)
    rng = np.random.default_rng(11)
    X = np.stack([rng.uniform(0, Lx, 40), rng.uniform(0, Ly, 40)], axis=1)
    h = 1e-6
    for t in (0.0, 0.37, 0.9, 2.1):
        fd = (m.displacement(X, t + h) - m.displacement(X, t - h)) / (2 * h)
        np.testing.assert_allclose(m.velocity(X, t), fd, rtol=0, atol=1e-9)
    assert np.abs(m.displacement(X, 0.0)).max() == 0.0
    pts = np.array([[Lx / 4, Ly / 4], [Lx / 4, Ly / 12], [Lx / 4, 3 * Ly / 4]])
    S = np.array([1.0, 0.5, -1.0])
    np.testing.assert_allclose(m.displacement(pts, T / 4), A * np.stack([S, S], 1), rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(m.velocity(pts, 0.0), A * 2 * math.pi / T * np.stack([S, S], 1), rtol=1e-14)
    np.testing.assert_allclose(m.velocity(pts, T / 4), 0.0, atol=1e-16)
    np.testing.assert_allclose(m.displacement(X + [Lx, -Ly], 0.7), m.displacement(X, 0.7), atol=1e-15)


def _vertex_tracking_error(nsteps, t_end=0.3):
    mesh = inputs.periodic_square_mesh(3, jitter=0.1)
    o = OracleSolver(mesh, 1, Ma=0.1, Re=100, motion=Motion(0.05, 1.0))
    q0 = _state(o, o.X, lambda x, y: inputs.free_stream(x, y, 1.0, 0.0))
    _, xv, t = o.run(q0, o.X.copy(), 0.0, t_end / nsteps, nsteps)
    assert abs(t - t_end) < 1e-14
    return np.abs(xv - (o.X + o.motion.displacement(o.X, t_end))).max()


def test_rk4_vertices_track_the_prescribed_displacement():
    """Sec. 5: the vertices advance with the stages' RK4 (nodes c, weights b) and the analytic
    velocity at the Lagrangian X.  That velocity does not depend on x, so the step is
    Simpson's rule in time: x_n - (X + d(X, t_n)) falls like dt^4 (16x per halving).
    A wrong weight, node time or velocity factor breaks the level or the rate."""
    e1, e2, e3 = _vertex_tracking_error(3), _vertex_tracking_error(6), _vertex_tracking_error(12)
    assert e3 < 1e-7, e3
    for a, b in ((e1, e2), (e2, e3)):
        assert 13.0 < a / b < 19.0, (e1, e2, e3)
