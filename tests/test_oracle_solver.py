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
    rho, ru, rv = physics.macroscopic(q.transpose(0, 2, 1), o.c)
    return o.integral(0.5 * (ru ** 2 + rv ** 2) / rho, xv) / (4 * math.pi ** 2)


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
