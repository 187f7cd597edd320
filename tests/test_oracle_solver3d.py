"""Pins for the oracle's 3D ALE right-hand side and SARK step on tetrahedra (Secs. 2-5)."""
import math

import numpy as np
import pytest

from oracle import physics3d
from oracle.solver3d import OracleSolver3D, WaveMotion
from paper_2607_00199_b300 import inputs

TWO_PI = 2.0 * math.pi


def _state(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v, w = flow(xn[..., 0], xn[..., 1], xn[..., 2])
    return np.ascontiguousarray(physics3d.equilibrium_state(rho, u, v, w, o.c).transpose(0, 2, 1))


def test_connectivity_is_an_involution():
    mesh = inputs.periodic_box_tet_mesh(3, 4, 3, jitter=0.1)
    o = OracleSolver3D(mesh, 3, Ma=0.1, Re=100)
    for e in range(o.K):
        for f in range(4):
            e2, f2 = o.nbr_elem[e, f], o.nbr_face[e, f]
            assert o.nbr_elem[e2, f2] == e and o.nbr_face[e2, f2] == f
            back = {int(o.nbr_node[e2, f2, k]) for k in range(o.ref.Nfp)}
            assert back == set(int(i) for i in o.ref.fmask[f])


def test_geometry_of_the_kuhn_cells():
    """Volumes sum to the box volume; normals of a face and of its neighbour's copy are opposite."""
    mesh = inputs.periodic_box_tet_mesh(3, 3, 4, L=(1.0, 2.0, 3.0), jitter=0.15)
    o = OracleSolver3D(mesh, 2, Ma=0.1, Re=100)
    Ginv, J, n, fs = o.geometry(o.X)
    assert abs(J.sum() * 4.0 / 3.0 - 6.0) < 1e-12
    for e in range(o.K):
        for f in range(4):
            e2, f2 = o.nbr_elem[e, f], o.nbr_face[e, f]
            np.testing.assert_allclose(n[e, f], -n[e2, f2], atol=1e-13)
            # Fscale J is the physical face area / 2 on both sides
            assert abs(fs[e, f] * J[e] - fs[e2, f2] * J[e2]) < 1e-13


@pytest.mark.parametrize('vel', [(1.0, 0.0, 0.0), (1.0, 1.0, 1.0)])
def test_free_stream_preserved_on_the_deforming_mesh(vel):
    """GCL (Sec. 5): a uniform state on the moving mesh stays uniform to round-off."""
    L = (8.0, 2.0, 2.0)
    mesh = inputs.periodic_box_tet_mesh(8, 3, 3, L=L)
    motion = WaveMotion(A0=0.02, A1=0.08, Lx=8.0)
    o = OracleSolver3D(mesh, 2, Ma=0.1, Re=500, motion=motion)
    q0 = _state(o, o.X, lambda x, y, z: (np.ones_like(x), vel[0] + 0 * x, vel[1] + 0 * x, vel[2] + 0 * x))
    lam = np.array([0] * 4 + [1] * 6) / o.tau
    F = o.rhs(q0, o.X + motion.displacement(o.X, 0.3), motion.velocity(o.X, 0.3))
    assert np.abs(F - lam[None, :, None] * q0).max() <= 1e-12 * np.abs(lam[None, :, None] * q0).max()
    dt = inputs.cfl_dt_3d(mesh, 2, o.c, 0.5)
    q, xv, _ = o.run(q0, o.X.copy(), 0.0, dt, 10)
    assert np.abs(q - q0).max() < 1e-13
    assert np.abs(xv - o.X).max() > 1e-4       # the mesh did move


def _plane_wave_error(n, N, moving):
    L = TWO_PI
    mesh = inputs.periodic_box_tet_mesh(n, 3, 3, L=(L, L, L))
    motion = WaveMotion(A0=0.05, A1=0.0, Lx=L, wavelength=L, omega=TWO_PI, r0sq=4.0, yc=math.pi, zc=math.pi) \
        if moving else WaveMotion()
    o = OracleSolver3D(mesh, N, c=1.0, tau=float('inf'), motion=motion)
    lam, R = np.linalg.eigh(physics3d.ATX)
    j = int(np.argmax(lam))                      # speed sqrt3 along x
    speed, r = -lam[j] * o.c, R[:, j]            # A_x = -c Atilde_x
    qbar = physics3d.equilibrium_state(1.0, 0.2, 0.1, 0.0, 1.0)

    def exact(xv, t):
        x = o.node_coords(xv)[..., 0]
        return qbar[None, :, None] + 0.1 * r[None, :, None] * np.cos(x + speed * t)[:, None, :]

    T = 0.3
    dt = 0.5 * inputs.min_altitude_3d(mesh) / (math.sqrt(3.0) * (N + 1) ** 2)
    steps = int(math.ceil(T / dt))
    dt = T / steps
    q, xv, _ = o.run(exact(o.X, 0.0), o.X.copy(), 0.0, dt, steps)
    err = q - exact(xv, T)
    _, J, _, _ = o.geometry(xv)
    return math.sqrt(np.einsum('e,ij,efi,efj->', J, o.ref.M, err, err))


@pytest.mark.parametrize('N,moving', [(1, False), (2, False), (2, True)])
def test_plane_wave_converges_at_order_N_plus_1(N, moving):
    """An exact plane wave of the linear system (collision off): the L2 error falls at
    the rate N+1 under h-refinement along the wave direction."""
    e1 = _plane_wave_error(6, N, moving)
    e2 = _plane_wave_error(12, N, moving)
    rate = math.log2(e1 / e2)
    assert rate > N + 1 - 0.35, (e1, e2, rate)


def test_mass_conserved_on_a_static_mesh():
    mesh = inputs.periodic_box_tet_mesh(4, 3, 3, L=(8.0, 2.0, 2.0), jitter=0.1)
    o = OracleSolver3D(mesh, 2, Ma=0.1, Re=200)
    q0 = _state(o, o.X, lambda x, y, z: inputs.random_flow_3d(x, y, z, seed=5))
    dt = inputs.cfl_dt_3d(mesh, 2, o.c, 0.5)
    m0 = o.integral(q0[:, 0], o.X)
    q, xv, _ = o.run(q0, o.X.copy(), 0.0, dt, 5)
    assert abs(o.integral(q[:, 0], xv) - m0) < 1e-13 * abs(m0)
    assert np.abs(q - q0).max() > 1e-6


@pytest.mark.slow
def test_shear_wave_decays_at_nu_k_squared():
    """u = eps sin(k z) e^{-nu k^2 t} (incompressible shear wave): the Galerkin-Boltzmann
    system recovers the viscosity nu = tau RT = 1/Re (Sec. 2) under the (Ma, Re) reading."""
    Lz = TWO_PI
    mesh = inputs.periodic_box_tet_mesh(3, 3, 8, L=(1.0, 1.0, Lz))
    Ma, Re = 0.1, 5.0
    o = OracleSolver3D(mesh, 2, Ma=Ma, Re=Re)
    eps = 0.05
    q0 = _state(o, o.X, lambda x, y, z: (np.ones_like(x), eps * np.sin(z), 0 * x, 0 * x))
    T = 0.2
    dt = inputs.cfl_dt_3d(mesh, 2, o.c, 0.5)
    steps = int(math.ceil(T / dt))
    dt = T / steps
    q, xv, _ = o.run(q0, o.X.copy(), 0.0, dt, steps)
    z = o.node_coords(xv)[..., 2]
    amp = lambda qq: o.integral(qq[:, 1] * o.c * np.sin(z), xv) / o.integral(np.sin(z) ** 2, xv)
    rate = -math.log(amp(q) / amp(q0)) / T
    print('shear-wave decay rate %.5f, nu k^2 = %.5f' % (rate, 1.0 / Re))
    assert abs(rate - 1.0 / Re) < 0.03 / Re, rate
