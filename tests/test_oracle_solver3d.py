"""Pins for the oracle's 3D ALE right-hand side and SARK step on tetrahedra (Secs. 2-5)."""
import math

import numpy as np
import pytest

from oracle import physics3d
from oracle.solver3d import OracleSolver3D, TGVMotion3D, WaveMotion
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


# ---- the moving 3D Taylor-Green vortex (Sec. 7.2) ----------------------------------------

def test_tgv_deformation_closed_forms():
    """Eq. TGV_deformation: the velocity is the time derivative of the displacement, the
    displacement vanishes at t = 0 and T/2 and peaks (amplitude A) at T/4, it is periodic on
    the cube [-L/2, L/2]^3, and each component is independent of its own coordinate."""
    m = TGVMotion3D()
    rng = np.random.default_rng(3)
    X = rng.uniform(-math.pi, math.pi, size=(50, 3))
    h = 1e-5
    for t in (0.0, 1.3, 7.9):
        fd = (m.displacement(X, t + h) - m.displacement(X, t - h)) / (2 * h)
        np.testing.assert_allclose(m.velocity(X, t), fd, atol=1e-9)
    assert np.abs(m.displacement(X, 0.0)).max() == 0.0
    assert np.abs(m.displacement(X, 10.0)).max() < 1e-15
    corner = np.array([[-math.pi / 2, -math.pi / 2, -math.pi / 2]])   # S = sin(pi/2) = 1 there
    np.testing.assert_allclose(m.displacement(corner, 5.0), [[math.pi / 6] * 3], rtol=1e-15)
    for d in range(3):
        Xs = X.copy()
        Xs[:, d] += 2 * math.pi
        np.testing.assert_allclose(m.displacement(Xs, 3.0), m.displacement(X, 3.0), atol=1e-14)
        Xm = X.copy()
        Xm[:, d] = rng.uniform(-math.pi, math.pi, size=50)
        np.testing.assert_array_equal(m.displacement(Xm, 3.0)[:, d], m.displacement(X, 3.0)[:, d])


@pytest.mark.parametrize('vel', [(0.0, 0.0, 0.0), (1.0, 0.3, -0.2)])
def test_free_stream_preserved_on_the_tgv_deforming_cube(vel):
    """GCL with all three grid-velocity components non-zero: a uniform state stays uniform."""
    mesh = inputs.tgv_box_tet_mesh(4, jitter=0.1)
    motion = TGVMotion3D(T=2.0)      # a faster period so that the mesh moves visibly in 10 steps
    o = OracleSolver3D(mesh, 2, Ma=0.1, Re=1600, motion=motion)
    q0 = _state(o, o.X, lambda x, y, z: (np.ones_like(x), vel[0] + 0 * x, vel[1] + 0 * x, vel[2] + 0 * x))
    dt = inputs.cfl_dt_3d(mesh, 2, o.c, 0.5)
    q, xv, _ = o.run(q0, o.X.copy(), 0.0, dt, 10)
    assert np.abs(q - q0).max() < 1e-13
    assert min(np.abs(xv[:, d] - o.X[:, d]).max() for d in range(3)) > 1e-3


def test_tgv_diagnostics_closed_forms():
    """Sec. 7.2 E_K: for u = sin x cos y cos z, v = -cos x sin y cos z, w = 0 and rho = 1 the
    mean of |u|^2 / 2 over the cube is 1/8 and every momentum integral vanishes.  On the
    unjittered cube every element is a translate of one of 6 shapes, so the integral of an
    interpolant is a translation-invariant rule over n cells per direction, exact for
    e^{i k.x} with every |k_d| < n (here |k_d| <= 2 < n = 3).  A periodic deformation
    keeps the volume (2 pi)^3, and a uniform density integrates to it on the deformed mesh."""
    mesh = inputs.tgv_box_tet_mesh(3)
    o = OracleSolver3D(mesh, 3, Ma=0.1, Re=1600, motion=TGVMotion3D())
    flow = lambda x, y, z: (np.ones_like(x),) + inputs.taylor_green_3d(x, y, z, 0.1)[1:]
    d = o.diagnostics(_state(o, o.X, flow), o.X)
    assert abs(d['kinetic_energy'] - 0.125) < 1e-13
    assert abs(d['volume'] - TWO_PI ** 3) < 1e-11
    for k in ('momentum_x', 'momentum_y', 'momentum_z'):
        assert abs(d[k]) < 1e-12
    # the interpolant is not exact: a frequency-3 mode is aliased to the mean by the same rule
    d3 = o.diagnostics(_state(o, o.X, lambda x, y, z: (np.ones_like(x), np.sin(3 * x), 0 * x, 0 * x)), o.X)
    assert abs(d3['kinetic_energy'] - 0.25) > 1e-3
    mesh = inputs.tgv_box_tet_mesh(4, jitter=0.1)
    o = OracleSolver3D(mesh, 2, Ma=0.1, Re=1600, motion=TGVMotion3D())
    xv = o.X + o.motion.displacement(o.X, 5.0)
    d = o.diagnostics(_state(o, xv, lambda x, y, z: (np.ones_like(x), 0 * x, 0 * x, 0 * x)), xv)
    assert abs(d['volume'] - TWO_PI ** 3) < 1e-10 and abs(d['mass'] - TWO_PI ** 3) < 1e-10
    assert abs(d['kinetic_energy']) == 0.0


def test_tgv_mass_and_energy():
    """The TGV state on the static cube keeps its mass to round-off; on the deforming cube
    the nodal (non-conservative) ALE form keeps it to truncation error only.  The kinetic
    energy decays in both."""
    mesh = inputs.tgv_box_tet_mesh(3)
    for motion, tol in ((TGVMotion3D(A=0.0), 1e-13), (TGVMotion3D(T=2.0), 1e-7)):
        o = OracleSolver3D(mesh, 2, Ma=0.1, Re=100, motion=motion)
        q0 = _state(o, o.X, lambda x, y, z: inputs.taylor_green_3d(x, y, z, 0.1))
        dt = inputs.cfl_dt_3d(mesh, 2, o.c, 0.5)
        d0 = o.diagnostics(q0, o.X)
        q, xv, _ = o.run(q0, o.X.copy(), 0.0, dt, 8)
        d1 = o.diagnostics(q, xv)
        assert abs(d1['mass'] - d0['mass']) < tol * d0['mass']
        assert d1['kinetic_energy'] < d0['kinetic_energy']


# ---- the deforming channel's traveling wave and its RK4 vertex integration (Sec. 5) ---------

def test_channel_wave_velocity_is_the_time_derivative_of_the_displacement():
    """y += A(x) sin(k x - omega t) exp(-r^2 / r0^2), A(x) = A0 + A1 x / Lx, r the distance to
    the centreline (yc, zc): the velocity equals a central difference of the displacement, only
    the y component moves, and closed-form values on the centreline (x = 4: sin(8 pi - omega t))
    and at r^2 = r0^2 (a factor 1/e) hold."""
    m = WaveMotion(A0=0.02, A1=0.08, Lx=8.0)
    rng = np.random.default_rng(5)
    X = np.stack([rng.uniform(0, 8, 40), rng.uniform(0, 2, 40), rng.uniform(0, 2, 40)], axis=1)
    h = 1e-6
    for t in (0.0, 0.21, 0.75, 1.6):
        fd = (m.displacement(X, t + h) - m.displacement(X, t - h)) / (2 * h)
        np.testing.assert_allclose(m.velocity(X, t), fd, rtol=0, atol=1e-9)
        assert np.abs(m.displacement(X, t)[:, [0, 2]]).max() == 0.0
        assert np.abs(m.velocity(X, t)[:, [0, 2]]).max() == 0.0
    centre = np.array([[4.0, 1.0, 1.0]])
    amp = 0.02 + 0.08 * 0.5
    np.testing.assert_allclose(m.displacement(centre, 0.75)[0, 1], amp, rtol=1e-14)    # sin(8 pi - 3 pi / 2) = 1
    np.testing.assert_allclose(m.velocity(centre, 0.0)[0, 1], -TWO_PI * amp, rtol=1e-14)
    off = np.array([[4.0, 1.5, 1.0]])                                                  # r^2 = 0.25 = r0^2
    np.testing.assert_allclose(m.displacement(off, 0.75)[0, 1], amp / math.e, rtol=1e-14)
    # wavelength 1: shifting x by one wavelength changes only the amplitude ramp
    a1 = m.displacement(X, 0.4)[:, 1] / (0.02 + 0.08 * X[:, 0] / 8)
    Xs = X + [1.0, 0.0, 0.0]
    a2 = m.displacement(Xs, 0.4)[:, 1] / (0.02 + 0.08 * Xs[:, 0] / 8)
    np.testing.assert_allclose(a1, a2, atol=1e-14)


def _vertex_tracking_error_3d(nsteps, t_end=0.3):
    mesh = inputs.periodic_box_tet_mesh(3, 3, 3, jitter=0.1)
    motion = WaveMotion(A0=0.02, A1=0.08, Lx=8.0)
    o = OracleSolver3D(mesh, 1, Ma=0.1, Re=500, motion=motion)
    q0 = _state(o, o.X, lambda x, y, z: (np.ones_like(x), np.full_like(x, 0.3), np.zeros_like(x), np.zeros_like(x)))
    _, xv, t = o.run(q0, o.X.copy(), 0.0, t_end / nsteps, nsteps)
    # the wave does not vanish at t = 0 and the mesh starts undeformed at X, so the vertices
    # follow X + d(X, t) - d(X, 0)
    return np.abs(xv - (o.X + motion.displacement(o.X, t_end) - motion.displacement(o.X, 0.0))).max()


def test_rk4_vertices_track_the_channel_wave():
    """Sec. 5 in 3D: RK4 with the analytic velocity at the Lagrangian X is Simpson's rule in
    time, so the vertices follow X + d(X, t) - d(X, 0) with an error falling like dt^4."""
    e1, e2, e3 = _vertex_tracking_error_3d(3), _vertex_tracking_error_3d(6), _vertex_tracking_error_3d(12)
    assert e3 < 1e-6, e3
    for a, b in ((e1, e2), (e2, e3)):
        assert 13.0 < a / b < 19.0, (e1, e2, e3)
