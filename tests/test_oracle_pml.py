"""Pins for the oracle's perfectly matched layer (a reading: the paper prints no PML
equations; see oracle/pml.py): exact split of the advective terms, convergence to the exact
solution of the stretched system for a Fourier mode (q at rate N+1, Phi at rate N), sigma = 0 leaving the
scheme unchanged bit for bit, a uniform stream steady with the layer on the plunging
airfoil mesh, and absorption of an outgoing wave."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import physics
from oracle.pml import PML, sigma_max_for_reflection
from oracle.solver import Motion, OracleSolver
from paper_2607_00199_b300 import inputs

TWO_PI = 2.0 * math.pi


def _state(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v = flow(xn[..., 0], xn[..., 1])
    return np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))


def test_split_along_and_across_the_layer_is_exact():
    """R_e + R_t = L: the volume split through e e^T + t t^T = I and the face weights
    (n.e)^2 + (n.t)^2 = 1, on the O-grid's radial layer (collision off, moving mesh)."""
    mesh = inputs.naca_ogrid_mesh(24, 8, R=5.0)
    pml = PML('radial', centre=(0.5, 0.0), r0=2.0, d=3.0, sigma_max=1.0)
    o = OracleSolver(mesh, 3, c=10.0, tau=float('inf'), motion=Motion(0.25, 2.0, kind='plunge'), pml=pml)
    assert 0 < o.pml_layer.sum() < o.K
    q = _state(o, o.X, lambda x, y: inputs.random_flow(x, y, 11, amp=0.05))
    vv = o.motion.velocity(o.X, 0.3)
    xv = o.X + o.motion.displacement(o.X, 0.3)
    F, Re = o.rhs(q, xv, vv, along_pml=True)
    e = o.pml_dir.copy()
    o.pml_dir = np.stack([-e[..., 1], e[..., 0]], axis=-1)        # the tangential direction
    _, Rt = o.rhs(q, xv, vv, along_pml=True)
    assert np.abs(Re + Rt - F).max() <= 1e-12 * np.abs(F).max()
    assert np.abs(Re).max() > 0.1 * np.abs(F).max() and np.abs(Rt).max() > 0.1 * np.abs(F).max()


def _mode_error(n, N, sigma=1.0, alpha=0.5, T=0.5):
    """Uniform layer along x on the periodic square, collision off, static mesh: for
    q = Re(qhat e^{ikx}), Phi = Re(phihat e^{ikx}) the stretched system is the 12 x 12 ODE
    d/dt [qhat; phihat] = [[ik A_x, -sigma], [ik A_x, -(alpha + sigma)]] [qhat; phihat]."""
    mesh = inputs.periodic_square_mesh(n, L=TWO_PI)
    pml = PML('uniform', sigma_max=sigma, alpha=alpha, direction=(1.0, 0.0))
    o = OracleSolver(mesh, N, c=1.0, tau=float('inf'), pml=pml)
    rng = np.random.default_rng(7)
    q0hat = rng.normal(size=6)
    Ax, _ = physics.flux_matrices(o.c)
    I6 = np.eye(6)
    Mb = np.block([[1j * Ax, -sigma * I6], [1j * Ax, -(alpha + sigma) * I6]])
    zT = scipy.linalg.expm(T * Mb) @ np.concatenate([q0hat, np.zeros(6)])
    x = o.node_coords(o.X)[..., 0]                                   # (K, Np)
    q0 = np.ascontiguousarray(q0hat[None, :, None] * np.cos(x)[:, None, :])
    dt = 0.4 * inputs.min_altitude(mesh) / (math.sqrt(3.0) * (N + 1) ** 2)
    steps = int(math.ceil(T / dt))
    q, phi, _, _ = o.run_pml(q0, np.zeros_like(q0), o.X.copy(), 0.0, T / steps, steps)
    wave = np.exp(1j * x)[:, None, :]
    qex = np.real(zT[None, :6, None] * wave)
    pex = np.real(zT[None, 6:, None] * wave)
    _, J, _, _ = o.geometry(o.X)
    norm = lambda d: math.sqrt(np.einsum('e,ij,efi,efj->', J, o.ref.M, d, d))
    return norm(q - qex), norm(phi - pex), np.abs(zT[6:]).max()


@pytest.mark.parametrize('N', [1, 2, 3])
def test_layer_converges_to_the_stretched_mode(N):
    """q converges at rate N+1 as without the layer; Phi, the time integral of a DG
    directional derivative (accurate to O(h^N)), at rate N."""
    (eq1, ep1, p1), (eq2, ep2, _) = _mode_error(4, N), _mode_error(8, N)
    assert p1 > 0.05                      # the auxiliary fields are far from zero
    assert math.log2(eq1 / eq2) > N + 1 - 0.4, (eq1, eq2)
    assert math.log2(ep1 / ep2) > N - 0.4, (ep1, ep2)


def test_sigma_zero_leaves_the_scheme_unchanged():
    mesh = inputs.naca_ogrid_mesh(24, 8, R=5.0)
    pml = PML('radial', centre=(0.5, 0.0), r0=2.0, d=3.0, sigma_max=0.0, alpha=0.3)
    motion = Motion(0.25, 2.0, kind='plunge')
    o = OracleSolver(mesh, 2, Ma=0.1, Re=200, motion=motion, pml=pml)
    ref = OracleSolver(mesh, 2, Ma=0.1, Re=200, motion=motion)
    q0 = _state(o, o.X, lambda x, y: (1.0 + 0.01 * np.exp(-((x - 0.5) ** 2 + y ** 2)), 1.0 + 0 * x, 0 * x))
    dt = inputs.cfl_dt(mesh, 2, o.c, 0.5)
    q, phi, _, _ = o.run_pml(q0, np.zeros_like(q0), o.X.copy(), 0.0, dt, 3)
    qr, _, _ = ref.run(q0, o.X.copy(), 0.0, dt, 3)
    np.testing.assert_array_equal(q, qr)


def test_free_stream_steady_with_the_layer():
    mesh = inputs.naca_ogrid_mesh(24, 8, R=5.0)
    far = (1.0, 1.0, 0.2)
    c = 10.0
    pml = PML('radial', centre=(0.5, 0.0), r0=2.0, d=3.0, sigma_max=sigma_max_for_reflection(c, 3.0), alpha=0.1)
    mesh['bc'] = np.where(mesh['bc'] > 0, inputs.BC_FARFIELD, 0).astype(np.int8)   # no wall: a pure stream
    o = OracleSolver(mesh, 3, Ma=0.1, Re=1000, motion=Motion(0.25, 2.0, kind='plunge'), far_state=far, pml=pml)
    q0 = _state(o, o.X, lambda x, y: (np.ones_like(x), far[1] + 0 * x, far[2] + 0 * x))
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    q, phi, _, _ = o.run_pml(q0, np.zeros_like(q0), o.X.copy(), 0.0, dt, 5)
    assert np.abs(q - q0).max() < 1e-13 and np.abs(phi).max() < 1e-11


def _pulse_run(nx, x0, Lx, layer, T=3.5, N=2):
    """Pressure pulse at (3, 1) in the channel [x0, x0 + Lx] x [0, 2] (periodic in y, far
    field at both ends), collision off, c = 1; returns {element centroid: q} at time T."""
    mesh = inputs.wall_channel_mesh(nx, 4, Lx, 2.0)
    mesh['X'] = mesh['X'] + np.array([x0, 0.0])
    mesh['bc'] = np.where(mesh['bc'] > 0, inputs.BC_FARFIELD, 0).astype(np.int8)
    rest = (1.0, 0.0, 0.0)
    o = OracleSolver(mesh, N, c=1.0, tau=float('inf'), far_state=rest, pml=layer)
    q0 = _state(o, o.X, lambda x, y: (1.0 + 0.01 * np.exp(-8.0 * ((x - 3.0) ** 2 + (y - 1.0) ** 2)), 0 * x, 0 * x))
    dt = inputs.cfl_dt(mesh, N, 1.0, 0.5)
    steps = int(math.ceil(T / dt))
    if layer is None:
        q, _, _ = o.run(q0, o.X.copy(), 0.0, T / steps, steps)
    else:
        q, _, _, _ = o.run_pml(q0, np.zeros_like(q0), o.X.copy(), 0.0, T / steps, steps)
    cen = o.element_vertices(o.X).mean(axis=1)
    return {tuple(np.round(cc, 9)): q[e] for e, cc in enumerate(cen)}, o


def test_layer_absorbs_outgoing_waves():
    """Reflections: the channel [0, 6] against the same grid on [-4, 10], where nothing
    reflected at the far ends returns by T = 3.5 (fastest speed sqrt3: 12.5 units there and
    back).  In the centre |x - 3| < 1.5 the far-field ends alone send back the obliquely
    incident waves; slab layers 1.5 deep at both ends (sigma_max for a 1e-6
    normal-incidence reflection of the continuous layer) cut that error by more than 3x
    (measured 5.5x)."""
    ref, _ = _pulse_run(56, -4.0, 14.0, None)
    errs = []
    for layer in (None, PML('slab', centre=(3.0, 1.0), r0=1.5, d=1.5, direction=(1.0, 0.0),
                            sigma_max=sigma_max_for_reflection(1.0, 1.5))):
        got, o = _pulse_run(24, 0.0, 6.0, layer)
        d2 = sum(float(np.sum((q - ref[k]) ** 2)) for k, q in got.items() if abs(k[0] - 3.0) < 1.5)
        errs.append(math.sqrt(d2))
    assert errs[0] > 1e-4 and errs[1] < errs[0] / 3, errs
