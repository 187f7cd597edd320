"""GPU parity on renumbered meshes: elements listed in a seeded random order and each
element's vertices in a seeded random orientation-preserving order (inputs.renumber_mesh),
so that faces meet in every pairing of local face numbers (and, in 3D, every face-vertex
permutation) and the library's element reordering starts from a scrambled order.  The CUDA
path (through the C ABI) and the FP64 oracle receive the same renumbered mesh.

Tolerances as for the generated meshes: FP64 relative L2 <= 1e-12 per right-hand side and
<= 1e-10 after steps; GB_MIXED <= 1e-5.
"""
import math

import numpy as np
import pytest

from oracle import physics, physics3d
from oracle.pml import PML, sigma_max_for_reflection
from oracle.solver import Motion, OracleSolver
from oracle.solver3d import OracleSolver3D, WaveMotion
from paper_2607_00199_b300 import inputs
from parity_metrics import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from paper_2607_00199_b300 import gb  # noqa: E402  (loads libgb.so; fails loudly if missing)

WAVE = dict(A0=0.02, A1=0.08, Lx=8.0, wavelength=1.0, omega=2 * math.pi, r0sq=0.25, yc=1.0, zc=1.0)
PLUNGE = (0.25, 2.0)
FAR = (1.0, 1.0, 0.0)




def rest(F):
    r = np.zeros(F)
    r[0] = 1.0
    return r


def stream():
    return torch.cuda.current_stream().cuda_stream


def gpu_rhs(s, q, t):
    dt = torch.float64 if s.precision == gb.GB_FP64 else torch.float32
    qq = q - rest(q.shape[1])[None, :, None] if s.precision == gb.GB_MIXED else q
    qd = torch.from_numpy(np.ascontiguousarray(qq)).to('cuda', dt)
    Fd = torch.empty_like(qd)
    s.rhs(t, qd, Fd)
    torch.cuda.synchronize()
    return Fd.double().cpu().numpy()


def state2(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v = flow(xn[..., 0], xn[..., 1])
    return np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))


def state3(o, xv, seed):
    xn = o.node_coords(xv)
    rho, u, v, w = inputs.random_flow_3d(xn[..., 0], xn[..., 1], xn[..., 2], seed)
    return np.ascontiguousarray(physics3d.equilibrium_state(rho, u, v, w, o.c).transpose(0, 2, 1))


def periodic2(n, N, precision, seed=5):
    mesh, _ = inputs.renumber_mesh(inputs.periodic_square_mesh(n, jitter=0.1), seed=seed)
    o = OracleSolver(mesh, N, Ma=0.1, Re=100.0, motion=Motion(0.05, 1.0))
    s = gb.Solver(mesh, N, 0.1, 100.0, precision=precision, stream=stream())
    s.set_motion(0.05, 1.0)
    return mesh, o, s


@pytest.mark.parametrize('N', [1, 2, 3, 4, 5, 6])
def test_rhs_on_a_renumbered_periodic_mesh(N):
    mesh, o, s = periodic2(5, N, gb.GB_FP64)          # K = 50: ragged against every tile size
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = state2(o, xv, lambda x, y: inputs.random_flow(x, y, 40 + N))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    F = gpu_rhs(s, q, t)
    assert rel_err(F, F_or) <= 1e-12
    for f in range(6):
        assert rel_err(F[:, f], F_or[:, f]) <= 1e-11, f
    np.testing.assert_allclose(s.nodes(), o.node_coords(xv), atol=1e-14)


@pytest.mark.parametrize('N', [1, 2, 3, 4, 5, 6])
def test_mixed_rhs_on_a_renumbered_periodic_mesh(N):
    mesh, o, s = periodic2(5, N, gb.GB_MIXED)
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = state2(o, xv, lambda x, y: inputs.random_flow(x, y, 50 + N))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    F = gpu_rhs(s, q, t)
    assert rel_err(F, F_or) <= 1e-5
    for f in range(6):
        assert rel_err(F[:, f], F_or[:, f]) <= 1e-4, f


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_steps_on_a_renumbered_periodic_mesh(precision):
    N = 4
    mesh, o, s = periodic2(7, N, precision, seed=8)
    q0 = state2(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1))
    dt = inputs.cfl_dt(mesh, N, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 20)
    q, t = s.fields()
    q_or, x_or, t_or = o.run(q0, o.X.copy(), 0.0, dt, 20)
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-13)
    assert abs(t - t_or) < 1e-14
    R = rest(6)[None, :, None]
    if precision == gb.GB_FP64:
        assert rel_err(q, q_or) <= 1e-10
    else:
        assert rel_err(q - R, q_or - R) <= 1e-5


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_rhs_on_a_renumbered_airfoil_grid(precision):
    """Wall and far-field faces whose local numbers were rotated with their elements."""
    mesh, _ = inputs.renumber_mesh(inputs.naca_ogrid_mesh(24, 9, R=5.0), seed=12)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=1000.0, motion=Motion(*PLUNGE, kind='plunge'), far_state=FAR)
    s = gb.Solver(mesh, 3, 0.1, 1000.0, precision=precision, stream=stream(), far_state=FAR)
    s.set_motion(*PLUNGE, kind=gb.GB_MOTION_PLUNGE)
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)

    def flow(x, y):
        rho, u, v = inputs.random_flow(x, y, 21, amp=0.02)
        return rho, 1.0 + 0.2 * u, 0.2 * v

    q = state2(o, xv, flow)
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    assert rel_err(gpu_rhs(s, q, t), F_or) <= (1e-12 if precision == gb.GB_FP64 else 1e-5)


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_layer_on_a_renumbered_airfoil_grid(precision):
    """The perfectly matched layer's element list and auxiliary fields follow the caller's
    (scrambled) element numbers: ids ascending in that numbering, Phi in that order."""
    mesh, _ = inputs.renumber_mesh(inputs.naca_ogrid_mesh(24, 9, R=5.0, growth=1.1), seed=13)
    pml = PML('radial', centre=(0.5, 0.0), r0=2.5, d=2.5, sigma_max=sigma_max_for_reflection(10.0, 2.5), alpha=0.2)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=1000.0, motion=Motion(*PLUNGE, kind='plunge'), far_state=FAR, pml=pml)
    s = gb.Solver(mesh, 3, 0.1, 1000.0, precision=precision, stream=stream(), far_state=FAR)
    s.set_motion(*PLUNGE, kind=gb.GB_MOTION_PLUNGE)
    s.set_pml(gb.GB_PML_RADIAL, centre=(0.5, 0.0), r0=2.5, d=2.5, sigma_max=pml.sigma_max, power=2.0, alpha=0.2)

    def flow(x, y):
        rho, u, v = inputs.random_flow(x, y, 23, amp=0.02)
        return rho, 1.0 + 0.2 * u, 0.2 * v

    q0 = state2(o, o.X, flow)
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 10)
    q, _ = s.fields()
    phi, ids = s.pml_fields()
    q_or, phi_or, _, _ = o.run_pml(q0, np.zeros_like(q0), o.X.copy(), 0.0, dt, 10)
    np.testing.assert_array_equal(ids, np.nonzero(o.pml_layer)[0])
    assert 0 < len(ids) < o.K
    assert rel_err(q, q_or) <= (1e-10 if precision == gb.GB_FP64 else 1e-5)
    assert rel_err(phi, phi_or[o.pml_layer]) <= (1e-9 if precision == gb.GB_FP64 else 1e-3)


def periodic3(dims, N, precision, seed=3):
    mesh, _ = inputs.renumber_mesh(inputs.periodic_box_tet_mesh(*dims, jitter=0.1), seed=seed)
    o = OracleSolver3D(mesh, N, Ma=0.1, Re=500.0, motion=WaveMotion(**WAVE))
    s = gb.Solver(mesh, N, 0.1, 500.0, precision=precision, stream=stream())
    s.set_wave_motion(**WAVE)
    return mesh, o, s


@pytest.mark.parametrize('N', [1, 2, 3, 4])
def test_rhs_on_a_renumbered_tetrahedral_mesh(N):
    mesh, o, s = periodic3((5, 3, 3), N, gb.GB_FP64)  # K = 270
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = state3(o, xv, 60 + N)
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    F = gpu_rhs(s, q, t)
    assert rel_err(F, F_or) <= 1e-12
    for f in range(10):
        assert rel_err(F[:, f], F_or[:, f]) <= 1e-11, f


@pytest.mark.parametrize('N,shape', [(1, 8), (2, 8), (3, 7), (2, 16), (3, 16)])
def test_mixed_rhs_on_a_renumbered_tetrahedral_mesh(N, shape):
    """Both 3D mixed kernels (the tensor-core kernel with its most warps per CTA, and the
    one-thread-per-node kernel, shape 16) on a mesh whose faces meet in every pairing and
    orientation."""
    mesh, o, s = periodic3((5, 3, 3), N, gb.GB_MIXED)
    s.set_launch_config(shape)
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = state3(o, xv, 70 + N)
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    assert rel_err(gpu_rhs(s, q, t), F_or) <= 1e-5


@pytest.mark.parametrize('shape', [7, 16])
def test_mixed_steps_on_a_renumbered_tetrahedral_mesh(shape):
    mesh, o, s = periodic3((6, 3, 3), 3, gb.GB_MIXED, seed=5)
    s.set_launch_config(shape)
    q0 = np.ascontiguousarray(state3(o, o.X, 90))
    dt = inputs.cfl_dt_3d(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 6)
    q, _ = s.fields()
    q_or, x_or, _ = o.run(q0, o.X.copy(), 0.0, dt, 6)
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-14)
    assert rel_err(q, q_or) <= 1e-5


def test_steps_on_a_renumbered_tetrahedral_mesh():
    mesh, o, s = periodic3((6, 3, 3), 2, gb.GB_FP64, seed=4)
    q0 = np.ascontiguousarray(state3(o, o.X, 80))
    dt = inputs.cfl_dt_3d(mesh, 2, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 10)
    q, _ = s.fields()
    q_or, x_or, _ = o.run(q0, o.X.copy(), 0.0, dt, 10)
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-14)
    assert rel_err(q, q_or) <= 1e-10
