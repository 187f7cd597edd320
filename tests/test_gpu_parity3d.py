"""GPU parity in 3D: the tetrahedral CUDA path (through the C ABI, dim = 3) against the
FP64 3D oracle, element by element on the same seeded inputs.

Tolerances as in 2D: FP64 relative L2 <= 1e-12 per right-hand side (<= 1e-11 per field)
and <= 1e-10 after the step runs; GB_MIXED (FP32 perturbations) <= 1e-5 relative L2
against the FP64 oracle.
"""
import math

import numpy as np
import pytest

from oracle import physics3d
from oracle.solver3d import OracleSolver3D, WaveMotion
from paper_2607_00199_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from paper_2607_00199_b300 import gb  # noqa: E402  (loads libgb.so; fails loudly if missing)

REST = np.zeros(10)
REST[0] = 1.0
WAVE = dict(A0=0.02, A1=0.08, Lx=8.0, wavelength=1.0, omega=2 * math.pi, r0sq=0.25, yc=1.0, zc=1.0)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_state(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v, w = flow(xn[..., 0], xn[..., 1], xn[..., 2])
    return np.ascontiguousarray(physics3d.equilibrium_state(rho, u, v, w, o.c).transpose(0, 2, 1))


def make_pair(dims, N, Ma, Re, jitter=0.0, precision=gb.GB_FP64, L=(8.0, 2.0, 2.0), wave=WAVE):
    mesh = inputs.periodic_box_tet_mesh(*dims, L=L, jitter=jitter)
    o = OracleSolver3D(mesh, N, Ma=Ma, Re=Re, motion=WaveMotion(**wave))
    s = gb.Solver(mesh, N, Ma, Re, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    s.set_wave_motion(**wave)
    return mesh, o, s


def gpu_rhs(s, q, t):
    dt = torch.float64 if s.precision == gb.GB_FP64 else torch.float32
    qq = q - REST[None, :, None] if s.precision == gb.GB_MIXED else q
    qd = torch.from_numpy(np.ascontiguousarray(qq)).to('cuda', dt)
    Fd = torch.empty_like(qd)
    s.rhs(t, qd, Fd)
    torch.cuda.synchronize()
    return Fd.double().cpu().numpy()


@pytest.mark.parametrize('N', [1, 2, 3, 4])
def test_rhs_parity_all_orders_ragged(N):
    # 5 x 3 x 3 cells: K = 270, not a multiple of any tile size; jittered, moved vertices
    mesh, o, s = make_pair((5, 3, 3), N, 0.1, 500.0, jitter=0.1)
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = oracle_state(o, xv, lambda x, y, z: inputs.random_flow_3d(x, y, z, 17 + N))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    F_gpu = gpu_rhs(s, q, t)
    assert rel_l2(F_gpu, F_or) <= 1e-12
    for f in range(10):
        assert rel_l2(F_gpu[:, f], F_or[:, f]) <= 1e-11, f


def test_nodes_and_vertices_match_oracle():
    mesh, o, s = make_pair((4, 3, 3), 3, 0.1, 500.0, jitter=0.1)
    np.testing.assert_allclose(s.nodes(), o.node_coords(o.X), atol=1e-13)
    np.testing.assert_allclose(s.vertices(), o.X, atol=0)


@pytest.mark.parametrize('N,steps', [(2, 20), (3, 10)])
def test_step_parity_moving_mesh(N, steps):
    mesh, o, s = make_pair((6, 3, 3), N, 0.1, 500.0, jitter=0.05)
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.channel_flow_3d(x, y, z, 0.1))
    dt = inputs.cfl_dt_3d(mesh, N, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, steps)
    q_gpu, t_gpu = s.fields()
    q_or, x_or, t_or = o.run(q0, o.X.copy(), 0.0, dt, steps)
    assert abs(t_gpu - t_or) < 1e-14
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-14)
    assert rel_l2(q_gpu, q_or) <= 1e-10


@pytest.mark.parametrize('vel', [(1.0, 0.0, 0.0), (1.0, 1.0, 1.0)])
def test_free_stream_gcl_gpu(vel):
    mesh, o, s = make_pair((8, 3, 3), 3, 0.1, 500.0)
    q0 = oracle_state(o, o.X, lambda x, y, z: (np.ones_like(x), vel[0] + 0 * x, vel[1] + 0 * x, vel[2] + 0 * x))
    dt = inputs.cfl_dt_3d(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 25)
    q, _ = s.fields()
    assert np.abs(q - q0).max() < 1e-13
    assert np.abs(s.vertices() - o.X).max() > 1e-4


@pytest.mark.parametrize('N', [1, 2, 3, 4])
def test_mixed_rhs_all_orders(N):
    mesh, o, s = make_pair((5, 3, 3), N, 0.1, 500.0, jitter=0.1, precision=gb.GB_MIXED)
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = oracle_state(o, xv, lambda x, y, z: inputs.random_flow_3d(x, y, z, 29 + N))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    assert rel_l2(gpu_rhs(s, q, t), F_or) <= 1e-5


@pytest.mark.parametrize('N', [2, 3])
def test_mixed_step_error(N):
    mesh, o, s = make_pair((6, 3, 3), N, 0.1, 500.0, jitter=0.05, precision=gb.GB_MIXED)
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.channel_flow_3d(x, y, z, 0.1))
    dt = inputs.cfl_dt_3d(mesh, N, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 10)
    q_gpu, _ = s.fields()
    q_or, _, _ = o.run(q0, o.X.copy(), 0.0, dt, 10)
    e = rel_l2(q_gpu, q_or)
    ep = rel_l2(q_gpu - REST[None, :, None], q_or - REST[None, :, None])
    print('3D mixed N=%d: fields %.2e, perturbation %.2e' % (N, e, ep))
    assert e <= 1e-5 and ep <= 1e-4


def test_full_size_cfg4_rhs_and_step():
    """The deforming-channel workload at full size: 64 x 16 x 16 hexes -> K = 98304
    tetrahedra, N = 3, 10 fields, Ma 0.1, Re 500; one RHS and one SARK step against the
    oracle on every element."""
    mesh, o, s = make_pair((64, 16, 16), 3, 0.1, 500.0)
    assert o.K == 98304
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.channel_flow_3d(x, y, z, 0.1))
    t = 0.21
    F_or = o.rhs(q0, o.X, o.motion.velocity(o.X, t))
    assert rel_l2(gpu_rhs(s, q0, t), F_or) <= 1e-12
    dt = inputs.cfl_dt_3d(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 1)
    q_gpu, _ = s.fields()
    q_or, _ = o.step(q0, o.X.copy(), 0.0, dt)
    assert rel_l2(q_gpu, q_or) <= 1e-12


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_graph_steps_equal_direct_steps(precision):
    mesh, o, s = make_pair((5, 3, 3), 2, 0.1, 500.0, jitter=0.1, precision=precision)
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.random_flow_3d(x, y, z, 3))
    dt = inputs.cfl_dt_3d(mesh, 2, o.c, 0.5)
    side = torch.cuda.Stream()
    s.set_stream(side.cuda_stream)
    s.set_fields(q0, 0.0)
    s.step(dt, 6)                     # one direct step, then a captured graph replayed
    qa, ta = s.fields()
    s.set_graph(False)
    s.set_vertices(o.X)
    s.set_fields(q0, 0.0)
    s.step(dt, 6)
    qb, tb = s.fields()
    assert ta == tb
    np.testing.assert_array_equal(qa, qb)


def test_status_nan_and_tangled_mesh():
    mesh, o, s = make_pair((4, 3, 3), 2, 0.1, 500.0)
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.channel_flow_3d(x, y, z, 0.1))
    bad = q0.copy()
    bad[3, 2, 1] = np.nan
    dt = inputs.cfl_dt_3d(mesh, 2, o.c, 0.5)
    s.set_fields(bad, 0.0)
    s.step(dt, 1)
    with pytest.raises(gb.GBError) as ei:
        s.sync()
    assert ei.value.code == gb.GB_ENAN
    s.set_fields(q0, 0.0)          # the solver stays usable
    s.step(dt, 1)
    s.sync()
    # an amplitude far beyond the cell size folds elements over
    s.set_wave_motion(**dict(WAVE, A0=5.0, A1=0.0))
    s.step(0.05, 3)
    with pytest.raises(gb.GBError) as ei:
        s.sync()
    assert ei.value.code == gb.GB_EMESH


def test_create_rejects_bad_3d_meshes():
    mesh = inputs.periodic_box_tet_mesh(3, 3, 3)
    flipped = dict(mesh)
    E = mesh['EToV'].copy()
    E[0, [1, 2]] = E[0, [2, 1]]
    flipped['EToV'] = E
    sh = mesh['shift'].copy()
    sh[0, [1, 2]] = sh[0, [2, 1]]
    flipped['shift'] = sh
    with pytest.raises(gb.GBError) as ei:
        gb.Solver(flipped, 2, 0.1, 100.0)
    assert ei.value.code == gb.GB_EMESH
    with pytest.raises(gb.GBError) as ei:
        gb.Solver(mesh, 5, 0.1, 100.0)
    assert ei.value.code == gb.GB_EINVAL
    s = gb.Solver(mesh, 2, 0.1, 100.0, precision=gb.GB_MIXED)
    with pytest.raises(gb.GBError):
        s.diagnostics()
    with pytest.raises(gb.GBError):
        s.set_motion(0.05, 1.0)
