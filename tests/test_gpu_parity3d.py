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
from oracle.solver3d import OracleSolver3D, TGVMotion3D, WaveMotion
from paper_2607_00199_b300 import inputs
from parity_metrics import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from paper_2607_00199_b300 import gb  # noqa: E402  (loads libgb.so; fails loudly if missing)

REST = np.zeros(10)
REST[0] = 1.0
WAVE = dict(A0=0.02, A1=0.08, Lx=8.0, wavelength=1.0, omega=2 * math.pi, r0sq=0.25, yc=1.0, zc=1.0)




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
    assert rel_err(F_gpu, F_or) <= 1e-12
    for f in range(10):
        assert rel_err(F_gpu[:, f], F_or[:, f]) <= 1e-11, f


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
    assert rel_err(q_gpu, q_or) <= 1e-10


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
    assert rel_err(gpu_rhs(s, q, t), F_or) <= 1e-5


@pytest.mark.parametrize('N', [2, 3])
def test_mixed_step_error(N):
    mesh, o, s = make_pair((6, 3, 3), N, 0.1, 500.0, jitter=0.05, precision=gb.GB_MIXED)
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.channel_flow_3d(x, y, z, 0.1))
    dt = inputs.cfl_dt_3d(mesh, N, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 10)
    q_gpu, _ = s.fields()
    q_or, _, _ = o.run(q0, o.X.copy(), 0.0, dt, 10)
    e = rel_err(q_gpu, q_or)
    ep = rel_err(q_gpu - REST[None, :, None], q_or - REST[None, :, None])
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
    assert rel_err(gpu_rhs(s, q0, t), F_or) <= 1e-12
    dt = inputs.cfl_dt_3d(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 1)
    q_gpu, _ = s.fields()
    q_or, _ = o.step(q0, o.X.copy(), 0.0, dt)
    assert rel_err(q_gpu, q_or) <= 1e-12


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
        s.set_motion(0.05, 1.0)                     # GB_MOTION_SINXY is 2D only
    for bad in (dict(T=0.0), dict(T=float('nan')), dict(L=0.0)):
        with pytest.raises(gb.GBError) as ei:
            s.set_tgv_motion(**bad)
        assert ei.value.code == gb.GB_EINVAL


# ---- the moving 3D Taylor-Green vortex (Sec. 7.2): three grid-velocity components -------

def make_tgv_pair(n, N, precision=gb.GB_FP64, jitter=0.1, Re=1600.0, T=2.0):
    """Cube [-pi, pi]^3 of n^3 hexes (6 tets each), deformation of Eq. TGV_deformation with
    A = pi/6, L = 2 pi and a short period T so that the mesh moves visibly in a few steps."""
    mesh = inputs.tgv_box_tet_mesh(n, jitter=jitter)
    o = OracleSolver3D(mesh, N, Ma=0.1, Re=Re, motion=TGVMotion3D(T=T))
    s = gb.Solver(mesh, N, 0.1, Re, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    s.set_tgv_motion(T=T)
    return mesh, o, s


def tgv_flow(x, y, z):
    return inputs.taylor_green_3d(x, y, z, 0.1)


@pytest.mark.parametrize('N', [1, 2, 3, 4])
def test_tgv_rhs_parity(N):
    mesh, o, s = make_tgv_pair(4, N)          # K = 384: ragged against every tile size
    t = 0.7
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = oracle_state(o, xv, tgv_flow)
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    F = gpu_rhs(s, q, t)
    assert rel_err(F, F_or) <= 1e-12
    # per field, against max(|F_f|, 1e-4 |F|): the relaxation of the stress moments dominates
    # this near-equilibrium state, fields 1..4 are 2e-5..1e-4 of |F|, and their rounding error
    # scales with the advection terms summed into them, not with their small sum
    total = np.linalg.norm(F_or)
    for f in range(10):
        ref = max(np.linalg.norm(F_or[:, f]), 1e-4 * total)
        assert np.linalg.norm(F[:, f] - F_or[:, f]) <= 1e-11 * ref, f


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_tgv_steps_follow_oracle(precision):
    mesh, o, s = make_tgv_pair(4, 3, precision)
    q0 = oracle_state(o, o.X, tgv_flow)
    dt = inputs.cfl_dt_3d(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 8)
    q_gpu, t_gpu = s.fields()
    q_or, x_or, t_or = o.run(q0, o.X.copy(), 0.0, dt, 8)
    assert abs(t_gpu - t_or) < 1e-14
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-14)
    assert min(np.abs(x_or[:, d] - o.X[:, d]).max() for d in range(3)) > 1e-3
    assert rel_err(q_gpu, q_or) <= (1e-10 if precision == gb.GB_FP64 else 1e-5)


def test_tgv_free_stream_gcl_gpu():
    mesh, o, s = make_tgv_pair(4, 3)
    q0 = oracle_state(o, o.X, lambda x, y, z: (np.ones_like(x), 1.0 + 0 * x, 0.3 + 0 * x, -0.2 + 0 * x))
    s.set_fields(q0, 0.0)
    s.step(inputs.cfl_dt_3d(mesh, 3, o.c, 0.5), 25)
    q, _ = s.fields()
    assert np.abs(q - q0).max() < 1e-13


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_diagnostics3d_parity(precision):
    """Sec. 7.2 integrals of the GPU state against the oracle's on the same fields and
    vertices (both reduce in FP64), at t = 0 (closed forms of the unjittered cube: E_K = 1/8
    at rho = 1, volume (2 pi)^3) and after steps on the deforming mesh."""
    mesh, o, s = make_tgv_pair(3, 3, precision, jitter=0.0)
    flow1 = lambda x, y, z: (np.ones_like(x),) + tgv_flow(x, y, z)[1:]
    s.set_fields(oracle_state(o, o.X, flow1), 0.0)
    d = s.diagnostics()
    tol = 1e-13 if precision == gb.GB_FP64 else 1e-7
    assert abs(d['kinetic_energy'] - 0.125) <= tol and abs(d['volume'] - (2 * math.pi) ** 3) <= 1e-11
    s2 = s.diagnostics()
    assert s2 == d                               # fixed reduction order
    lib_d = np.zeros(5)
    s._c(gb.lib.gb_diagnostics(s.h, gb._ptr(lib_d)))
    np.testing.assert_array_equal(lib_d, [d['mass'], d['kinetic_energy'], d['momentum_x'], d['momentum_y'],
                                          d['volume']])
    mesh, o, s = make_tgv_pair(4, 3, precision)
    s.set_fields(oracle_state(o, o.X, tgv_flow), 0.0)
    s.step(inputs.cfl_dt_3d(mesh, 3, o.c, 0.5), 6)
    d = s.diagnostics()
    want = o.diagnostics(s.fields()[0], s.vertices())
    for k in want:
        assert abs(d[k] - want[k]) <= 1e-12 * max(1.0, abs(want[k])), (k, d[k], want[k])


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_diagnostics3d_history(precision):
    """Records taken at the end of the recorded steps (inside the step's CUDA graph) equal
    gb_diagnostics of a twin stepped one step at a time, and the oracle's run in FP64."""
    mesh, o, a = make_tgv_pair(3, 2, precision)
    _, _, b = make_tgv_pair(3, 2, precision)
    q0 = oracle_state(o, o.X, tgv_flow)
    dt = inputs.cfl_dt_3d(mesh, 2, o.c, 0.5)
    a.set_fields(q0, 0.0)
    b.set_fields(q0, 0.0)
    a.set_diagnostics(1, 16)
    a.step(dt, 6)
    h = a.diagnostics_history()
    assert h['total'] == 6 and len(h['t']) == 6
    q, xv, t = q0, o.X.copy(), 0.0
    for k in range(6):
        b.step(dt, 1)
        d = b.diagnostics()
        assert h['t'][k] == b.fields()[1]
        for key, hk in (('mass', 'mass'), ('kinetic_energy', 'kinetic_energy'), ('momentum_x', 'momentum_x'),
                        ('momentum_y', 'momentum_y'), ('volume', 'area')):
            assert abs(h[hk][k] - d[key]) <= 1e-13 * (abs(d[key]) + d['mass']), (k, key)
        q, xv = o.step(q, xv, t, dt)
        t += dt
        if precision == gb.GB_FP64:
            want = o.diagnostics(q, xv)
            assert abs(h['kinetic_energy'][k] - want['kinetic_energy']) <= 1e-11 * want['kinetic_energy']
    assert h['kinetic_energy'][-1] < h['kinetic_energy'][0]
    # every 4th step into a ring of 2
    a.set_diagnostics(4, 2)
    t0 = a.fields()[1]
    a.step(dt, 9)
    h = a.diagnostics_history()
    assert h['total'] == 2 and np.allclose(h['t'], [t0 + 4 * dt, t0 + 8 * dt], rtol=0, atol=1e-12)
    a.set_diagnostics(0)
    assert len(a.diagnostics_history()['t']) == 0


def test_full_size_tgv_rhs_and_step():
    """The moving Taylor-Green vortex at the paper's per-GPU load (24^3 x 6 = 82944
    tetrahedra, N = 3, Re 1600, A = pi/6, T = 20): one RHS of both precisions and one FP64
    SARK step against the oracle on every element."""
    mesh = inputs.tgv_box_tet_mesh(24)
    motion = TGVMotion3D()
    o = OracleSolver3D(mesh, 3, Ma=0.1, Re=1600.0, motion=motion)
    assert o.K == 82944
    t = 3.0
    xv = o.X + motion.displacement(o.X, t)
    q = oracle_state(o, xv, tgv_flow)
    F_or = o.rhs(q, xv, motion.velocity(o.X, t))
    for precision, tol in ((gb.GB_FP64, 1e-12), (gb.GB_MIXED, 1e-5)):
        s = gb.Solver(mesh, 3, 0.1, 1600.0, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
        s.set_tgv_motion()
        s.set_vertices(xv)
        assert rel_err(gpu_rhs(s, q, t), F_or) <= tol
        s.close()
    s = gb.Solver(mesh, 3, 0.1, 1600.0, stream=torch.cuda.current_stream().cuda_stream)
    s.set_tgv_motion()
    q0 = oracle_state(o, o.X, tgv_flow)
    dt = inputs.cfl_dt_3d(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 1)
    q_or, x_or = o.step(q0, o.X.copy(), 0.0, dt)
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-14)
    assert rel_err(s.fields()[0], q_or) <= 1e-12
