"""GPU parity with boundary faces (walls and far field) and the rigid plunge: the CUDA path
through gb_create_bounded against the FP64 oracle on the same seeded inputs.  Tolerances as
for periodic meshes: FP64 1e-12 per RHS and 1e-10 after steps; GB_MIXED 1e-5."""
import math

import numpy as np
import pytest

from oracle import physics
from oracle.solver import Motion, OracleSolver
from paper_2607_00199_b300 import inputs
from parity_metrics import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from paper_2607_00199_b300 import gb  # noqa: E402

REST = np.array([1.0, 0, 0, 0, 0, 0])
PLUNGE = (0.25, 2.0)        # h(t) = 0.25 sin(2 pi 0.5 t)
FAR = (1.0, 1.0, 0.0)




def oracle_state(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v = flow(xn[..., 0], xn[..., 1])
    return np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))


def airfoil_flow(x, y):
    """Free stream with a smooth seeded disturbance (inputs for parity, not a solution)."""
    rho, u, v = inputs.random_flow(x, y, 21, amp=0.02)
    return rho, 1.0 + 0.2 * u, 0.2 * v


def make_pair(mesh, N, precision=gb.GB_FP64, Re=1000.0, motion=PLUNGE, far=FAR):
    o = OracleSolver(mesh, N, Ma=0.1, Re=Re, motion=Motion(*motion, kind='plunge'), far_state=far)
    s = gb.Solver(mesh, N, 0.1, Re, precision=precision, stream=torch.cuda.current_stream().cuda_stream,
                  far_state=far)
    s.set_motion(*motion, kind=gb.GB_MOTION_PLUNGE)
    return o, s


def gpu_rhs(s, q, t):
    dt = torch.float64 if s.precision == gb.GB_FP64 else torch.float32
    qq = q - REST[None, :, None] if s.precision == gb.GB_MIXED else q
    qd = torch.from_numpy(np.ascontiguousarray(qq)).to('cuda', dt)
    Fd = torch.empty_like(qd)
    s.rhs(t, qd, Fd)
    torch.cuda.synchronize()
    return Fd.double().cpu().numpy()


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
@pytest.mark.parametrize('N', [1, 2, 3, 4])
def test_rhs_parity_ogrid(N, precision):
    mesh = inputs.naca_ogrid_mesh(24, 9, R=5.0)      # K = 432: ragged against every tile size
    o, s = make_pair(mesh, N, precision)
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = oracle_state(o, xv, airfoil_flow)
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    F = gpu_rhs(s, q, t)
    if precision == gb.GB_FP64:
        assert rel_err(F, F_or) <= 1e-12
        for f in range(6):
            assert rel_err(F[:, f], F_or[:, f]) <= 1e-11, f
    else:
        assert rel_err(F, F_or) <= 1e-5


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_steps_on_the_plunging_airfoil(precision):
    mesh = inputs.naca_ogrid_mesh(24, 9, R=5.0, growth=1.1)
    o, s = make_pair(mesh, 3, precision)
    q0 = oracle_state(o, o.X, airfoil_flow)
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 12)
    q_gpu, t_gpu = s.fields()
    q_or, x_or, t_or = o.run(q0, o.X.copy(), 0.0, dt, 12)
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-14)
    assert abs(t_gpu - t_or) < 1e-14
    assert rel_err(q_gpu, q_or) <= (1e-10 if precision == gb.GB_FP64 else 1e-5)


def test_standing_wave_between_walls_gpu():
    mesh = inputs.wall_channel_mesh(6, 3, 1.0, 0.5)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=100.0)
    s = gb.Solver(mesh, 3, 0.1, 100.0, stream=torch.cuda.current_stream().cuda_stream)
    q0 = oracle_state(o, o.X, lambda x, y: (1.0 + 0.01 * np.cos(math.pi * x), 0 * x, 0 * x))
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 20)
    q_gpu, _ = s.fields()
    q_or, _, _ = o.run(q0, o.X.copy(), 0.0, dt, 20)
    assert rel_err(q_gpu, q_or) <= 1e-10
    assert np.abs(q_gpu - q0).max() > 1e-5


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_free_stream_with_far_field_on_a_plunging_channel(precision):
    mesh = inputs.wall_channel_mesh(6, 4, 2.0, 1.0)
    mesh['bc'] = np.where(mesh['bc'] > 0, inputs.BC_FARFIELD, 0).astype(np.int8)
    far = (1.0, 1.0, 0.3)
    o, s = make_pair(mesh, 3, precision, far=far)
    q0 = oracle_state(o, o.X, lambda x, y: (np.ones_like(x), 1.0 + 0 * x, 0.3 + 0 * x))
    s.set_fields(q0, 0.0)
    s.step(inputs.cfl_dt(mesh, 3, o.c, 0.5), 20)
    q, _ = s.fields()
    assert np.abs(q - q0).max() < (1e-13 if precision == gb.GB_FP64 else 1e-5)
    assert np.abs(s.vertices()[:, 1] - o.X[:, 1]).max() > 1e-4


def test_full_size_airfoil_rhs():
    """The plunging-airfoil workload at full size: 256 x 192 O-grid quads -> K = 98304
    triangles, N = 4; one RHS of both precisions against the oracle on every element."""
    mesh = inputs.naca_ogrid_mesh(256, 192)
    o, s = make_pair(mesh, 4, gb.GB_FP64)
    assert o.K == 98304
    t = 0.4
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = oracle_state(o, xv, airfoil_flow)
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    assert rel_err(gpu_rhs(s, q, t), F_or) <= 1e-12
    s.close()
    sm = gb.Solver(mesh, 4, 0.1, 1000.0, precision=gb.GB_MIXED, stream=torch.cuda.current_stream().cuda_stream,
                   far_state=FAR)
    sm.set_motion(*PLUNGE, kind=gb.GB_MOTION_PLUNGE)
    sm.set_vertices(xv)
    assert rel_err(gpu_rhs(sm, q, t), F_or) <= 1e-5


def test_bounded_meshes_are_validated_and_not_grouped():
    mesh = inputs.wall_channel_mesh(4, 3, 1.0, 1.0)
    bad = dict(mesh)
    bad['bc'] = np.zeros_like(mesh['bc'])          # walls left untagged: open faces
    with pytest.raises(gb.GBError) as ei:
        gb.Solver(bad, 2, 0.1, 100.0)
    assert ei.value.code == gb.GB_EMESH
    s = gb.Solver(mesh, 2, 0.1, 100.0, precision=gb.GB_MIXED)
    g = gb.Group(2)
    with pytest.raises(gb.GBError):
        g.step([s], [1e-4], 1)
    with pytest.raises(gb.GBError):   # the tcgen05 kernel has no boundary-face variant
        s.set_launch_config(8)
    s.set_launch_config(4)
    with pytest.raises(gb.GBError) as ei:
        gb.Solver(mesh, 5, 0.1, 100.0)
    assert ei.value.code == gb.GB_EINVAL


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_recorded_diagnostics_on_the_plunging_airfoil(precision):
    """The record fused into the last stage of the boundary variant: every step's integrals
    equal those of gb_diagnostics on a twin stepped one step at a time (1e-13 relative to the
    mass), and in FP64 the oracle's integrals of the oracle's own run."""
    mesh = inputs.naca_ogrid_mesh(24, 9, R=5.0, growth=1.1)
    o, a = make_pair(mesh, 3, precision)
    _, b = make_pair(mesh, 3, precision)
    q0 = oracle_state(o, o.X, airfoil_flow)
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    a.set_fields(q0, 0.0)
    b.set_fields(q0, 0.0)
    a.set_diagnostics(1, 16)
    a.step(dt, 6)
    h = a.diagnostics_history()
    assert h['total'] == 6
    q, xv, t = q0, o.X.copy(), 0.0
    for k in range(6):
        b.step(dt, 1)
        d = b.diagnostics()
        assert h['t'][k] == b.fields()[1]
        for key in d:
            assert abs(h[key][k] - d[key]) <= 1e-13 * (abs(d[key]) + d['mass']), (k, key)
        q, xv = o.step(q, xv, t, dt)
        t += dt
        if precision == gb.GB_FP64:
            want = o.diagnostics(q, xv)
            for key in want:
                assert abs(h[key][k] - want[key]) <= 1e-11 * max(1.0, abs(want[key])), (k, key)
    # a plunge is rigid: the area of the domain (annulus minus airfoil) does not change
    assert np.ptp(h['area']) <= 1e-12 * h['area'][0]
