"""GPU parity of the 3D tensor-core stage kernel (GB_MIXED, N <= 3: 16-element warp tiles,
mma.sync TF32 split products) against the FP64 3D oracle, element by element, and against the
FP32 one-thread-per-node kernel (launch shape 16) on the same inputs.

Bars: 1e-5 (`rel_err`: relative L2 and element-wise against the array's largest value) to the
FP64 oracle; every warp count per CTA runs the same per-warp code and must agree bit for bit.
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
TC_SHAPES = (1, 2, 4)
SIMT = 16
TC_DEFAULT = {1: 8, 2: 8, 3: 7}        # the most warps per persistent CTA that fit


def oracle_state(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v, w = flow(xn[..., 0], xn[..., 1], xn[..., 2])
    return np.ascontiguousarray(physics3d.equilibrium_state(rho, u, v, w, o.c).transpose(0, 2, 1))


def channel(dims, N, jitter=0.1, Re=500.0):
    mesh = inputs.periodic_box_tet_mesh(*dims, L=(8.0, 2.0, 2.0), jitter=jitter)
    o = OracleSolver3D(mesh, N, Ma=0.1, Re=Re, motion=WaveMotion(**WAVE))
    return mesh, o


def mixed_solver(mesh, N, shape=None, Re=500.0, tgv=False):
    s = gb.Solver(mesh, N, 0.1, Re, precision=gb.GB_MIXED, stream=torch.cuda.current_stream().cuda_stream)
    if tgv:
        s.set_tgv_motion(T=2.0)
    else:
        s.set_wave_motion(**WAVE)
    if shape is not None:
        s.set_launch_config(shape)
    return s


def rhs_mixed(s, q, t, q_offset=0, F_offset=0):
    """F of the perturbation state through gb_rhs; the device buffers may start
    q_offset / F_offset floats into an allocation (unaligned views)."""
    qq = np.ascontiguousarray(q - REST[None, :, None]).astype(np.float32).ravel()
    qbuf = torch.zeros(qq.size + 4, dtype=torch.float32, device='cuda')
    qbuf[q_offset:q_offset + qq.size] = torch.from_numpy(qq).cuda()
    Fbuf = torch.full((qq.size + 4,), float('nan'), dtype=torch.float32, device='cuda')
    qd, Fd = qbuf[q_offset:q_offset + qq.size], Fbuf[F_offset:F_offset + qq.size]
    s.rhs(t, qd, Fd)
    torch.cuda.synchronize()
    return Fd.double().cpu().numpy().reshape(q.shape)


@pytest.mark.parametrize('N', [1, 2, 3])
def test_tc3_rhs_every_shape(N):
    # 5 x 3 x 3 cells: K = 270 = 16 x 16 + 14, a ragged last tile; jittered, moved vertices
    mesh, o = channel((5, 3, 3), N)
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    q = oracle_state(o, xv, lambda x, y, z: inputs.random_flow_3d(x, y, z, 41 + N))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    F = {}
    for shape in TC_SHAPES + (TC_DEFAULT[N], SIMT):
        s = mixed_solver(mesh, N, shape)
        s.set_vertices(xv)
        assert s.launch_config() == shape
        F[shape] = rhs_mixed(s, q, t)
        s.close()
        e = rel_err(F[shape], F_or)
        print('N=%d shape %d: %.2e against the FP64 oracle' % (N, shape, e))
        assert e <= 1e-5, shape
    for shape in TC_SHAPES[1:] + (TC_DEFAULT[N],):
        np.testing.assert_array_equal(F[shape], F[TC_SHAPES[0]])
    assert rel_err(F[TC_DEFAULT[N]], F[SIMT]) <= 1e-5


def test_tc3_is_the_default_for_orders_up_to_3():
    mesh, _ = channel((3, 3, 3), 1)
    for N, want in ((1, TC_DEFAULT[1]), (2, TC_DEFAULT[2]), (3, TC_DEFAULT[3]), (4, SIMT)):
        s = mixed_solver(mesh, N)
        assert s.launch_config() == want, N
        if N == 4:
            for bad in TC_SHAPES:
                with pytest.raises(gb.GBError) as ei:
                    s.set_launch_config(bad)
                assert ei.value.code == gb.GB_EINVAL
        for bad in (0, 9, 12, 17) + ((8,) if N == 3 else ()):
            with pytest.raises(gb.GBError) as ei:
                s.set_launch_config(bad)
            assert ei.value.code == gb.GB_EINVAL
        s.close()
    f = gb.Solver(mesh, 3, 0.1, 500.0, precision=gb.GB_FP64)
    assert f.launch_config() == 0
    with pytest.raises(gb.GBError) as ei:
        f.set_launch_config(2)
    assert ei.value.code == gb.GB_EINVAL


def test_tc3_unaligned_device_buffers():
    """q_dev 4 bytes past a 16-byte boundary: the tile is staged by 4-byte copies, same
    values as the aligned call; F_dev not 8-byte aligned: the call runs on the
    one-thread-per-node kernel (node-pair stores need 8-byte alignment)."""
    N = 3
    mesh, o = channel((4, 3, 3), N)
    t = 0.4
    xv = o.X + o.motion.displacement(o.X, t)
    q = oracle_state(o, xv, lambda x, y, z: inputs.random_flow_3d(x, y, z, 5))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    s = mixed_solver(mesh, N, 2)
    s.set_vertices(xv)
    F_al = rhs_mixed(s, q, t)
    np.testing.assert_array_equal(rhs_mixed(s, q, t, q_offset=1), F_al)
    np.testing.assert_array_equal(rhs_mixed(s, q, t, q_offset=2, F_offset=2), F_al)
    F_odd = rhs_mixed(s, q, t, F_offset=1)
    assert np.isfinite(F_odd).all()
    assert rel_err(F_odd, F_or) <= 1e-5
    simt = mixed_solver(mesh, N, SIMT)
    simt.set_vertices(xv)
    np.testing.assert_array_equal(F_odd, rhs_mixed(simt, q, t))


@pytest.mark.parametrize('N,steps', [(2, 12), (3, 10)])
def test_tc3_steps_follow_oracle(N, steps):
    mesh, o = channel((6, 3, 3), N, jitter=0.05)
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.channel_flow_3d(x, y, z, 0.1))
    dt = inputs.cfl_dt_3d(mesh, N, o.c, 0.5)
    q_or, x_or, t_or = o.run(q0, o.X.copy(), 0.0, dt, steps)
    out = {}
    for shape in (1, TC_DEFAULT[N], SIMT):
        s = mixed_solver(mesh, N, shape)
        s.set_fields(q0, 0.0)
        s.step(dt, steps)
        out[shape], t_gpu = s.fields()
        assert abs(t_gpu - t_or) < 1e-14
        np.testing.assert_allclose(s.vertices(), x_or, atol=1e-14)
        e = rel_err(out[shape], q_or)
        ep = rel_err(out[shape] - REST[None, :, None], q_or - REST[None, :, None])
        print('N=%d shape %d, %d steps: fields %.2e, perturbation %.2e' % (N, shape, steps, e, ep))
        assert e <= 1e-5 and ep <= 1e-4, shape
        s.close()
    np.testing.assert_array_equal(out[1], out[TC_DEFAULT[N]])


def test_tc3_tgv_steps_and_free_stream():
    mesh = inputs.tgv_box_tet_mesh(4, jitter=0.1)
    o = OracleSolver3D(mesh, 3, Ma=0.1, Re=1600.0, motion=TGVMotion3D(T=2.0))
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.taylor_green_3d(x, y, z, 0.1))
    dt = inputs.cfl_dt_3d(mesh, 3, o.c, 0.5)
    s = mixed_solver(mesh, 3, Re=1600.0, tgv=True)
    assert s.launch_config() == TC_DEFAULT[3]
    s.set_fields(q0, 0.0)
    s.step(dt, 8)
    q_or, x_or, _ = o.run(q0, o.X.copy(), 0.0, dt, 8)
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-14)
    assert rel_err(s.fields()[0], q_or) <= 1e-5
    # a uniform stream stays uniform on the deforming cube (GCL), to FP32 rounding
    qf = oracle_state(o, o.X, lambda x, y, z: (np.ones_like(x), 1.0 + 0 * x, 0.3 + 0 * x, -0.2 + 0 * x))
    s.set_vertices(o.X)
    s.set_fields(qf, 0.0)
    s.step(dt, 25)
    assert np.abs(s.fields()[0] - qf).max() < 1e-5


def test_tc3_graph_replay_and_nan_status():
    mesh, o = channel((5, 3, 3), 3)
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.random_flow_3d(x, y, z, 3))
    dt = inputs.cfl_dt_3d(mesh, 3, o.c, 0.5)
    s = mixed_solver(mesh, 3)
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
    bad = q0.copy()
    bad[7, 4, 2] = np.nan
    s.set_fields(bad, 0.0)
    s.step(dt, 1)
    with pytest.raises(gb.GBError) as ei:
        s.sync()
    assert ei.value.code == gb.GB_ENAN
    s.set_fields(q0, 0.0)             # the solver stays usable
    s.step(dt, 1)
    s.sync()


def test_tc3_full_size_channel_rhs_and_step():
    """The deforming channel at full size (64 x 16 x 16 hexes -> K = 98304 tetrahedra, N = 3,
    Ma 0.1, Re 500) on the tensor-core kernel: one RHS and one SARK step against the FP64
    oracle on every element."""
    mesh, o = channel((64, 16, 16), 3, jitter=0.0)
    assert o.K == 98304
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.channel_flow_3d(x, y, z, 0.1))
    t = 0.21
    s = mixed_solver(mesh, 3)
    assert s.launch_config() == TC_DEFAULT[3]
    F_or = o.rhs(q0, o.X, o.motion.velocity(o.X, t))
    assert rel_err(rhs_mixed(s, q0, t), F_or) <= 1e-5
    dt = inputs.cfl_dt_3d(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 1)
    q_or, x_or = o.step(q0, o.X.copy(), 0.0, dt)
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-14)
    q_gpu = s.fields()[0]
    assert rel_err(q_gpu, q_or) <= 1e-5
    assert rel_err(q_gpu - REST[None, :, None], q_or - REST[None, :, None]) <= 1e-4


def test_tc3_tuner_choice_is_one_of_the_two_kernels():
    """The first step of an untuned GB_MIXED solver times both 3D kernels on its own state and
    keeps one; the tuning launches leave the state alone, so the fields equal a solver fixed to
    the chosen kernel bit for bit."""
    mesh, o = channel((5, 3, 3), 3, jitter=0.05)
    q0 = oracle_state(o, o.X, lambda x, y, z: inputs.channel_flow_3d(x, y, z, 0.1))
    dt = inputs.cfl_dt_3d(mesh, 3, o.c, 0.5)
    tuned = mixed_solver(mesh, 3)
    assert tuned.launch_config() == TC_DEFAULT[3]      # before the first step
    tuned.set_fields(q0, 0.0)
    tuned.step(dt, 4)
    pick = tuned.launch_config()
    assert pick in (TC_DEFAULT[3], SIMT)
    fixed = mixed_solver(mesh, 3, pick)
    fixed.set_fields(q0, 0.0)
    fixed.step(dt, 4)
    qa, ta = tuned.fields()
    qb, tb = fixed.fields()
    assert ta == tb
    np.testing.assert_array_equal(qa, qb)
    q_or, _, _ = o.run(q0, o.X.copy(), 0.0, dt, 4)
    assert rel_err(qa, q_or) <= 1e-5
