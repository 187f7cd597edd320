"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs.

Tolerances (FP64 path): relative L2 <= 1e-12 for one right-hand side and
<= 1e-10 after 100 SARK steps.  Mixed path: relative L2 of the fields against
the FP64 oracle <= 1e-5 (also reported relative to the perturbation size).
"""
import math

import numpy as np
import pytest

from oracle import physics
from oracle.solver import Motion, OracleSolver
from paper_2607_00199_b300 import inputs
from parity_metrics import rel_err, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from paper_2607_00199_b300 import gb  # noqa: E402  (loads libgb.so; fails loudly if missing)

REST = np.array([1.0, 0, 0, 0, 0, 0])




def oracle_state(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v = flow(xn[..., 0], xn[..., 1])
    return np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))


def make_pair(n, N, Ma, Re, A, T, jitter=0.0, precision=gb.GB_FP64, L=2 * math.pi):
    mesh = inputs.periodic_square_mesh(n, L=L, jitter=jitter)
    o = OracleSolver(mesh, N, Ma=Ma, Re=Re, motion=Motion(A, T, L, L))
    s = gb.Solver(mesh, N, Ma, Re, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    s.set_motion(A, T, L, L)
    return mesh, o, s


def gpu_rhs(s, q, t):
    dt = torch.float64 if s.precision == gb.GB_FP64 else torch.float32
    qq = q - REST[None, :, None] if s.precision == gb.GB_MIXED else q
    qd = torch.from_numpy(np.ascontiguousarray(qq)).to('cuda', dt)
    Fd = torch.empty_like(qd)
    s.rhs(t, qd, Fd)
    torch.cuda.synchronize()
    return Fd.double().cpu().numpy()


@pytest.mark.parametrize('N', [1, 2, 3, 4, 5, 6])
def test_rhs_parity_all_orders_ragged(N):
    # n = 5: K = 50 elements, not a multiple of any tile size; jittered, moved vertices
    mesh, o, s = make_pair(5, N, 0.1, 100.0, 0.05, 1.0, jitter=0.1)
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = oracle_state(o, xv, lambda x, y: inputs.random_flow(x, y, 11 + N))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    F_gpu = gpu_rhs(s, q, t)
    assert rel_err(F_gpu, F_or) <= 1e-12
    for f in range(6):
        assert rel_err(F_gpu[:, f], F_or[:, f]) <= 1e-11, f


def test_rhs_parity_cfg1():
    # 2D moving Taylor-Green vortex: 16x16 quads -> K = 512, N = 3, Ma 0.1, Re 100
    mesh, o, s = make_pair(16, 3, 0.1, 100.0, 0.05, 1.0)
    t = 0.17
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = oracle_state(o, xv, lambda x, y: inputs.taylor_green(x, y, 0.1))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    assert rel_err(gpu_rhs(s, q, t), F_or) <= 1e-12


def test_nodes_match_oracle():
    mesh, o, s = make_pair(6, 4, 0.1, 100.0, 0.05, 1.0, jitter=0.1)
    xv = o.X + o.motion.displacement(o.X, 0.2)
    s.set_vertices(xv)
    np.testing.assert_allclose(s.nodes(), o.node_coords(xv), atol=1e-14)


def run_both(n, N, Ma, Re, A, T, nsteps, flow, jitter=0.0, precision=gb.GB_FP64, cfl=0.5):
    mesh, o, s = make_pair(n, N, Ma, Re, A, T, jitter=jitter, precision=precision)
    q0 = oracle_state(o, o.X, flow)
    dt = inputs.cfl_dt(mesh, N, o.c, cfl)
    s.set_fields(q0, 0.0)
    s.step(dt, nsteps)
    q_gpu, t_gpu = s.fields()
    x_gpu = s.vertices()
    q_or, x_or, t_or = o.run(q0, o.X.copy(), 0.0, dt, nsteps)
    return q_gpu, q_or, x_gpu, x_or, t_gpu, t_or, q0


def test_step_parity_cfg1_100_steps():
    tg = lambda x, y: inputs.taylor_green(x, y, 0.1)
    q_gpu, q_or, x_gpu, x_or, t_gpu, t_or, q0 = run_both(16, 3, 0.1, 100.0, 0.05, 1.0, 100, tg)
    assert abs(t_gpu - t_or) <= 1e-15 * max(1.0, t_or)
    np.testing.assert_allclose(x_gpu, x_or, atol=1e-13)
    assert rel_err(q_gpu, q_or) <= 1e-10
    assert rel_err(q_gpu - REST[None, :, None], q_or - REST[None, :, None]) <= 1e-10


@pytest.mark.parametrize('u0,v0', [(1.0, 0.0), (1.0, 1.0)])
def test_free_stream_gcl_gpu(u0, v0):
    fs = lambda x, y: inputs.free_stream(x, y, u0, v0)
    q_gpu, q_or, x_gpu, x_or, t_gpu, t_or, q0 = run_both(16, 3, 0.1, 100.0, 0.05, 1.0, 100, fs)
    assert np.abs(x_gpu - x_or).max() < 1e-13 and np.abs(x_gpu - mesh_X(16)).max() > 1e-3
    assert np.abs(q_gpu - q0).max() <= 1e-13


def mesh_X(n):
    return inputs.periodic_square_mesh(n)['X']


def test_full_size_cfg2_rhs_and_step():
    # 256x256 quads -> K = 131072 jittered triangles, N = 4, Ma 0.1, Re 1000: the benchmark workload
    mesh, o, s = make_pair(256, 4, 0.1, 1000.0, 0.05, 1.0, jitter=0.1)
    q0 = oracle_state(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1))
    t = 0.0
    F_or = o.rhs(q0, o.X, o.motion.velocity(o.X, t))
    assert rel_err(gpu_rhs(s, q0, t), F_or) <= 1e-12
    dt = inputs.cfl_dt(mesh, 4, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 1)
    q_gpu, _ = s.fields()
    q_or, x_or = o.step(q0, o.X.copy(), 0.0, dt)
    assert rel_err(q_gpu, q_or) <= 1e-11
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-13)


@pytest.mark.parametrize('N', [2, 5])
def test_step_parity_other_orders(N):
    flow = lambda x, y: inputs.random_flow(x, y, 3)
    q_gpu, q_or, *_ = run_both(7, N, 0.1, 300.0, 0.04, 0.6, 20, flow, jitter=0.1)
    assert rel_err(q_gpu, q_or) <= 1e-10


def test_smallest_mesh():
    # n = 3: K = 18, every element is on the periodic boundary
    flow = lambda x, y: inputs.random_flow(x, y, 5)
    q_gpu, q_or, *_ = run_both(3, 3, 0.1, 100.0, 0.05, 1.0, 10, flow)
    assert rel_err(q_gpu, q_or) <= 1e-11


def test_mixed_precision_error_cfg1():
    tg = lambda x, y: inputs.taylor_green(x, y, 0.1)
    q_gpu, q_or, x_gpu, x_or, *_ = run_both(16, 3, 0.1, 100.0, 0.05, 1.0, 100, tg, precision=gb.GB_MIXED)
    np.testing.assert_allclose(x_gpu, x_or, atol=1e-13)     # geometry stays FP64
    assert rel_err(q_gpu, q_or) <= 1e-5
    assert rel_err(q_gpu - REST[None, :, None], q_or - REST[None, :, None]) <= 1e-5


@pytest.mark.parametrize('N', [1, 2, 3, 4, 5, 6])
def test_mixed_rhs_all_orders_ragged(N):
    # K = 50: two 32-element interleave blocks, the second one partly padding
    mesh, o, s = make_pair(5, N, 0.1, 100.0, 0.05, 1.0, jitter=0.1, precision=gb.GB_MIXED)
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = oracle_state(o, xv, lambda x, y: inputs.random_flow(x, y, 21 + N))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    F_gpu = gpu_rhs(s, q, t)
    assert rel_err(F_gpu, F_or) <= 1e-5
    for f in range(6):
        assert rel_err(F_gpu[:, f], F_or[:, f]) <= 1e-4, f


@pytest.mark.parametrize('N', [2, 4, 5])
def test_mixed_step_other_orders(N):
    flow = lambda x, y: inputs.random_flow(x, y, 4)
    q_gpu, q_or, *_ = run_both(7, N, 0.1, 300.0, 0.04, 0.6, 20, flow, jitter=0.1, precision=gb.GB_MIXED)
    assert rel_err(q_gpu - REST[None, :, None], q_or - REST[None, :, None]) <= 1e-5


def test_mixed_full_size_cfg2_step():
    mesh, o, s = make_pair(256, 4, 0.1, 1000.0, 0.05, 1.0, jitter=0.1, precision=gb.GB_MIXED)
    q0 = oracle_state(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1))
    dt = inputs.cfl_dt(mesh, 4, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 2)
    q_gpu, _ = s.fields()
    q_or, x_or, _ = o.run(q0, o.X.copy(), 0.0, dt, 2)
    assert rel_err(q_gpu - REST[None, :, None], q_or - REST[None, :, None]) <= 1e-5
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-13)


def test_mixed_checkpoint_and_status():
    mesh, o, s = make_pair(9, 3, 0.1, 100.0, 0.05, 1.0, jitter=0.1, precision=gb.GB_MIXED)
    q0 = oracle_state(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1))
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    q_back, _ = s.fields()
    # the FP32 perturbation round trip keeps rho to ~1e-8
    assert np.abs(q_back - q0).max() < 1e-7
    s.step(dt, 10)
    q10, t10 = s.fields()
    s.set_fields(q0, 0.0)
    s.set_vertices(o.X)
    s.step(dt, 10)
    assert np.array_equal(s.fields()[0], q10)
    bad = q0.copy()
    bad[5, 4, 2] = np.inf
    s.set_fields(bad, 0.0)
    s.step(dt, 1)
    with pytest.raises(gb.GBError) as ei:
        s.fields()
    assert ei.value.code == gb.GB_ENAN


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
@pytest.mark.parametrize('N', [2, 4])
def test_diagnostics_parity(precision, N):
    # Sec. 7.2 kinetic energy and the conserved integrals of the GPU state after
    # a few steps (ragged K = 98, jittered, moved mesh) against the oracle's on
    # the same fields and vertices; both reduce in FP64
    mesh, o, s = make_pair(7, N, 0.1, 200.0, 0.05, 1.0, jitter=0.1, precision=precision)
    q0 = oracle_state(o, o.X, lambda x, y: inputs.random_flow(x, y, 5 + N))
    s.set_fields(q0, 0.0)
    d0 = s.diagnostics()
    want0 = o.diagnostics(s.fields()[0], s.vertices())
    s.step(inputs.cfl_dt(mesh, N, o.c, 0.5), 7)
    d1 = s.diagnostics()
    want1 = o.diagnostics(s.fields()[0], s.vertices())
    for d, want in ((d0, want0), (d1, want1)):
        for k in want:
            assert abs(d[k] - want[k]) <= 1e-13 * max(1.0, abs(want[k])), (k, d[k], want[k])
    # the stepping itself conserves mass to rounding over such a short run
    assert abs(d1['mass'] - d0['mass']) <= (1e-11 if precision == gb.GB_FP64 else 1e-5) * d0['mass']
    assert s.diagnostics() == d1        # deterministic reduction order


def test_diagnostics_full_size_cfg2():
    # K = 131072, N = 4 moving Taylor-Green vortex: closed forms at t = 0
    # (mass 4 pi^2, E_K = 1/4) and oracle parity on the stepped state
    for precision in (gb.GB_FP64, gb.GB_MIXED):
        mesh, o, s = make_pair(256, 4, 0.1, 1000.0, 0.05, 1.0, jitter=0.1, precision=precision)
        s.set_fields(oracle_state(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1)), 0.0)
        d = s.diagnostics()
        tol = 1e-12 if precision == gb.GB_FP64 else 1e-6
        assert abs(d['mass'] - 4 * math.pi ** 2) <= tol * 40 and abs(d['kinetic_energy'] - 0.25) <= tol
        s.step(inputs.cfl_dt(mesh, 4, o.c, 0.5), 3)
        d = s.diagnostics()
        want = o.diagnostics(s.fields()[0], s.vertices())
        for k in want:
            assert abs(d[k] - want[k]) <= 1e-12 * max(1.0, abs(want[k])), (precision, k)
        s.close()


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_diagnostics_history_equals_on_demand(precision):
    # records taken inside the step (fused into the last stage kernel, and its CUDA graph) equal
    # gb_diagnostics after each step taken one by one: the same times bit for bit, the same
    # integrals up to the order of the FP64 summation (1e-13 relative)
    mesh, o, a = make_pair(6, 3, 0.1, 200.0, 0.05, 1.0, jitter=0.1, precision=precision)
    b = gb.Solver(mesh, 3, 0.1, 200.0, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    b.set_motion(0.05, 1.0)
    if precision == gb.GB_MIXED:
        # the fused record runs the last stage on the 4-warp kernel: both solvers on that
        # kernel, so that their states stay bitwise equal
        a.set_launch_config(4)
        b.set_launch_config(4)
    q0 = oracle_state(o, o.X, lambda x, y: inputs.random_flow(x, y, 21))
    a.set_fields(q0, 0.0)
    b.set_fields(q0, 0.0)
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    a.set_diagnostics(1, 64)
    a.step(dt, 10)
    h = a.diagnostics_history()
    assert h['total'] == 10 and len(h['t']) == 10
    for k in range(10):
        b.step(dt, 1)
        d = b.diagnostics()
        assert h['t'][k] == b.fields()[1]
        for key in d:
            assert abs(h[key][k] - d[key]) <= 1e-13 * (abs(d[key]) + d['mass']), (k, key, h[key][k], d[key])
    # every 3rd step into a ring of 2: the records of steps 3, 6, 9 were written, 6 and 9 kept
    a.set_diagnostics(3, 2)
    t0 = a.fields()[1]
    a.step(dt, 10)
    h = a.diagnostics_history()
    assert h['total'] == 3 and len(h['t']) == 2
    assert np.allclose(h['t'], [t0 + 6 * dt, t0 + 9 * dt], rtol=0, atol=1e-12)
    a.set_diagnostics(0)
    assert len(a.diagnostics_history()['t']) == 0
    with pytest.raises(gb.GBError):
        a.set_diagnostics(-1)
    with pytest.raises(gb.GBError):
        a.set_diagnostics(1, 0)


def test_recorded_kinetic_energy_follows_oracle():
    # Sec. 7.2 E_K(t) of a moving Taylor-Green vortex, recorded every step on the GPU
    # (FP64 path), against the oracle's integrals of the oracle's own run
    mesh, o, s = make_pair(5, 3, 0.1, 50.0, 0.05, 1.0, jitter=0.1)
    q = oracle_state(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1))
    s.set_fields(q, 0.0)
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    s.set_diagnostics(1, 16)
    s.step(dt, 8)
    h = s.diagnostics_history()
    xv, t = o.X.copy(), 0.0
    for k in range(8):
        q, xv = o.step(q, xv, t, dt)
        t += dt
        d = o.diagnostics(q, xv)
        assert abs(h['t'][k] - t) <= 1e-14 * max(1.0, t)
        for key in ('mass', 'kinetic_energy', 'momentum_x', 'momentum_y', 'area'):
            assert abs(h[key][k] - d[key]) <= 1e-12 * max(1.0, abs(d[key])), (k, key)
    assert h['kinetic_energy'][-1] < h['kinetic_energy'][0]     # viscous decay


def test_mixed_rhs_matches_fp64_rhs():
    mesh, o, s = make_pair(8, 4, 0.1, 100.0, 0.05, 1.0, jitter=0.1, precision=gb.GB_MIXED)
    xv = o.X + o.motion.displacement(o.X, 0.1)
    s.set_vertices(xv)
    q = oracle_state(o, xv, lambda x, y: inputs.taylor_green(x, y, 0.1))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, 0.1))
    assert rel_err(gpu_rhs(s, q, 0.1), F_or) <= 1e-5


def test_nan_is_reported():
    mesh, o, s = make_pair(6, 3, 0.1, 100.0, 0.0, 1.0)
    q = oracle_state(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1))
    q[3, 2, 1] = np.nan
    s.set_fields(q, 0.0)
    s.step(1e-4, 2)
    with pytest.raises(gb.GBError) as ei:
        s.fields()
    assert ei.value.code == gb.GB_ENAN
    s.set_fields(oracle_state(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1)), 0.0)
    s.step(1e-4, 1)
    s.fields()       # status was cleared; the solver is usable again


def test_tangled_mesh_is_reported():
    # amplitude larger than the cell size tangles the mesh within a quarter period
    mesh, o, s = make_pair(8, 2, 0.1, 100.0, 1.5, 1.0)
    s.set_fields(oracle_state(o, o.X, lambda x, y: inputs.free_stream(x, y)), 0.0)
    s.step(0.01, 30)
    with pytest.raises(gb.GBError) as ei:
        s.fields()
    assert ei.value.code == gb.GB_EMESH


def test_checkpoint_resume_is_bitwise():
    mesh, o, s = make_pair(10, 3, 0.1, 100.0, 0.05, 1.0, jitter=0.1)
    q0 = oracle_state(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1))
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 100)
    q100, t100 = s.fields()
    s.set_fields(q0, 0.0)
    s.set_vertices(o.X)
    s.step(dt, 50)
    q50, t50 = s.fields()
    x50 = s.vertices()
    s2 = gb.Solver(mesh, 3, 0.1, 100.0, stream=torch.cuda.current_stream().cuda_stream)
    s2.set_motion(0.05, 1.0)
    s2.set_fields(q50, t50)
    s2.set_vertices(x50)
    s2.step(dt, 50)
    q100b, t100b = s2.fields()
    assert t100b == t100
    assert np.array_equal(q100b, q100)


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_graph_steps_equal_direct_steps(precision):
    # gb_step on a non-default stream replays one captured step; it must match direct launches
    stream = torch.cuda.Stream()
    mesh = inputs.periodic_square_mesh(9, jitter=0.1)
    outs = []
    for use_graph in (True, False):
        s = gb.Solver(mesh, 3, 0.1, 200.0, precision=precision, stream=stream.cuda_stream)
        s.set_graph(use_graph)
        s.set_motion(0.05, 0.8)
        xy = s.nodes()
        rho, u, v = inputs.taylor_green(xy[..., 0], xy[..., 1], 0.1)
        from paper_2607_00199_b300 import state
        s.set_fields(state.equilibrium_fields(rho, u, v, s.c), 0.0)
        dt = inputs.cfl_dt(mesh, 3, s.c, 0.5)
        s.step(dt, 7)
        s.step(dt * 0.9, 5)          # a new dt rebuilds the graph
        outs.append(s.fields() + (s.vertices(),))
        s.close()
    (qa, ta, xa), (qb, tb, xb) = outs
    assert ta == tb and np.array_equal(qa, qb) and np.array_equal(xa, xb)


@pytest.mark.parametrize('N', [3, 4])
def test_launch_shapes_give_identical_results_and_tuner_picks_one(N):
    # every shape computes the same tiles in the same order: bitwise equal results
    stream = torch.cuda.Stream()
    mesh = inputs.periodic_square_mesh(11, jitter=0.1)
    from paper_2607_00199_b300 import state
    outs = []
    shapes = [1, 2, 4]          # the mma.sync kernel's warp tiles: the same tiles, bitwise equal
    for w in shapes + [None]:
        s = gb.Solver(mesh, N, 0.1, 300.0, precision=gb.GB_MIXED, stream=stream.cuda_stream)
        if w is not None:
            s.set_launch_config(w)
        s.set_motion(0.04, 0.9)
        xy = s.nodes()
        rho, u, v = inputs.taylor_green(xy[..., 0], xy[..., 1], 0.1)
        s.set_fields(state.equilibrium_fields(rho, u, v, s.c), 0.0)
        dt = inputs.cfl_dt(mesh, N, s.c, 0.5)
        s.step(dt, 6)
        q, t = s.fields()
        if w is None:
            picked = s.launch_config()
            assert picked in shapes + [8]
        else:
            assert s.launch_config() == w
            outs.append(q)
        s.close()
    for q in outs[1:]:
        assert np.array_equal(q, outs[0])
    with pytest.raises(gb.GBError):
        f = gb.Solver(mesh, 2, 0.1, 100.0, precision=gb.GB_FP64, stream=stream.cuda_stream)
        f.set_launch_config(2)
    for bad in (3, 5, 0, 16):
        with pytest.raises(gb.GBError):
            gb.Solver(mesh, N, 0.1, 100.0, precision=gb.GB_MIXED, stream=stream.cuda_stream).set_launch_config(bad)


# ---- the tcgen05 kernel (launch shape 8: 128-element CTA tiles, tensor-memory accumulators) ----

def _um_pair(n, N, Re=100.0, A=0.05, T=1.0, jitter=0.1):
    mesh, o, s = make_pair(n, N, 0.1, Re, A, T, jitter=jitter, precision=gb.GB_MIXED)
    s.set_launch_config(8)
    return mesh, o, s


@pytest.mark.parametrize('N', [1, 2, 3, 4])
@pytest.mark.parametrize('n', [5, 11, 23])
def test_tcgen05_rhs_against_oracle(N, n):
    # K = 50 (one partial tile), 242 (one full tile and a ragged one), 1058 (8 full tiles and a
    # ragged one); neighbours inside the tile, across tiles (the halo) and across the periodic
    # boundary
    mesh, o, s = _um_pair(n, N)
    t = 0.3
    xv = o.X + o.motion.displacement(o.X, t)
    s.set_vertices(xv)
    q = oracle_state(o, xv, lambda x, y: inputs.random_flow(x, y, 41 + N + n))
    F_or = o.rhs(q, xv, o.motion.velocity(o.X, t))
    F = gpu_rhs(s, q, t)
    assert s.launch_config() == 8
    assert rel_err(F, F_or) <= 1e-5
    for f in range(6):
        assert rel_l2(F[:, f], F_or[:, f]) <= 1e-4, f


@pytest.mark.parametrize('N', [1, 2, 3, 4])
def test_tcgen05_steps_against_oracle(N):
    flow = lambda x, y: inputs.random_flow(x, y, 4)
    mesh, o, s = _um_pair(7, N, Re=300.0, A=0.04, T=0.6)
    q0 = oracle_state(o, o.X, flow)
    dt = inputs.cfl_dt(mesh, N, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 20)
    q_gpu, t_gpu = s.fields()
    q_or, x_or, t_or = o.run(q0, o.X.copy(), 0.0, dt, 20)
    assert abs(t_gpu - t_or) <= 1e-15 * max(1.0, t_or)
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-13)
    assert rel_err(q_gpu, q_or) <= 1e-5
    assert rel_err(q_gpu - REST[None, :, None], q_or - REST[None, :, None]) <= 1e-5


def test_tcgen05_full_size_rhs_and_steps():
    # the benchmark workload: K = 131072 jittered triangles, N = 4, Ma 0.1, Re 1000, 1024 tiles
    mesh, o, s = _um_pair(256, 4, Re=1000.0)
    q0 = oracle_state(o, o.X, lambda x, y: inputs.taylor_green(x, y, 0.1))
    F_or = o.rhs(q0, o.X, o.motion.velocity(o.X, 0.0))
    assert rel_err(gpu_rhs(s, q0, 0.0), F_or) <= 1e-5
    dt = inputs.cfl_dt(mesh, 4, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, 2)
    q_gpu, _ = s.fields()
    q_or, x_or, _ = o.run(q0, o.X.copy(), 0.0, dt, 2)
    assert rel_err(q_gpu, q_or) <= 1e-5
    assert rel_err(q_gpu - REST[None, :, None], q_or - REST[None, :, None]) <= 1e-5
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-13)


def test_tcgen05_graph_replay_and_repeats_are_bitwise():
    # the kernel's arithmetic order is fixed (one issuing thread per accumulator, fixed
    # k-step order): repeated runs, graph replay and direct launches agree bit for bit
    mesh = inputs.periodic_square_mesh(20, jitter=0.1)
    outs = []
    for graph in (True, False, True):
        s = gb.Solver(mesh, 4, 0.1, 300.0, precision=gb.GB_MIXED, stream=torch.cuda.current_stream().cuda_stream)
        s.set_launch_config(8)
        s.set_graph(graph)
        s.set_motion(0.04, 0.9)
        xy = s.nodes()
        from paper_2607_00199_b300 import state
        rho, u, v = inputs.taylor_green(xy[..., 0], xy[..., 1], 0.1)
        s.set_fields(state.equilibrium_fields(rho, u, v, s.c), 0.0)
        s.step(inputs.cfl_dt(mesh, 4, s.c, 0.5), 7)
        outs.append(s.fields()[0])
        s.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_tcgen05_status_nan_and_tangle():
    mesh, o, s = _um_pair(6, 3, A=0.0)
    q0 = oracle_state(o, o.X, lambda x, y: inputs.random_flow(x, y, 2))
    q0[3, 2, 4] = np.nan
    s.set_fields(q0, 0.0)
    s.step(1e-4, 1)
    with pytest.raises(gb.GBError) as ei:
        s.fields()
    assert ei.value.code == gb.GB_ENAN
    s.close()
    # a mesh folded by a large motion amplitude: J <= 0 is reported, not silently stepped
    mesh, o, s = _um_pair(8, 2, A=1.5, T=1.0, jitter=0.0)
    s.set_fields(oracle_state(o, o.X, lambda x, y: inputs.free_stream(x, y)), 0.0)
    s.step(0.01, 30)
    with pytest.raises(gb.GBError) as ei:
        s.fields()
    assert ei.value.code == gb.GB_EMESH
    s.close()


def test_tcgen05_full_size_25_steps_against_fp64():
    # 1024 tiles over 148 CTAs: every CTA runs several tiles back to back, which exercises the
    # cross-tile prefetches and hand-offs that one-tile meshes do not.  The mixed error after 25
    # steps is ~4e-8 of the fields (~5e-7 of the perturbation); the bound catches any tile
    # whose staged data or tensor-memory columns are reused too early
    from paper_2607_00199_b300 import state
    mesh = inputs.periodic_square_mesh(256, jitter=0.1)
    out = {}
    for prec, shape in ((gb.GB_FP64, None), (gb.GB_MIXED, 8)):
        s = gb.Solver(mesh, 4, 0.1, 1000.0, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
        if shape:
            s.set_launch_config(shape)
        s.set_motion(0.05, 1.0)
        xy = s.nodes()
        rho, u, v = inputs.taylor_green(xy[..., 0], xy[..., 1], 0.1)
        s.set_fields(state.equilibrium_fields(rho, u, v, s.c), 0.0)
        s.step(inputs.cfl_dt(mesh, 4, s.c, 0.5), 25)
        out[prec] = s.fields()[0]
        s.close()
    qf, qm = out[gb.GB_FP64], out[gb.GB_MIXED]
    assert rel_err(qm, qf) <= 1e-6
    assert rel_err(qm - REST[None, :, None], qf - REST[None, :, None]) <= 1e-5
