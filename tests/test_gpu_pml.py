"""GPU parity of the perfectly matched layer (the reading of oracle/pml.py) through the C ABI
(gb_set_pml): the fields q and the auxiliary fields Phi after SARK steps against the FP64
oracle on the same seeded inputs, for a uniform layer on a periodic moving mesh, the radial
layer of the plunging O-grid and slab layers at the far-field ends of a channel.
Tolerances as for the stage kernels: FP64 1e-10 after steps, GB_MIXED 1e-5 (relative L2)."""
import math

import numpy as np
import pytest

from oracle import physics
from oracle.pml import PML, sigma_max_for_reflection
from oracle.solver import Motion, OracleSolver
from paper_2607_00199_b300 import inputs
from parity_metrics import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from paper_2607_00199_b300 import gb  # noqa: E402

KINDS = {'radial': gb.GB_PML_RADIAL, 'slab': gb.GB_PML_SLAB, 'uniform': gb.GB_PML_UNIFORM}




def oracle_state(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v = flow(xn[..., 0], xn[..., 1])
    return np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))


def set_layer(s, pml):
    s.set_pml(KINDS[pml.kind], centre=tuple(pml.centre), r0=pml.r0, d=pml.d, sigma_max=pml.sigma_max,
              power=pml.power, alpha=pml.alpha, direction=tuple(pml.direction))


def run_pair(mesh, N, pml, precision, motion, flow, steps, Re=200.0, far=(1.0, 1.0, 0.0), kind='sinxy'):
    o = OracleSolver(mesh, N, Ma=0.1, Re=Re, motion=Motion(*motion, kind=kind), far_state=far, pml=pml)
    kw = {'far_state': far} if 'bc' in mesh else {}
    s = gb.Solver(mesh, N, 0.1, Re, precision=precision, stream=torch.cuda.current_stream().cuda_stream, **kw)
    s.set_motion(*motion, kind=gb.GB_MOTION_PLUNGE if kind == 'plunge' else None)
    set_layer(s, pml)
    q0 = oracle_state(o, o.X, flow)
    dt = inputs.cfl_dt(mesh, N, o.c, 0.5)
    s.set_fields(q0, 0.0)
    s.step(dt, steps)
    q_gpu, _ = s.fields()
    phi_gpu, ids = s.pml_fields()
    q_or, phi_or, x_or, _ = o.run_pml(q0, np.zeros_like(q0), o.X.copy(), 0.0, dt, steps)
    np.testing.assert_array_equal(ids, np.nonzero(o.pml_layer)[0])
    np.testing.assert_allclose(s.vertices(), x_or, atol=1e-14)
    return q_gpu, q_or, phi_gpu, phi_or[o.pml_layer], q0, s, o


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
@pytest.mark.parametrize('N', [2, 3, 4])
def test_uniform_layer_on_a_moving_periodic_mesh(N, precision):
    mesh = inputs.periodic_square_mesh(6, jitter=0.1)           # K = 72: ragged against the tiles
    pml = PML('uniform', sigma_max=2.0, alpha=0.5, direction=(0.8, 0.6))
    q, qo, phi, phio, q0, s, o = run_pair(mesh, N, pml, precision, (0.05, 1.0),
                                          lambda x, y: inputs.random_flow(x, y, 31 + N), 8)
    tol = 1e-10 if precision == gb.GB_FP64 else 1e-5
    assert rel_err(q, qo) <= tol
    assert np.abs(phio).max() > 1e-3
    assert rel_err(phi, phio) <= (1e-10 if precision == gb.GB_FP64 else 1e-4)
    assert rel_err(q - q0, qo - q0) <= (1e-9 if precision == gb.GB_FP64 else 1e-3)


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_radial_layer_on_the_plunging_airfoil(precision):
    mesh = inputs.naca_ogrid_mesh(24, 9, R=5.0, growth=1.1)
    c = 10.0
    pml = PML('radial', centre=(0.5, 0.0), r0=2.5, d=2.5, sigma_max=sigma_max_for_reflection(c, 2.5), alpha=0.2)

    def flow(x, y):
        rho, u, v = inputs.random_flow(x, y, 21, amp=0.02)
        return rho, 1.0 + 0.2 * u, 0.2 * v

    q, qo, phi, phio, q0, s, o = run_pair(mesh, 3, pml, precision, (0.25, 2.0), flow, 12, Re=1000.0, kind='plunge')
    assert 0 < len(phio) < o.K
    assert rel_err(q, qo) <= (1e-10 if precision == gb.GB_FP64 else 1e-5)
    assert rel_err(phi, phio) <= (1e-9 if precision == gb.GB_FP64 else 1e-3)


def test_slab_layers_at_the_channel_ends():
    mesh = inputs.wall_channel_mesh(12, 4, 6.0, 2.0)
    mesh['bc'] = np.where(mesh['bc'] > 0, inputs.BC_FARFIELD, 0).astype(np.int8)
    c = 10.0
    pml = PML('slab', centre=(3.0, 1.0), r0=1.5, d=1.5, direction=(1.0, 0.0), sigma_max=sigma_max_for_reflection(c, 1.5))
    # a pulse astride the right-hand layer's inner edge, so that Phi is driven from the start
    flow = lambda x, y: (1.0 + 0.01 * np.exp(-8.0 * ((x - 4.6) ** 2 + (y - 1.0) ** 2)), 0 * x, 0 * x)
    q, qo, phi, phio, q0, s, o = run_pair(mesh, 3, pml, gb.GB_FP64, (0.0, 1.0), flow, 20, far=(1.0, 0.0, 0.0))
    assert np.abs(phio).max() > 1e-4
    assert rel_err(q, qo) <= 1e-10 and rel_err(phi, phio) <= 1e-9


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_empty_layer_and_removal_leave_the_scheme_unchanged(precision):
    mesh = inputs.naca_ogrid_mesh(24, 9, R=5.0, growth=1.1)
    mk = lambda: gb.Solver(mesh, 2, 0.1, 500.0, precision=precision, far_state=(1.0, 1.0, 0.0),
                           stream=torch.cuda.current_stream().cuda_stream)
    a, b, c_ = mk(), mk(), mk()
    a.set_pml(gb.GB_PML_RADIAL, centre=(0.5, 0.0), r0=2.0, d=3.0, sigma_max=0.0)       # sigma = 0: no layer
    assert a.pml_fields()[0].shape[0] == 0
    c_.set_pml(gb.GB_PML_RADIAL, centre=(0.5, 0.0), r0=2.0, d=3.0, sigma_max=5.0)
    assert c_.pml_fields()[0].shape[0] > 0
    c_.set_pml(None)
    assert c_.pml_fields()[0].shape[0] == 0
    o = OracleSolver(mesh, 2, Ma=0.1, Re=500.0)
    q0 = oracle_state(o, o.X, lambda x, y: (1.0 + 0.01 * np.exp(-((x - 0.5) ** 2 + y ** 2)), 1.0 + 0 * x, 0 * x))
    dt = inputs.cfl_dt(mesh, 2, o.c, 0.5)
    out = []
    for s in (a, b, c_):
        s.set_fields(q0, 0.0)
        s.step(dt, 5)
        out.append(s.fields()[0])
    np.testing.assert_array_equal(out[0], out[1])
    np.testing.assert_array_equal(out[2], out[1])


def test_layer_state_resets_records_and_rejections():
    mesh = inputs.naca_ogrid_mesh(24, 9, R=5.0, growth=1.1)
    far = (1.0, 1.0, 0.0)
    s = gb.Solver(mesh, 3, 0.1, 1000.0, precision=gb.GB_MIXED, far_state=far,
                  stream=torch.cuda.current_stream().cuda_stream)
    twin = gb.Solver(mesh, 3, 0.1, 1000.0, precision=gb.GB_MIXED, far_state=far,
                     stream=torch.cuda.current_stream().cuda_stream)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=1000.0, far_state=far)
    q0 = oracle_state(o, o.X, lambda x, y: (1.0 + 0.02 * np.exp(-((x - 3.0) ** 2 + y ** 2)), 1.0 + 0 * x, 0 * x))
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    for x in (s, twin):
        x.set_pml(gb.GB_PML_RADIAL, centre=(0.5, 0.0), r0=2.5, d=2.5, sigma_max=30.0, alpha=0.1)
        x.set_fields(q0, 0.0)
    # records with a layer (separate reduction launches after the correction) equal the
    # on-demand integrals of a twin stepped one step at a time
    s.set_diagnostics(1, 8)
    s.step(dt, 4)
    h = s.diagnostics_history()
    for k in range(4):
        twin.step(dt, 1)
        d = twin.diagnostics()
        for key in d:
            assert abs(h[key][k] - d[key]) <= 1e-13 * (abs(d[key]) + d['mass']), (k, key)
    phi, _ = s.pml_fields()
    assert np.abs(phi).max() > 0
    s.set_fields(q0, 0.0)                                   # Phi back to zero
    assert np.abs(s.pml_fields()[0]).max() == 0
    with pytest.raises(gb.GBError):
        gb.Group(2).step([s], [dt], 1)
    for bad in (dict(sigma_max=-1.0), dict(d=0.0), dict(alpha=float('nan')), dict(kind=7)):
        kw = dict(kind=gb.GB_PML_RADIAL, centre=(0.5, 0.0), r0=2.5, d=2.5, sigma_max=1.0)
        kw.update(bad)
        with pytest.raises(gb.GBError) as ei:
            s.set_pml(**kw)
        assert ei.value.code == gb.GB_EINVAL
    s3 = gb.Solver(inputs.periodic_box_tet_mesh(3, 3, 3), 2, 0.1, 100.0)
    with pytest.raises(gb.GBError):
        s3.set_pml(gb.GB_PML_UNIFORM, sigma_max=1.0)


def test_full_size_airfoil_with_the_outer_layer():
    """The plunging-airfoil workload at full size (256 x 192 O-grid, K = 98304, N = 4) with
    the outer 3-chord layer (r = 17..20 about mid-chord): one SARK step of both precisions
    against the oracle on every element, q and Phi."""
    mesh = inputs.naca_ogrid_mesh(256, 192)
    c = 10.0
    pml = PML('radial', centre=(0.5, 0.0), r0=17.0, d=3.0, sigma_max=sigma_max_for_reflection(c, 3.0), alpha=1.0)
    far = (1.0, 1.0, 0.0)
    o = OracleSolver(mesh, 4, Ma=0.1, Re=1000.0, motion=Motion(0.25, 2.0, kind='plunge'), far_state=far, pml=pml)

    def flow(x, y):
        rho, u, v = inputs.random_flow(x, y, 5, amp=0.02)
        return rho, 1.0 + 0.2 * u, 0.2 * v

    q0 = oracle_state(o, o.X, flow)
    dt = inputs.cfl_dt(mesh, 4, o.c, 0.5)
    # two steps so that Phi (zero at t = 0) enters the second step's stages
    q_or, phi_or, _, _ = o.run_pml(q0, np.zeros_like(q0), o.X.copy(), 0.0, dt, 2)
    assert 0.02 * o.K < o.pml_layer.sum() < 0.2 * o.K
    for precision, tq, tp in ((gb.GB_FP64, 1e-12, 1e-10), (gb.GB_MIXED, 1e-5, 1e-3)):
        s = gb.Solver(mesh, 4, 0.1, 1000.0, precision=precision, far_state=far,
                      stream=torch.cuda.current_stream().cuda_stream)
        s.set_motion(0.25, 2.0, kind=gb.GB_MOTION_PLUNGE)
        set_layer(s, pml)
        s.set_fields(q0, 0.0)
        s.step(dt, 2)
        q, _ = s.fields()
        phi, ids = s.pml_fields()
        np.testing.assert_array_equal(ids, np.nonzero(o.pml_layer)[0])
        assert rel_err(q, q_or) <= tq
        assert rel_err(phi, phi_or[o.pml_layer]) <= tp
        s.close()


@pytest.mark.parametrize('precision', [gb.GB_FP64, gb.GB_MIXED])
def test_graph_replay_with_the_layer_equals_direct_launches(precision):
    """The layer's launches join the step's CUDA graph: replayed steps equal direct launches
    bit for bit (fields and Phi)."""
    mesh = inputs.naca_ogrid_mesh(24, 9, R=5.0, growth=1.1)
    far = (1.0, 1.0, 0.0)
    o = OracleSolver(mesh, 3, Ma=0.1, Re=1000.0, far_state=far)
    q0 = oracle_state(o, o.X, lambda x, y: (1.0 + 0.02 * np.exp(-((x - 3.0) ** 2 + y ** 2)), 1.0 + 0 * x, 0 * x))
    dt = inputs.cfl_dt(mesh, 3, o.c, 0.5)
    side = torch.cuda.Stream()
    out = []
    for graph in (True, False):
        s = gb.Solver(mesh, 3, 0.1, 1000.0, precision=precision, far_state=far, stream=side.cuda_stream)
        s.set_motion(0.25, 2.0, kind=gb.GB_MOTION_PLUNGE)
        s.set_pml(gb.GB_PML_RADIAL, centre=(0.5, 0.0), r0=2.5, d=2.5, sigma_max=30.0, alpha=0.1)
        s.set_graph(graph)
        s.set_fields(q0, 0.0)
        s.step(dt, 7)
        out.append((s.fields(), s.pml_fields()[0]))
        s.close()
    (qa, ta), pa = out[0]
    (qb, tb), pb = out[1]
    assert ta == tb
    np.testing.assert_array_equal(qa, qb)
    np.testing.assert_array_equal(pa, pb)
    assert np.abs(pa).max() > 0
