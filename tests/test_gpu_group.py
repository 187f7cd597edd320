"""GPU tests of batched stepping (gb_group_step) and of the continuous-batching
serving loop: each request's result is the same alone and in the mix."""
import numpy as np
import pytest

from paper_2607_00199_b300 import inputs, state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from paper_2607_00199_b300 import gb, serve  # noqa: E402

STREAM = None


def _stream():
    global STREAM
    if STREAM is None:
        STREAM = torch.cuda.Stream()
    return STREAM.cuda_stream


def _solver(n, N, A, T, Re, jitter=0.1, precision=gb.GB_MIXED, shape=None):
    # shape 4: alone on the same warp-tile kernel as the group (bitwise comparable)
    mesh = inputs.periodic_square_mesh(n, jitter=jitter)
    s = gb.Solver(mesh, N, 0.1, Re, precision=precision, stream=_stream())
    if shape is not None:
        s.set_launch_config(shape)
    s.set_motion(A, T)
    xy = s.nodes()
    rho, u, v = inputs.taylor_green(xy[..., 0], xy[..., 1], 0.1)
    q0 = state.equilibrium_fields(rho, u, v, s.c)
    s.set_fields(q0, 0.0)
    return s, q0, inputs.cfl_dt(mesh, N, s.c, 0.5)


@pytest.mark.parametrize('N', [3, 4])
def test_group_step_is_bitwise_equal_to_alone(N):
    specs = [(5, 0.05, 1.0, 100.0), (9, 0.03, 0.7, 500.0), (12, 0.08, 1.6, 1500.0)]
    grouped = [_solver(n, N, A, T, Re) for (n, A, T, Re) in specs]
    g = gb.Group(8, _stream())
    g.step([s for s, _, _ in grouped], [dt for _, _, dt in grouped], 15)
    for (n, A, T, Re), (sg, q0, dt) in zip(specs, grouped):
        qg, tg = sg.fields()
        xg = sg.vertices()
        sa, _, dta = _solver(n, N, A, T, Re, shape=4)
        assert dta == dt
        sa.step(dt, 15)
        qa, ta = sa.fields()
        assert ta == tg
        assert np.array_equal(qa, qg)
        assert np.array_equal(sa.vertices(), xg)
        sa.close()
        sg.close()
    g.close()


def test_group_records_diagnostics_like_alone():
    specs = [(5, 0.05, 1.0, 100.0), (8, 0.03, 0.7, 500.0)]
    grouped = [_solver(n, 3, A, T, Re) for (n, A, T, Re) in specs]
    grouped[0][0].set_diagnostics(1, 32)
    grouped[1][0].set_diagnostics(2, 32)
    g = gb.Group(4, _stream())
    g.step([s for s, _, _ in grouped], [dt for _, _, dt in grouped], 6)
    for (n, A, T, Re), (sg, _, dt), every in zip(specs, grouped, (1, 2)):
        sa, _, _ = _solver(n, 3, A, T, Re, shape=4)
        sa.set_diagnostics(every, 32)
        sa.step(dt, 6)
        hg, ha = sg.diagnostics_history(), sa.diagnostics_history()
        assert hg['total'] == ha['total'] == 6 // every
        assert np.array_equal(hg['t'], ha['t'])
        # alone, the record is fused into the last stage kernel; in a group it is a separate
        # reduction: the same integrals of the same (bitwise equal) states, summed in another order
        for key in ('mass', 'kinetic_energy', 'momentum_x', 'momentum_y', 'area'):
            np.testing.assert_allclose(hg[key], ha[key], rtol=1e-13, atol=1e-13 * float(ha['mass'].max()), err_msg=key)
        q_g, _ = sg.fields()
        q_a, _ = sa.fields()
        np.testing.assert_array_equal(q_g, q_a)
        sa.close()
        sg.close()
    g.close()


def test_group_rejects_mismatched_members():
    a, _, dta = _solver(4, 2, 0.05, 1.0, 100.0)
    b, _, dtb = _solver(4, 3, 0.05, 1.0, 100.0)
    c, _, dtc = _solver(4, 2, 0.05, 1.0, 100.0, precision=gb.GB_FP64)
    g = gb.Group(4, _stream())
    for members, dts in (([a, b], [dta, dtb]), ([a, c], [dta, dtc])):
        with pytest.raises(gb.GBError) as ei:
            g.step(members, dts, 1)
        assert ei.value.code == gb.GB_EINVAL
    with pytest.raises(gb.GBError):
        g.step([a], [-1.0], 1)
    g.close()


def test_predicted_footprint_is_conservative():
    for n, N in ((32, 2), (16, 5), (64, 4)):
        s, _, _ = _solver(n, N, 0.05, 1.0, 100.0, jitter=0.0)
        s.fields()
        s.diagnostics()
        assert serve.predicted_device_bytes(2 * n * n, N) >= s.device_bytes
        s.close()


def test_serving_results_equal_alone_and_budget_respected():
    # a small stream: several sizes and orders, arrivals spread over ~30 ms, some
    # requests arrive while others run; the budget holds about three at a time
    # (the last one is large: a unit of its own, stepped with gb_step on its tuned shape)
    reqs = []
    sizes = [(8, 2), (12, 3), (6, 2), (10, 3), (16, 4), (8, 4), (14, 2), (128, 3)]
    for i, (n, N) in enumerate(sizes):
        reqs.append({'id': i, 'arrival': 0.005 * i, 'n': n, 'N': N, 'A': 0.02 + 0.01 * i,
                     'T': 0.6 + 0.2 * i, 'Re': 150.0 + 200.0 * i, 'Ma': 0.1, 'K': 2 * n * n})
    budget = 3 * serve.predicted_device_bytes(2 * 16 * 16, 4) + serve.predicted_device_bytes(2 * 128 * 128, 3)
    setup = torch.cuda.Stream()
    srv = serve.Server(budget, _stream(), steps_per_request=12, keep_fields=True, setup_stream=setup.cuda_stream,
                       alone_ms={(2 * n * n, N): 1.0 for n, N in sizes})
    stats = srv.run(reqs)
    assert stats['peak_device_bytes'] <= budget
    assert set(srv.results) == set(range(len(reqs)))
    assert stats['slowdown_vs_alone']['p50'] > 0
    for spec in reqs:
        rq = serve.Request(spec, _stream())
        if spec['K'] < srv.large_k:
            rq.solver.set_launch_config(4)   # the warp-tile kernel of the groups
        rq.solver.step(rq.dt, 12)
        q_alone, _ = rq.solver.fields()
        rq.solver.close()
        q_mix = srv.results[spec['id']]
        rel = np.linalg.norm(q_mix - q_alone) / np.linalg.norm(q_alone)
        assert rel <= 1e-5, (spec['id'], rel)
        assert np.array_equal(q_mix, q_alone)
    assert stats['step_latency_ms']['p99'] >= stats['step_latency_ms']['p50'] > 0



@pytest.mark.parametrize('N', [2, 4])
def test_group_shapes_are_bitwise_equal_and_tuned(N):
    # the group kernel's warps per CTA (4, 2, 1) change only which warp takes which tile: the
    # same results bit for bit; untuned, the group picks one of them
    specs = [(5, 0.05, 1.0, 100.0), (9, 0.03, 0.7, 500.0)]
    outs = []
    for w in (4, 2, 1, None):
        grouped = [_solver(n, N, A, T, Re) for (n, A, T, Re) in specs]
        g = gb.Group(4, _stream())
        if w:
            g.set_launch_config(N, w)
        g.step([s for s, _, _ in grouped], [dt for _, _, dt in grouped], 5)
        assert g.launch_config(N) == w if w else g.launch_config(N) in (1, 2, 4)
        outs.append([s.fields()[0] for s, _, _ in grouped])
        for s, _, _ in grouped:
            s.close()
        g.close()
    for o in outs[1:]:
        for qa, qb in zip(o, outs[0]):
            assert np.array_equal(qa, qb)
    g = gb.Group(2, _stream())
    with pytest.raises(gb.GBError):
        g.set_launch_config(N, 3)
    g.close()
