"""GPU test of gb_rhs_noalloc, the allocation-free right-hand side.

Callers whose device memory is managed by their own pool or budget cannot let
a library call cudaMalloc; gb_rhs_noalloc evaluates the GB_MIXED right-hand
side with its scratch in a static device array instead.  It runs the same
conversion and stage kernels as gb_rhs on the same data, so through the C ABI
its F must equal gb_rhs's bit for bit, on two calls in a row (the array keeps
the previous call's contents), also after a call that left non-finite values
in the array; it must refuse meshes larger than the array.

This file is named so that pytest collects it last.
"""
import pytest

from paper_2607_00199_b300 import inputs, state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from paper_2607_00199_b300 import gb  # noqa: E402


def _case(n, N, seed):
    mesh = inputs.periodic_square_mesh(n, jitter=0.1)
    s = gb.Solver(mesh, N, 0.1, 100.0, precision=gb.GB_MIXED, stream=torch.cuda.current_stream().cuda_stream)
    s.set_motion(0.05, 1.0)
    xy = s.nodes()
    rho, u, v = inputs.random_flow(xy[..., 0], xy[..., 1], seed)
    q = state.equilibrium_fields(rho, u, v, s.c)
    q[:, 0, :] -= 1.0                      # GB_MIXED takes perturbations from the rest state
    return s, torch.from_numpy(q).to('cuda', torch.float32)


def _poison_scratch():
    """A call whose input is NaN everywhere, on a mesh of another order and size: it leaves
    non-finite values in the static array where the next call's padding and tail rows sit."""
    s, qd = _case(11, 2, 7)
    F = torch.empty_like(qd)
    s.rhs_noalloc(0.1, torch.full_like(qd, float('nan')), F)
    torch.cuda.synchronize()
    assert not torch.isfinite(F).any()
    s.close()


@pytest.mark.parametrize('n,N', [(16, 3), (9, 4)])
def test_noalloc_matches_gb_rhs_on_two_calls(n, N):
    _poison_scratch()
    s, qd = _case(n, N, 31 + N)
    F_ref = torch.empty_like(qd)
    s.rhs(0.2, qd, F_ref)
    # first call (sets up the scratch address on this device), then a second one on other data
    F1 = torch.full_like(qd, float('nan'))
    s.rhs_noalloc(0.2, qd, F1)
    torch.cuda.synchronize()
    assert torch.isfinite(F1).all()
    assert torch.equal(F1, F_ref)
    q2 = qd * 0.5
    F_ref2 = torch.empty_like(qd)
    s.rhs(0.4, q2, F_ref2)
    F2 = torch.full_like(qd, float('nan'))
    s.rhs_noalloc(0.4, q2, F2)
    torch.cuda.synchronize()
    assert torch.equal(F2, F_ref2)
    assert not torch.equal(F2, F1)
    s.close()


def test_noalloc_rejects_meshes_beyond_the_array():
    # N = 4 holds at most ~22.8k elements; 128 x 128 x 2 = 32768 is beyond it
    s, qd = _case(128, 4, 3)
    F = torch.empty_like(qd)
    with pytest.raises(gb.GBError) as ei:
        s.rhs_noalloc(0.0, qd, F)
    assert ei.value.code == gb.GB_EINVAL
    assert 'static array' in str(ei.value)
    s.close()


def test_noalloc_rejects_fp64_solvers_and_bad_time():
    mesh = inputs.periodic_square_mesh(4)
    s = gb.Solver(mesh, 2, 0.1, 100.0, precision=gb.GB_FP64, stream=torch.cuda.current_stream().cuda_stream)
    q = torch.zeros((s.K, 6, s.Np), dtype=torch.float64, device='cuda')
    with pytest.raises(gb.GBError) as ei:
        s.rhs_noalloc(0.0, q, torch.empty_like(q))
    assert ei.value.code == gb.GB_EINVAL
    s.close()
    s, qd = _case(4, 2, 1)
    with pytest.raises(gb.GBError) as ei:
        s.rhs_noalloc(float('nan'), qd, torch.empty_like(qd))
    assert ei.value.code == gb.GB_EINVAL and 'finite' in str(ei.value)
    s.close()
