"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/gb.h declares, and its host-side logic (reference operators, SARK
coefficients, argument and mesh validation) agrees with the oracle.  No call
here launches a kernel."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import operators, sark
from paper_2607_00199_b300 import gb, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, 'include', 'gb.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return sorted(set(re.findall(r'\b(gb_[a-z0-9_]+)\s*\(', src)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(gb.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def _lib_fmask(L, N):
    """Face node -> volume node map of the library's documented counter-clockwise order."""
    r, s = L['r'], L['s']
    faces = [np.nonzero(np.abs(s + 1) < 1e-10)[0], np.nonzero(np.abs(r + s) < 1e-10)[0], np.nonzero(np.abs(r + 1) < 1e-10)[0]]
    keys = [r, s, -s]            # position along each face in the counter-clockwise direction
    return [f[np.argsort(k[f])] for f, k in zip(faces, keys)]


@pytest.mark.parametrize('N', range(1, 7))
def test_reference_operators_match_oracle(N):
    L = gb.reference_operators(N)
    ref = operators.ReferenceElement(N)
    np.testing.assert_allclose(L['r'], ref.r, atol=1e-15)
    np.testing.assert_allclose(L['s'], ref.s, atol=1e-15)
    np.testing.assert_allclose(L['Dr'], ref.Dr, atol=1e-13 * N * N)
    np.testing.assert_allclose(L['Ds'], ref.Ds, atol=1e-13 * N * N)
    assert L['Nc'] == ref.Nc
    np.testing.assert_allclose(L['cr'], ref.cr, atol=1e-15)
    np.testing.assert_allclose(L['cs'], ref.cs, atol=1e-15)
    np.testing.assert_allclose(L['cw'], ref.cw, atol=1e-15)
    np.testing.assert_allclose(L['I'], ref.I, atol=1e-14)
    np.testing.assert_allclose(L['P'], ref.P, atol=1e-13)
    # LIFT columns: library face nodes run counter-clockwise; match them to the oracle's by volume node
    fm = _lib_fmask(L, N)
    Nfp = N + 1
    for f in range(3):
        for k in range(Nfp):
            j_or = f * Nfp + list(ref.fmask[f]).index(fm[f][k])
            np.testing.assert_allclose(L['LIFT'][:, f * Nfp + k], ref.LIFT[:, j_or], atol=1e-13 * N * N)


@pytest.mark.parametrize('gamma', [0.0, -1e-9, -1e-5, -1e-2, -0.7, -1.0, -1.3, -4.5, -60.0])
def test_sark_coefficients_match_printed_forms(gamma):
    E, A, B = gb.sark_coefficients(gamma)
    E2, A2, B2 = sark.sark_coefficients(gamma)
    np.testing.assert_allclose(E, E2, rtol=2e-16, atol=1e-300)
    np.testing.assert_allclose(A, np.array(A2), rtol=1e-15, atol=1e-17)
    np.testing.assert_allclose(B, np.array(B2), rtol=1e-15, atol=1e-17)


def test_sark_rejects_positive_gamma():
    with pytest.raises(gb.GBError):
        gb.sark_coefficients(0.5)


def _expect(code, fn):
    with pytest.raises(gb.GBError) as ei:
        fn()
    assert ei.value.code == code, str(ei.value)


def test_create_validation_errors():
    mesh = inputs.periodic_square_mesh(4)
    _expect(gb.GB_EINVAL, lambda: gb.Solver(mesh, 0, 0.1, 100))
    _expect(gb.GB_EINVAL, lambda: gb.Solver(mesh, 7, 0.1, 100))
    _expect(gb.GB_EINVAL, lambda: gb.Solver(mesh, 3, -0.1, 100))
    _expect(gb.GB_EINVAL, lambda: gb.Solver(mesh, 3, 0.1, 0.0))
    _expect(gb.GB_EINVAL, lambda: gb.Solver(mesh, 3, 0.1, 100, precision=7))
    bad = dict(mesh)
    bad['EToV'] = mesh['EToV'].copy()
    bad['EToV'][0, 0] = 10 ** 6
    _expect(gb.GB_EINVAL, lambda: gb.Solver(bad, 3, 0.1, 100))


def test_create_mesh_errors():
    mesh = inputs.periodic_square_mesh(4)
    # inverted element
    inv = dict(mesh)
    inv['EToV'] = mesh['EToV'].copy()
    inv['EToV'][3] = inv['EToV'][3][[0, 2, 1]]
    inv['shift'] = mesh['shift'].copy()
    inv['shift'][3] = inv['shift'][3][[0, 2, 1]]
    _expect(gb.GB_EMESH, lambda: gb.Solver(inv, 3, 0.1, 100))
    # open mesh (periodic offsets dropped): faces without a matching copy
    opn = dict(mesh)
    opn['shift'] = None
    _expect(gb.GB_EMESH, lambda: gb.Solver(opn, 3, 0.1, 100))
    # a missing element leaves faces unmatched
    cut = {'X': mesh['X'], 'EToV': mesh['EToV'][1:], 'shift': mesh['shift'][1:]}
    _expect(gb.GB_EMESH, lambda: gb.Solver(cut, 3, 0.1, 100))


def dissipation_rate(t, kinetic_energy):
    """epsilon = -dE_K/dt (Sec. 7.2) from a recorded series, by second-order finite
    differences (central inside, one-sided at the ends; uneven spacing allowed)."""
    t = np.asarray(t, dtype=np.float64)
    e = np.asarray(kinetic_energy, dtype=np.float64)
    if t.size < 3:
        raise ValueError('need at least 3 records')
    return -np.gradient(e, t, edge_order=2)


def test_dissipation_rate_of_an_exponential_decay():
    # E_K = E0 exp(-4 nu t) (incompressible Taylor-Green decay): epsilon = 4 nu E_K,
    # to the O(dt^2) error of the differences, on uneven sampling too
    nu = 0.01
    for t in (np.linspace(0.0, 2.0, 201), np.sort(np.concatenate([np.linspace(0, 2, 150), np.linspace(0.013, 1.97, 60)]))):
        e = 0.25 * np.exp(-4 * nu * t)
        eps = dissipation_rate(t, e)
        assert np.max(np.abs(eps - 4 * nu * e) / (4 * nu * e)) < 1e-4
    with pytest.raises(ValueError):
        dissipation_rate([0.0, 1.0], [1.0, 0.5])


@pytest.mark.parametrize('N', [1, 2, 3, 4])
def test_library_tet_operators_match_oracle(N):
    """The library's long-double tetrahedral builder (orthonormal modes through homogeneous
    Jacobi recurrences) against the oracle's (monomial route)."""
    from oracle import tet
    from paper_2607_00199_b300 import gb
    L = gb.reference_operators3d(N)
    R = tet.ReferenceTet(N)
    assert L['Nc'] == R.Nc
    for k in ('r', 's', 't', 'cr', 'cs', 'ct', 'cw'):
        np.testing.assert_allclose(L[k], getattr(R, k), atol=1e-15)
    for k in ('Dr', 'Ds', 'Dt', 'I', 'P'):
        np.testing.assert_allclose(L[k], getattr(R, k), atol=1e-13)
    np.testing.assert_allclose(L['LIFT'], R.LIFT, atol=2e-12)


def test_more_host_validation():
    """Checks that return before any device work: empty meshes, 3D and bounded order limits,
    far-field states, and NULL solvers or arguments for every later entry point."""
    mesh = inputs.periodic_square_mesh(4)
    empty = {'X': mesh['X'], 'EToV': mesh['EToV'][:0], 'shift': mesh['shift'][:0]}
    _expect(gb.GB_EINVAL, lambda: gb.Solver(empty, 3, 0.1, 100))
    box = inputs.periodic_box_tet_mesh(3, 3, 3)
    _expect(gb.GB_EINVAL, lambda: gb.Solver(box, 5, 0.1, 100))          # dim = 3: N <= 4
    ogrid = inputs.naca_ogrid_mesh(16, 6, R=5.0)
    _expect(gb.GB_EINVAL, lambda: gb.Solver(ogrid, 5, 0.1, 100))        # boundary faces: N <= 4
    _expect(gb.GB_EINVAL, lambda: gb.Solver(ogrid, 3, 0.1, 100, far_state=(0.0, 1.0, 0.0)))
    _expect(gb.GB_EINVAL, lambda: gb.Solver(ogrid, 3, 0.1, 100, far_state=(1.0, float('nan'), 0.0)))
    lib = gb.lib
    out = np.zeros(8)
    n = ctypes.c_int64()
    assert lib.gb_set_pml(None, None) == gb.GB_EINVAL
    assert lib.gb_pml_fields(None, None, None, ctypes.byref(n)) == gb.GB_EINVAL
    assert lib.gb_diagnostics3d(None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == gb.GB_EINVAL
    assert lib.gb_diagnostics(None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == gb.GB_EINVAL
    assert lib.gb_set_diagnostics(None, 1, 4) == gb.GB_EINVAL
    assert lib.gb_step(None, 1e-3, 1) == gb.GB_EINVAL
    assert lib.gb_set_motion(None, None) == gb.GB_EINVAL
    assert lib.gb_set_wave_motion(None, None) == gb.GB_EINVAL
