"""Pins for the oracle's reference operators (Sec. 3: D, LIFT, I, P and the cubature)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import operators


def exact_triangle_integral(a, b):
    """int over the reference triangle of r^a s^b, exactly (rational).

    With r = 2u - 1, s = 2v - 1 on the unit simplex, dr ds = 4 du dv and
    int u^i v^j = i! j! / (i + j + 2)!.
    """
    tot = Fraction(0)
    for i in range(a + 1):
        for j in range(b + 1):
            coef = math.comb(a, i) * math.comb(b, j) * 2 ** (i + j) * (-1) ** (a - i + b - j)
            tot += coef * Fraction(math.factorial(i) * math.factorial(j), math.factorial(i + j + 2))
    return 4 * tot


def test_exact_integral_sanity():
    assert exact_triangle_integral(0, 0) == 2            # area
    assert exact_triangle_integral(1, 0) == Fraction(-2, 3)   # centroid r = -1/3


@pytest.mark.parametrize('deg', [4, 6, 9, 12, 15])
def test_stroud_rule_exact(deg):
    r, s, w = operators.stroud_rule(deg)
    assert abs(w.sum() - 2.0) < 1e-14
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            assert abs(w @ (r ** a * s ** b) - float(exact_triangle_integral(a, b))) < 1e-13


@pytest.mark.parametrize('N', [2, 3, 4, 5])
def test_cubature_size_reading(N):
    ref = operators.ReferenceElement(N)
    q = math.ceil((3 * N + 1) / 2)
    assert ref.Nc == q * q
    assert {2: 16, 3: 25, 4: 49, 5: 64}[N] == ref.Nc


@pytest.mark.parametrize('N', range(1, 7))
def test_differentiation_exact_on_monomials(N):
    ref = operators.ReferenceElement(N)
    r, s = ref.r, ref.s
    for a in range(N + 1):
        for b in range(N + 1 - a):
            f = r ** a * s ** b
            fr = a * r ** (a - 1) * s ** b if a else 0 * f
            fs = b * r ** a * s ** (b - 1) if b else 0 * f
            np.testing.assert_allclose(ref.Dr @ f, fr, atol=5e-13)
            np.testing.assert_allclose(ref.Ds @ f, fs, atol=5e-13)


@pytest.mark.parametrize('N', range(1, 6))
def test_mass_matrix_integrates_products(N):
    ref = operators.ReferenceElement(N)
    r, s = ref.r, ref.s
    mons = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]
    for (a1, b1) in mons:
        for (a2, b2) in mons:
            got = (r ** a1 * s ** b1) @ ref.M @ (r ** a2 * s ** b2)
            assert abs(got - float(exact_triangle_integral(a1 + a2, b1 + b2))) < 1e-13


@pytest.mark.parametrize('N', range(1, 6))
def test_face_mass_integrates_products(N):
    ref = operators.ReferenceElement(N)
    r, s = ref.r, ref.s
    mons = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]
    Pt = np.polynomial.Polynomial
    # face parameterisations as polynomials in t (counter-clockwise faces)
    faces = [(Pt([0, 1]), Pt([-1])), (Pt([0, -1]), Pt([0, 1])), (Pt([-1]), Pt([0, -1]))]
    for f in range(3):
        cols = slice(f * ref.Nfp, (f + 1) * ref.Nfp)
        fr, fs = faces[f]
        for (a1, b1) in mons:
            for (a2, b2) in mons:
                p = (fr ** a1) * (fs ** b1) * (fr ** a2) * (fs ** b2)
                exact = p.integ()(1.0) - p.integ()(-1.0)
                g = r[ref.fmask[f]] ** a2 * s[ref.fmask[f]] ** b2
                got = (r ** a1 * s ** b1) @ ref.Mf[:, cols] @ g
                assert abs(got - exact) < 1e-12
    # LIFT = M^-1 Mf
    np.testing.assert_allclose(ref.M @ ref.LIFT, ref.Mf, atol=1e-12)


@pytest.mark.parametrize('N', range(1, 7))
def test_projection_is_identity_on_PN(N):
    ref = operators.ReferenceElement(N)
    np.testing.assert_allclose(ref.P @ ref.I, np.eye(ref.Np), atol=1e-12)


@pytest.mark.parametrize('N', [2, 3, 4])
def test_projection_is_L2_projection(N):
    # P f_c gives the P_N coefficients of the L2 projection of a non-polynomial f
    ref = operators.ReferenceElement(N)
    f = lambda r, s: np.exp(0.3 * r - 0.2 * s) / (1.5 + 0.2 * s)
    pf = ref.P @ f(ref.cr, ref.cs)
    # orthogonality of the residual to P_N, with a much finer rule
    hr, hs, hw = operators.stroud_rule(40)
    from oracle import basis
    ell = basis.lagrange_at(N, ref.r, ref.s, hr, hs)
    resid = f(hr, hs) - ell @ pf
    # the degree-3N rule makes the projection exact up to the rule's own error
    assert np.abs(ell.T @ (hw * resid)).max() < 1e-6
