"""Pins for the oracle's reference tetrahedron (Sec. 3 in 3D: Warp & Blend nodes, D, LIFT,
I, P and the cubature)."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest
import sympy as sp

from oracle import basis, tet


def exact_tet_integral(a, b, c):
    """int over the reference tetrahedron of r^a s^b t^c, exactly.

    r = 2 l1 - 1 (and s, t likewise); int l1^i l2^j l3^k dV = 6 |T| i! j! k! / (i+j+k+3)!
    with |T| = 4/3 (the Dirichlet integral over a simplex)."""
    tot = Fraction(0)
    for i in range(a + 1):
        for j in range(b + 1):
            for k in range(c + 1):
                coef = (math.comb(a, i) * math.comb(b, j) * math.comb(c, k) * 2 ** (i + j + k)
                        * (-1) ** (a - i + b - j + c - k))
                tot += coef * Fraction(8 * math.factorial(i) * math.factorial(j) * math.factorial(k),
                                       math.factorial(i + j + k + 3))
    return tot


def test_exact_integral_sanity():
    assert exact_tet_integral(0, 0, 0) == Fraction(4, 3)
    assert exact_tet_integral(1, 0, 0) / exact_tet_integral(0, 0, 0) == Fraction(-1, 2)   # centroid r = -1/2


@pytest.mark.parametrize('deg', [2, 4, 6, 9])
def test_tet_rule_exact(deg):
    r, s, t, w = tet.tet_rule(deg)
    assert abs(w.sum() - 4.0 / 3.0) < 1e-14
    for a, b, c in itertools.product(range(deg + 1), repeat=3):
        if a + b + c <= deg:
            assert abs(w @ (r ** a * s ** b * t ** c) - float(exact_tet_integral(a, b, c))) < 1e-13


@pytest.mark.parametrize('N', [1, 2, 3, 4])
def test_node_count_vertices_and_edges(N):
    r, s, t = tet.warp_blend_nodes(N)
    assert r.size == (N + 1) * (N + 2) * (N + 3) // 6
    lam = tet.barycentric(r, s, t)
    assert np.allclose(lam.sum(axis=1), 1.0) and lam.min() > -1e-13
    for v in tet.REF_VERTS:                       # the four vertices are nodes
        assert np.min(np.linalg.norm(np.stack([r, s, t], 1) - v, axis=1)) < 1e-13
    # nodes on every edge sit at the Gauss-Lobatto points of that edge
    gll = np.sort(tet.gll_on_edge(N))
    for a, b in itertools.combinations(range(4), 2):
        others = [k for k in range(4) if k not in (a, b)]
        on = np.all(np.abs(lam[:, others]) < 1e-12, axis=1)
        np.testing.assert_allclose(np.sort(lam[on, b]), gll, atol=1e-13)


@pytest.mark.parametrize('N', [1, 2])
def test_low_orders_are_equidistant(N):
    r, s, t = tet.warp_blend_nodes(N)
    lam = tet.barycentric(r, s, t)
    assert np.allclose(np.round(lam * N), lam * N, atol=1e-13)


@pytest.mark.parametrize('N', [2, 3, 4, 5])
def test_node_set_has_tetrahedral_symmetry(N):
    lam = tet.barycentric(*tet.warp_blend_nodes(N))
    key = lambda L: sorted(tuple(np.round(row, 10)) for row in L)
    base = key(lam)
    for p in tet.symmetry_maps():
        assert key(lam[:, p]) == base


@pytest.mark.parametrize('N', [2, 3, 4, 5])
def test_face_nodes_are_triangle_warp_blend_nodes(N):
    """On a face the 3D construction reduces to the 2D one with the same alpha (its face
    blend is 1 and the other faces' blends vanish)."""
    lam = tet.barycentric(*tet.warp_blend_nodes(N))
    r2, s2 = basis.warp_blend_nodes(N, alpha=tet.alpha_tet(N))
    tri = np.stack([-(r2 + s2) / 2, (1 + r2) / 2, (1 + s2) / 2], 1)
    key = lambda L: sorted(tuple(np.round(row, 10)) for row in L)
    for fv in tet.FACE_VERTS:
        opp = ({0, 1, 2, 3} - set(fv)).pop()
        on = np.abs(lam[:, opp]) < 1e-12
        assert key(lam[on][:, list(fv)]) == key(tri)


@pytest.mark.parametrize('N', [1, 2, 3, 4])
def test_differentiation_exact_on_monomials(N):
    R = tet.ReferenceTet(N)
    r, s, t = R.r, R.s, R.t
    for a, b, c in itertools.product(range(N + 1), repeat=3):
        if a + b + c > N:
            continue
        f = r ** a * s ** b * t ** c
        d = [a * r ** max(a - 1, 0) * s ** b * t ** c, b * r ** a * s ** max(b - 1, 0) * t ** c,
             c * r ** a * s ** b * t ** max(c - 1, 0)]
        for D, ex in zip((R.Dr, R.Ds, R.Dt), d):
            np.testing.assert_allclose(D @ f, ex, atol=1e-12)


@pytest.mark.parametrize('N', [1, 2, 3])
def test_mass_matrix_integrates_monomials(N):
    R = tet.ReferenceTet(N)
    for (a, b, c), (d, e, g) in itertools.product(itertools.product(range(N + 1), repeat=3), repeat=2):
        if a + b + c > N or d + e + g > N:
            continue
        f1 = R.r ** a * R.s ** b * R.t ** c
        f2 = R.r ** d * R.s ** e * R.t ** g
        assert abs(f1 @ R.M @ f2 - float(exact_tet_integral(a + d, b + e, c + g))) < 1e-12


def _exact_face_integral(f, expr):
    """int over face f (parameter measure: area 2) of a sympy polynomial in r, s, t."""
    m1, m2 = sp.symbols('m1 m2')
    mu = [1 - m1 - m2, m1, m2]
    V = tet.REF_VERTS[list(tet.FACE_VERTS[f])]
    rr, ss, tt = (sum(sp.Rational(int(V[k][d])) * mu[k] for k in range(3)) for d in range(3))
    r, s, t = sp.symbols('r s t')
    g = sp.expand(expr.subs({r: rr, s: ss, t: tt}, simultaneous=True))
    # unit triangle (area 1/2) -> parameter triangle of area 2: factor 4
    return 4 * sp.integrate(sp.integrate(g, (m2, 0, 1 - m1)), (m1, 0, 1))


@pytest.mark.parametrize('N', [1, 2, 3])
def test_face_mass_and_lift(N):
    R = tet.ReferenceTet(N)
    r, s, t = sp.symbols('r s t')
    np.testing.assert_allclose(R.M @ R.LIFT, R.Mf, atol=1e-13)
    pairs = [((0, 0, 0), (0, 0, 0)), ((1, 0, 0), (0, 1, 0)), ((0, 0, 1), (N, 0, 0)), ((0, 1, 0), (0, 0, N))]
    for f in range(4):
        fm = R.fmask[f]
        for (a, b, c), (d, e, g) in pairs:
            p = R.r ** a * R.s ** b * R.t ** c
            qv = R.r ** d * R.s ** e * R.t ** g
            got = p @ R.Mf[:, f * R.Nfp:(f + 1) * R.Nfp] @ qv[fm]
            want = float(_exact_face_integral(f, r ** a * s ** b * t ** c * r ** d * s ** e * t ** g))
            assert abs(got - want) < 1e-12, (f, a, b, c, d, e, g)


@pytest.mark.parametrize('N', [1, 2, 3, 4])
def test_cubature_and_projection(N):
    R = tet.ReferenceTet(N)
    q = math.ceil((3 * N + 1) / 2)
    assert R.Nc == q ** 3
    np.testing.assert_allclose(R.P @ R.I, np.eye(R.Np), atol=1e-12)
    # P is the L2 projection: M P g = int l_i g for a smooth non-polynomial g, at the rule
    g = np.exp(0.3 * R.cr - 0.2 * R.cs + 0.1 * R.ct)
    np.testing.assert_allclose(R.M @ (R.P @ g), R.I.T @ (R.cw * g), atol=1e-13)


def test_reference_normals_and_face_areas():
    """Outward unit normals and face area / parameter area of the reference faces."""
    for f, fv in enumerate(tet.FACE_VERTS):
        P = tet.REF_VERTS[list(fv)]
        n = np.cross(P[1] - P[0], P[2] - P[0])
        area = 0.5 * np.linalg.norm(n)
        opp = tet.REF_VERTS[({0, 1, 2, 3} - set(fv)).pop()]
        n = n / np.linalg.norm(n)
        if n @ (P[0] - opp) < 0:
            n = -n
        np.testing.assert_allclose(n, tet.REF_NORMALS[f], atol=1e-15)
        assert abs(area / 2.0 - tet.REF_FACE_JAC[f]) < 1e-14
