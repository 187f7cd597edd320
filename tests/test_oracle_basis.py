"""Pins for the oracle's nodes and modal basis (Sec. 3: Warp & Blend nodes, P_N basis)."""
import math
import os

import numpy as np
import pytest

from oracle import basis, operators

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')


def test_gauss_lobatto_closed_forms():
    # textbook closed forms of the Gauss-Lobatto-Legendre points
    np.testing.assert_allclose(basis.gauss_lobatto(2), [-1, 0, 1], atol=1e-15)
    np.testing.assert_allclose(basis.gauss_lobatto(3), [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], atol=1e-15)
    np.testing.assert_allclose(basis.gauss_lobatto(4), [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], atol=1e-15)
    a = math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21)
    b = math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21)
    np.testing.assert_allclose(basis.gauss_lobatto(5), [-1, -b, -a, a, b, 1], atol=1e-15)


@pytest.mark.parametrize('N', range(1, 9))
def test_warp_blend_counts_and_edges(N):
    r, s = basis.warp_blend_nodes(N)
    assert r.size == (N + 1) * (N + 2) // 2
    gll = basis.gauss_lobatto(N)
    # the nodes on each edge are exactly the Gauss-Lobatto points of that edge
    edge0 = np.sort(r[np.abs(s + 1) < 1e-12])
    edge2 = np.sort(s[np.abs(r + 1) < 1e-12])
    edge1 = np.sort(s[np.abs(r + s) < 1e-12])
    for e in (edge0, edge1, edge2):
        np.testing.assert_allclose(e, gll, atol=2e-15)
    # all nodes inside the closed triangle
    assert np.all(r >= -1 - 1e-14) and np.all(s >= -1 - 1e-14) and np.all(r + s <= 1e-14)


@pytest.mark.parametrize('N', range(1, 9))
def test_warp_blend_threefold_symmetry(N):
    r, s = basis.warp_blend_nodes(N)
    L = np.stack([(1 + s) / 2, -(r + s) / 2, (1 + r) / 2], axis=1)    # (L1, L2, L3)
    rot = L[:, [1, 2, 0]]
    refl = L[:, [0, 2, 1]]
    for P in (rot, refl):
        d = np.abs(P[:, None, :] - L[None, :, :]).sum(-1)
        assert d.min(axis=1).max() < 1e-13


def test_low_order_nodes_equidistant():
    for N in (1, 2):
        r, s = basis.warp_blend_nodes(N)
        req = [(-1 + 2 * m / N, -1 + 2 * n / N) for n in range(N + 1) for m in range(N + 1 - n)]
        np.testing.assert_allclose(np.stack([r, s], 1), np.array(req), atol=1e-15)


def _lebesgue(N, alpha=None, M=200):
    r, s = basis.warp_blend_nodes(N, alpha)
    i, j = np.meshgrid(np.arange(M + 1), np.arange(M + 1), indexing='ij')
    m = i + j <= M
    ell = basis.lagrange_at(N, r, s, -1 + 2 * i[m] / M, -1 + 2 * j[m] / M)
    return np.abs(ell).sum(1).max()


def test_lebesgue_constants_match_published_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, 'wb_lebesgue_triangle.txt')) if l.strip() and l[0] != '#']
    for N, lam in rows:
        got = _lebesgue(int(N))
        assert abs(got - float(lam)) <= 0.0051 + 0.002, (N, got, lam)


@pytest.mark.parametrize('N', [6, 7])
def test_published_alpha_is_local_lebesgue_minimum(N):
    a = basis.alpha_opt(N)
    lam0 = _lebesgue(N, a, M=90)
    assert lam0 < _lebesgue(N, a - 0.05, M=90)
    assert lam0 < _lebesgue(N, a + 0.05, M=90)


@pytest.mark.parametrize('N', range(1, 7))
def test_modal_basis_orthonormal(N):
    cr, cs, cw = operators.stroud_rule(2 * N)
    V = basis.vandermonde(N, cr, cs)
    np.testing.assert_allclose(V.T @ np.diag(cw) @ V, np.eye(V.shape[1]), atol=1e-13)


@pytest.mark.parametrize('N', range(1, 7))
def test_modal_gradients_match_finite_differences(N):
    rng = np.random.default_rng(N)
    r = rng.uniform(-0.9, 0.3, 20)
    s = rng.uniform(-0.9, -0.1, 20)
    s = np.minimum(s, -r - 0.05)
    h = 1e-6
    Vr, Vs = basis.grad_vandermonde(N, r, s)
    fdr = (basis.vandermonde(N, r + h, s) - basis.vandermonde(N, r - h, s)) / (2 * h)
    fds = (basis.vandermonde(N, r, s + h) - basis.vandermonde(N, r, s - h)) / (2 * h)
    np.testing.assert_allclose(Vr, fdr, atol=1e-7)
    np.testing.assert_allclose(Vs, fds, atol=1e-7)
