"""Polynomial machinery on the reference triangle, FP64 (oracle; test infrastructure only).

Paper, Sec. 3: the solution on each element is a degree-N polynomial written in
the Lagrange basis of the Warp & Blend nodes (Warburton, J. Eng. Math. 2006).
This module builds those nodes and an orthonormal modal basis from their
published definitions:

* Gauss-Lobatto points: the end points plus the roots of P'_N, i.e. the
  Gauss-Jacobi(1,1) points of degree N-1 (scipy's Golub-Welsch rule).
* Warp & Blend nodes: equidistant barycentric nodes in the equilateral
  triangle, displaced along each edge direction by the 1D warp that takes
  equidistant points to Gauss-Lobatto points, blended into the interior by
  4*L_a*L_b*(1 + (alpha*L_c)^2), with Warburton's optimised alpha.
* Orthonormal (Dubiner/Koornwinder) basis
  psi_ij(r,s) = sqrt(2) Pn_i(a) Pn_j^{(2i+1,0)}(b) (1-b)^i,
  a = 2(1+r)/(1-s) - 1, b = s, with Pn the L2-normalised Jacobi polynomials.

Reference triangle: vertices (-1,-1), (1,-1), (-1,1) (counter-clockwise).
Node order: rows of constant L1 (the barycentric coordinate of vertex
(-1,1)), bottom row first; inside a row, increasing L3 (towards (1,-1)).

Pins: Gauss-Lobatto points against closed forms; Warp & Blend edge nodes are
Gauss-Lobatto points, the node set has the triangle's 3-fold symmetry, and the
published alpha is a local minimiser of the Lebesgue constant (the property it
was chosen for); the basis is orthonormal under an exact cubature.
"""
import math

import numpy as np
from scipy.special import eval_jacobi, gammaln, roots_jacobi

# Warburton (2006), optimised blend parameter alpha for triangles, N = 1..15;
# alpha = 5/3 beyond that.
_ALPHA_OPT = (0.0000, 0.0000, 1.4152, 0.1001, 0.2751, 0.9800, 1.0999,
              1.2832, 1.3648, 1.4773, 1.4959, 1.5743, 1.5770, 1.6223, 1.6258)


def alpha_opt(N):
    """Warburton's optimised blend parameter for order N (triangles)."""
    return _ALPHA_OPT[N - 1] if N <= len(_ALPHA_OPT) else 5.0 / 3.0


def jacobi_norm2(n, alpha, beta):
    """Squared L2 norm of P_n^{(alpha,beta)} under weight (1-x)^alpha (1+x)^beta."""
    logv = ((alpha + beta + 1) * math.log(2.0) - math.log(2 * n + alpha + beta + 1)
            + gammaln(n + alpha + 1) + gammaln(n + beta + 1)
            - gammaln(n + alpha + beta + 1) - gammaln(n + 1))
    return math.exp(logv)


def jacobi_normalized(x, alpha, beta, n):
    """Orthonormal Jacobi polynomial P_n^{(alpha,beta)}(x) / ||P_n||."""
    x = np.asarray(x, dtype=np.float64)
    return eval_jacobi(n, alpha, beta, x) / math.sqrt(jacobi_norm2(n, alpha, beta))


def jacobi_normalized_deriv(x, alpha, beta, n):
    """d/dx of the orthonormal Jacobi polynomial.

    Uses d/dx P_n^{(a,b)} = (n+a+b+1)/2 * P_{n-1}^{(a+1,b+1)}.
    """
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    dp = 0.5 * (n + alpha + beta + 1) * eval_jacobi(n - 1, alpha + 1, beta + 1, x)
    return dp / math.sqrt(jacobi_norm2(n, alpha, beta))


def gauss_lobatto(N):
    """N+1 Gauss-Lobatto-Legendre points on [-1, 1], ascending."""
    if N == 1:
        return np.array([-1.0, 1.0])
    interior, _ = roots_jacobi(N - 1, 1.0, 1.0)
    return np.concatenate(([-1.0], np.sort(interior), [1.0]))


def _lagrange_equidistant(N, r):
    """Matrix L[k, i] = l_i(r_k) of the Lagrange basis on N+1 equidistant points."""
    req = np.linspace(-1.0, 1.0, N + 1)
    r = np.asarray(r, dtype=np.float64)
    L = np.ones((r.size, N + 1))
    for i in range(N + 1):
        for j in range(N + 1):
            if j != i:
                L[:, i] *= (r - req[j]) / (req[i] - req[j])
    return L


def warp_factor(N, r):
    """1D warp divided by the edge blend (1 - r^2); zero at r = +-1.

    warp(r) interpolates (GLL point - equidistant point) on the equidistant
    points, so the warp moves equidistant points onto Gauss-Lobatto points.
    """
    r = np.asarray(r, dtype=np.float64)
    shift = gauss_lobatto(N) - np.linspace(-1.0, 1.0, N + 1)
    warp = _lagrange_equidistant(N, r) @ shift
    out = np.zeros_like(r)
    inside = np.abs(r) < 1.0 - 1e-10
    out[inside] = warp[inside] / (1.0 - r[inside] ** 2)
    return out


def warp_blend_nodes(N, alpha=None):
    """Warp & Blend nodes (r, s) on the reference triangle, in the documented order."""
    if alpha is None:
        alpha = alpha_opt(N)
    L1, L3 = [], []
    for n in range(N + 1):              # row index: L1 = n/N
        for m in range(N + 1 - n):      # in-row index: L3 = m/N
            L1.append(n / N)
            L3.append(m / N)
    L1 = np.array(L1)
    L3 = np.array(L3)
    L2 = 1.0 - L1 - L3
    # equilateral triangle: L1 -> (0, 2/sqrt3), L2 -> (-1, -1/sqrt3), L3 -> (1, -1/sqrt3)
    x = -L2 + L3
    y = (-L2 - L3 + 2.0 * L1) / math.sqrt(3.0)
    # edge opposite vertex c, between vertices a and b, tangent direction t_c
    blends = [(L2, L3, L1, 0.0), (L3, L1, L2, 2.0 * math.pi / 3.0), (L1, L2, L3, 4.0 * math.pi / 3.0)]
    for La, Lb, Lc, ang in blends:
        shift = 4.0 * La * Lb * warp_factor(N, Lb - La) * (1.0 + (alpha * Lc) ** 2)
        x = x + math.cos(ang) * shift
        y = y + math.sin(ang) * shift
    # back to barycentric coordinates, then to (r, s)
    l1 = (math.sqrt(3.0) * y + 1.0) / 3.0
    l2 = (-3.0 * x - math.sqrt(3.0) * y + 2.0) / 6.0
    l3 = (3.0 * x - math.sqrt(3.0) * y + 2.0) / 6.0
    r = -l2 + l3 - l1
    s = -l2 - l3 + l1
    return r, s


def rs_to_ab(r, s):
    """Collapsed coordinates a = 2(1+r)/(1-s) - 1 (a = -1 at s = 1), b = s."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    a = np.full_like(r, -1.0)
    ok = np.abs(1.0 - s) > 1e-14
    a[ok] = 2.0 * (1.0 + r[ok]) / (1.0 - s[ok]) - 1.0
    return a, s.copy()


def mode_indices(N):
    """Modal index pairs (i, j), i + j <= N, in a fixed order."""
    return [(i, j) for i in range(N + 1) for j in range(N + 1 - i)]


def simplex_mode(r, s, i, j):
    """Orthonormal triangle mode psi_ij evaluated at (r, s)."""
    a, b = rs_to_ab(r, s)
    return (math.sqrt(2.0) * jacobi_normalized(a, 0, 0, i)
            * jacobi_normalized(b, 2 * i + 1, 0, j) * (1.0 - b) ** i)


def simplex_mode_grad(r, s, i, j):
    """(d/dr, d/ds) of psi_ij, written as polynomials (no division by 1-s)."""
    a, b = rs_to_ab(r, s)
    f = jacobi_normalized(a, 0, 0, i)
    df = jacobi_normalized_deriv(a, 0, 0, i)
    g = jacobi_normalized(b, 2 * i + 1, 0, j)
    dg = jacobi_normalized_deriv(b, 2 * i + 1, 0, j)
    c = math.sqrt(2.0)
    one_b_im1 = (1.0 - b) ** (i - 1) if i >= 1 else np.zeros_like(b)
    dr = 2.0 * c * df * g * one_b_im1
    ds = c * (df * g * (1.0 + a) * one_b_im1 + f * dg * (1.0 - b) ** i - i * f * g * one_b_im1)
    return dr, ds


def vandermonde(N, r, s):
    """V[k, m] = psi_m(r_k, s_k) over the modes of mode_indices(N)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    modes = mode_indices(N)
    V = np.zeros((r.size, len(modes)))
    for m, (i, j) in enumerate(modes):
        V[:, m] = simplex_mode(r, s, i, j)
    return V


def grad_vandermonde(N, r, s):
    """(Vr, Vs): derivatives of the modes at the points."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    modes = mode_indices(N)
    Vr = np.zeros((r.size, len(modes)))
    Vs = np.zeros((r.size, len(modes)))
    for m, (i, j) in enumerate(modes):
        Vr[:, m], Vs[:, m] = simplex_mode_grad(r, s, i, j)
    return Vr, Vs


def lagrange_at(N, r_nodes, s_nodes, r, s):
    """Matrix of nodal Lagrange basis functions: out[k, i] = l_i(r_k, s_k)."""
    V = vandermonde(N, r_nodes, s_nodes)
    Vq = vandermonde(N, r, s)
    return np.linalg.solve(V.T, Vq.T).T


def lagrange_grad_at(N, r_nodes, s_nodes, r, s):
    """(d/dr l_i, d/ds l_i) at the points, as two [k, i] matrices."""
    V = vandermonde(N, r_nodes, s_nodes)
    Vr, Vs = grad_vandermonde(N, r, s)
    return np.linalg.solve(V.T, Vr.T).T, np.linalg.solve(V.T, Vs.T).T
