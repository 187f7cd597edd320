"""Reference tetrahedron: nodes and operators of the 3D nodal DG discretisation, FP64
(oracle; test infrastructure only).

Paper, Sec. 3: the scheme runs on straight-sided simplices in two and three
dimensions with the Lagrange basis of the Warp & Blend nodes (Warburton, J. Eng.
Math. 2006); the operators are D = M^-1 S, LIFT = M^-1 M^f and P = M^-1 I^T W.

Reference tetrahedron: vertices v0 = (-1,-1,-1), v1 = (1,-1,-1), v2 = (-1,1,-1),
v3 = (-1,-1,1); barycentric coordinates
    l0 = -(1 + r + s + t)/2, l1 = (1 + r)/2, l2 = (1 + s)/2, l3 = (1 + t)/2.
Faces (local vertex triples): face 0 = (0,1,2) on t = -1, face 1 = (0,1,3) on s = -1,
face 2 = (1,2,3) on r + s + t = -1, face 3 = (0,2,3) on r = -1.

Node order: equidistant lattice indices (i, j, k) with r-index i innermost, then s-index
j, then t-index k outermost (i + j + k <= N); the Warp & Blend map moves each lattice
node but keeps its place in the order.  Face nodes: the nodes lying on the face, in
increasing volume index.

Construction, in the method's own terms:
* Warp & Blend in 3D: the equidistant nodes of the equilateral tetrahedron (edge 2)
  are shifted, face by face, by the face warp -- for each edge of the face the 1D warp
  (equidistant -> Gauss-Lobatto on that edge, divided by the edge bubble) times
  4 la lb (1 + (alpha lc)^2) along the edge direction -- blended into the volume by
  lb lc ld (1 + (alpha la)^2) / ((lb + la/2)(lc + la/2)(ld + la/2)), la the coordinate
  of the vertex opposite the face; nodes on an edge of a face take that face's warp
  itself.  alpha is Warburton's optimised value for tetrahedra (0 for N <= 3).
* The nodal basis is written through monomials in (l1, l2, l3): l_i = sum_m C[m, i]
  mono_m with C the inverse monomial Vandermonde, so the derivative operators are the
  exact derivatives of the interpolating polynomials, Dr[i, j] = d/dr l_j(x_i).  (This
  route is independent of the orthonormal-basis construction of the library.)
* Integrals (mass, face mass, cubature) use conical-product Gauss rules exact for the
  degree at hand: on the tetrahedron Gauss-Legendre x Gauss-Jacobi(1,0) x
  Gauss-Jacobi(2,0) in collapsed coordinates (Stroud), on a face the triangle rule of
  oracle.operators mapped onto the face.  The face measure is the one in which every
  face has parameter area 2 (the reference triangle); the physical face scaling
  Fscale therefore includes the area ratio of face 2 (sqrt 3).
* Collision cubature (reading, as in 2D): Stroud rule exact for degree 3N, q =
  ceil((3N+1)/2) points per direction, N_c = q^3 (64 at N = 2, 125 at N = 3).

Pins (tests/test_oracle_tet.py): edge nodes are Gauss-Lobatto points, face nodes are
the 2D Warp & Blend nodes with the same alpha, the node set has the tetrahedron's
symmetry and is equidistant for N <= 2; Dr, Ds, Dt exact on monomials; mass, face
mass and cubature integrate monomials exactly (closed-form simplex integrals); P I is
the identity.
"""
import itertools
import math

import numpy as np
from scipy.special import roots_jacobi, roots_legendre

from . import basis
from .operators import stroud_rule

# Warburton (2006), optimised blend parameter for tetrahedra, N = 1..15 (1.0 beyond)
_ALPHA_TET = (0.0, 0.0, 0.0, 0.1002, 1.1332, 1.5608, 1.3413, 1.2577, 1.1603, 1.10153,
              0.6080, 0.4523, 0.8856, 0.8717, 0.9655)

REF_VERTS = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
FACE_VERTS = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))
# outward unit normals of the reference faces, and reference face area / parameter area 2
REF_NORMALS = np.array([[0.0, 0.0, -1.0], [0.0, -1.0, 0.0],
                        [1.0 / math.sqrt(3.0)] * 3, [-1.0, 0.0, 0.0]])
REF_FACE_JAC = np.array([1.0, 1.0, math.sqrt(3.0), 1.0])


def alpha_tet(N):
    return _ALPHA_TET[N - 1] if N <= len(_ALPHA_TET) else 1.0


def barycentric(r, s, t):
    """(l0, l1, l2, l3) of reference points, stacked on the last axis."""
    r, s, t = (np.asarray(v, dtype=np.float64) for v in (r, s, t))
    return np.stack([-(1.0 + r + s + t) / 2.0, (1.0 + r) / 2.0, (1.0 + s) / 2.0, (1.0 + t) / 2.0], axis=-1)


def lattice(N):
    """Equidistant lattice indices (i, j, k), i innermost, k outermost."""
    return [(i, j, k) for k in range(N + 1) for j in range(N + 1 - k) for i in range(N + 1 - j - k)]


def warp_blend_nodes(N, alpha=None):
    """Warp & Blend nodes (r, s, t) of order N on the reference tetrahedron."""
    if alpha is None:
        alpha = alpha_tet(N)
    idx = np.array(lattice(N), dtype=np.float64)
    lam = np.empty((idx.shape[0], 4))
    lam[:, 1] = idx[:, 0] / N
    lam[:, 2] = idx[:, 1] / N
    lam[:, 3] = idx[:, 2] / N
    lam[:, 0] = 1.0 - lam[:, 1:].sum(axis=1)
    # equilateral tetrahedron with edge 2
    V = np.array([[-1.0, -1.0 / math.sqrt(3.0), -1.0 / math.sqrt(6.0)],
                  [1.0, -1.0 / math.sqrt(3.0), -1.0 / math.sqrt(6.0)],
                  [0.0, 2.0 / math.sqrt(3.0), -1.0 / math.sqrt(6.0)],
                  [0.0, 0.0, 3.0 / math.sqrt(6.0)]])
    X = lam @ V
    tol = 1e-10
    shift = np.zeros_like(X)
    for face in FACE_VERTS:
        opp = ({0, 1, 2, 3} - set(face)).pop()
        La = lam[:, opp]
        fw = np.zeros_like(X)
        for a, b in ((face[0], face[1]), (face[1], face[2]), (face[2], face[0])):
            c = ({0, 1, 2, 3} - {a, b, opp}).pop()
            d = V[b] - V[a]
            d = d / np.linalg.norm(d)
            amount = 4.0 * lam[:, a] * lam[:, b] * basis.warp_factor(N, lam[:, b] - lam[:, a]) * (1.0 + (alpha * lam[:, c]) ** 2)
            fw += amount[:, None] * d[None, :]
        Lb, Lc, Ld = (lam[:, v] for v in face)
        blend = Lb * Lc * Ld
        denom = (Lb + 0.5 * La) * (Lc + 0.5 * La) * (Ld + 0.5 * La)
        ok = denom > tol
        blend[ok] = (1.0 + (alpha * La[ok]) ** 2) * blend[ok] / denom[ok]
        shift += blend[:, None] * fw
        on_edge = (La < tol) & (((Lb > tol).astype(int) + (Lc > tol) + (Ld > tol)) < 3)
        shift[on_edge] = fw[on_edge]
    X = X + shift
    # back to barycentric coordinates of the equilateral tetrahedron, then to (r, s, t)
    A = np.vstack([V.T, np.ones(4)])                    # [x; y; z; 1] = A lam
    lam2 = np.linalg.solve(A, np.vstack([X.T, np.ones(X.shape[0])])).T
    rst = lam2 @ REF_VERTS
    return rst[:, 0], rst[:, 1], rst[:, 2]


def monomial_exponents(N):
    return [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a) for c in range(N + 1 - a - b)]


def monomials(N, r, s, t):
    """mono[k, m] = l1^a l2^b l3^c at the points, with (a, b, c) = monomial_exponents(N)[m]."""
    lam = barycentric(r, s, t)
    out = np.empty((lam.shape[0], len(monomial_exponents(N))))
    for m, (a, b, c) in enumerate(monomial_exponents(N)):
        out[:, m] = lam[:, 1] ** a * lam[:, 2] ** b * lam[:, 3] ** c
    return out


def monomial_grads(N, r, s, t):
    """(d/dr, d/ds, d/dt) of the monomials; d l1/dr = d l2/ds = d l3/dt = 1/2."""
    lam = barycentric(r, s, t)
    ex = monomial_exponents(N)
    G = [np.zeros((lam.shape[0], len(ex))) for _ in range(3)]
    for m, e in enumerate(ex):
        for d in range(3):
            if e[d] == 0:
                continue
            p = list(e)
            p[d] -= 1
            G[d][:, m] = 0.5 * e[d] * lam[:, 1] ** p[0] * lam[:, 2] ** p[1] * lam[:, 3] ** p[2]
    return G


def tet_rule(degree):
    """Conical-product rule on the reference tetrahedron, exact for total degree <= degree.

    Collapsed coordinates: t = c, s = (1+b)(1-c)/2 - 1, r = (1+a)(1-b)(1-c)/4 - 1 with
    dr ds dt = (1-b)/2 ((1-c)/2)^2 da db dc; Gauss-Legendre in a, Gauss-Jacobi(1,0) in b
    and Gauss-Jacobi(2,0) in c, q = ceil((degree+1)/2) points each.  Points c-major,
    then b, then a.  Returns (r, s, t, w).
    """
    q = int(math.ceil((degree + 1) / 2.0))
    a, wa = roots_legendre(q)
    b, wb = roots_jacobi(q, 1.0, 0.0)
    c, wc = roots_jacobi(q, 2.0, 0.0)
    R, S, T, W = [], [], [], []
    for kc in range(q):
        for jb in range(q):
            for ia in range(q):
                T.append(c[kc])
                S.append((1.0 + b[jb]) * (1.0 - c[kc]) / 2.0 - 1.0)
                R.append((1.0 + a[ia]) * (1.0 - b[jb]) * (1.0 - c[kc]) / 4.0 - 1.0)
                W.append(wa[ia] * wb[jb] * wc[kc] / 8.0)
    return np.array(R), np.array(S), np.array(T), np.array(W)


def face_points(f, r2, s2):
    """Map points (r2, s2) of the reference triangle (-1,-1), (1,-1), (-1,1) onto face f:
    the triangle's vertices go to the face's vertices in FACE_VERTS order."""
    mu = np.stack([-(r2 + s2) / 2.0, (1.0 + r2) / 2.0, (1.0 + s2) / 2.0], axis=-1)
    P = mu @ REF_VERTS[list(FACE_VERTS[f])]
    return P[:, 0], P[:, 1], P[:, 2]


class ReferenceTet:
    """Reference operators of order N on the tetrahedron, from their integral definitions."""

    def __init__(self, N):
        self.N = N
        self.Np = (N + 1) * (N + 2) * (N + 3) // 6
        self.Nfp = (N + 1) * (N + 2) // 2
        self.r, self.s, self.t = warp_blend_nodes(N)
        Vm = monomials(N, self.r, self.s, self.t)
        self.C = np.linalg.inv(Vm)                        # l_i = sum_m C[m, i] mono_m

        def lagrange(r, s, t):
            return monomials(N, r, s, t) @ self.C         # [point, i]

        def lagrange_grads(r, s, t):
            return [g @ self.C for g in monomial_grads(N, r, s, t)]

        self.lagrange = lagrange
        Gr, Gs, Gt = lagrange_grads(self.r, self.s, self.t)
        self.Dr, self.Ds, self.Dt = Gr, Gs, Gt            # Dr[i, j] = d/dr l_j(x_i)
        qr, qs, qt, qw = tet_rule(2 * N)
        ell = lagrange(qr, qs, qt)
        self.M = ell.T @ np.diag(qw) @ ell
        self.Minv = np.linalg.inv(self.M)
        lam = barycentric(self.r, self.s, self.t)
        self.fmask = [np.nonzero(np.abs(lam[:, ({0, 1, 2, 3} - set(fv)).pop()]) < 1e-10)[0] for fv in FACE_VERTS]
        for fm in self.fmask:
            assert fm.size == self.Nfp
        # face mass, parameter measure (area 2 per face)
        fr2, fs2, fw2 = stroud_rule(2 * N)
        E = np.zeros((self.Np, 4 * self.Nfp))
        for f in range(4):
            pr, ps, pt = face_points(f, fr2, fs2)
            ellf = lagrange(pr, ps, pt)
            E[:, f * self.Nfp:(f + 1) * self.Nfp] = ellf.T @ np.diag(fw2) @ ellf[:, self.fmask[f]]
        self.Mf = E
        self.LIFT = self.Minv @ E
        cr, cs, ct, cw = tet_rule(3 * N)
        self.cr, self.cs, self.ct, self.cw = cr, cs, ct, cw
        self.Nc = cr.size
        self.I = lagrange(cr, cs, ct)                     # [Nc, Np]
        self.P = self.Minv @ self.I.T @ np.diag(cw)        # [Np, Nc]
        self.bary = lam                                    # P1 interpolation of vertex data


def symmetry_maps():
    """The 24 permutations of the four barycentric coordinates (the tetrahedron's symmetries)."""
    return list(itertools.permutations(range(4)))


def gll_on_edge(N):
    """Gauss-Lobatto parameters in [0, 1] along an edge (for the pins)."""
    return (basis.gauss_lobatto(N) + 1.0) / 2.0
