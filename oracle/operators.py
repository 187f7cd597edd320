"""Reference-element operators of the nodal DG discretisation (oracle; test infrastructure only).

Paper, Sec. 3 (definitions following the discrete form): on each element
    M_ij = int phi_i phi_j,  M^f_ij = int_face phi_i phi_j,  S_ij = int phi_i d(phi_j),
    D = M^-1 S,  LIFT = M^-1 M^f,  P = M^-1 I^T diag(w).
For an affine element M = J Mhat, S_x = J (r_x Shat_r + s_x Shat_s) and
M^f = sJ Mhat^f, so the physical operators are the reference ones times the
constant geometric factors.  The oracle therefore builds the reference
operators here by evaluating those integrals with exact quadrature, and the
solver applies the geometric factors.

Reading (index order of S): the paper prints S_ij = int phi_j d(phi_i); the
index order that makes D = M^-1 S the nodal derivative is S_ij = int phi_i
d(phi_j), used here.

Cubature for the collision term (Sec. 3): the paper asks for an
"appropriately high order" rule without naming it.  Reading: the Stroud
conical-product rule of degree 3N, i.e. q = ceil((3N+1)/2) Gauss-Legendre
points in a times q Gauss-Jacobi(1,0) points in b (collapsed coordinates),
N_c = q^2 points, ordered b-major (outer b, inner a).

Pins: Dr, Ds exact on monomials of degree <= N; the mass matrix, face mass and
cubature integrate monomials exactly (closed-form integrals over the
triangle); P I = identity on P_N.
"""
import math

import numpy as np
from scipy.special import roots_jacobi, roots_legendre

from . import basis


def cubature_degree(N):
    """Degree of the collision-term cubature rule: 3N (reading, see module doc)."""
    return 3 * N


def stroud_rule(degree):
    """Conical-product rule on the reference triangle, exact for total degree <= degree.

    int_T f dr ds = int_{-1}^{1} int_{-1}^{1} f(r(a,b), b) (1-b)/2 da db, with
    r = (1+a)(1-b)/2 - 1.  Gauss-Legendre in a and Gauss-Jacobi(1,0) in b
    (weight (1-b)) with q points each are exact for degree 2q-1 in each variable.
    Returns (r, s, w) with points ordered b-major.
    """
    q = int(math.ceil((degree + 1) / 2.0))
    a, wa = roots_legendre(q)
    b, wb = roots_jacobi(q, 1.0, 0.0)
    R, S, W = [], [], []
    for jb in range(q):
        for ia in range(q):
            R.append((1.0 + a[ia]) * (1.0 - b[jb]) / 2.0 - 1.0)
            S.append(b[jb])
            W.append(wa[ia] * wb[jb] / 2.0)
    return np.array(R), np.array(S), np.array(W)


def face_param(f, t):
    """Reference coordinates (r, s) of face f at face parameter t in [-1, 1].

    Faces run counter-clockwise: face 0 from (-1,-1) to (1,-1), face 1 from
    (1,-1) to (-1,1), face 2 from (-1,1) to (-1,-1).
    """
    t = np.asarray(t, dtype=np.float64)
    if f == 0:
        return t, -np.ones_like(t)
    if f == 1:
        return -t, t
    return -np.ones_like(t), -t


# reference outward unit normals and d(arc length)/dt of the three faces
REF_NORMALS = np.array([[0.0, -1.0], [1.0 / math.sqrt(2.0), 1.0 / math.sqrt(2.0)], [-1.0, 0.0]])
REF_FACE_JAC = np.array([1.0, math.sqrt(2.0), 1.0])


class ReferenceElement:
    """All reference operators of order N, built from their integral definitions."""

    def __init__(self, N):
        self.N = N
        self.Np = (N + 1) * (N + 2) // 2
        self.Nfp = N + 1
        self.r, self.s = basis.warp_blend_nodes(N)
        # exact quadrature for the mass/stiffness integrals (degree 2N)
        qr, qs, qw = stroud_rule(2 * N + 2)
        ell = basis.lagrange_at(N, self.r, self.s, qr, qs)            # [q, i]
        dell_r, dell_s = basis.lagrange_grad_at(N, self.r, self.s, qr, qs)
        W = np.diag(qw)
        self.M = ell.T @ W @ ell                       # M_ij = int l_i l_j
        self.Sr = ell.T @ W @ dell_r                   # S_ij = int l_i d/dr l_j
        self.Ss = ell.T @ W @ dell_s
        Minv = np.linalg.inv(self.M)
        self.Minv = Minv
        self.Dr = Minv @ self.Sr
        self.Ds = Minv @ self.Ss
        # face nodes: the nodes lying on each face (found geometrically)
        on_face = [np.abs(self.s + 1.0) < 1e-10,
                   np.abs(self.r + self.s) < 1e-10,
                   np.abs(self.r + 1.0) < 1e-10]
        self.fmask = [np.nonzero(m)[0] for m in on_face]
        for fm in self.fmask:
            assert fm.size == self.Nfp
        # face mass per face: Mf[i, k] = int_{-1}^{1} l_i(face(t)) l_{fmask[k]}(face(t)) dt
        t, wt = roots_legendre(N + 2)
        E = np.zeros((self.Np, 3 * self.Nfp))
        for f in range(3):
            fr, fs = face_param(f, t)
            ellf = basis.lagrange_at(N, self.r, self.s, fr, fs)     # [t, i]
            E[:, f * self.Nfp:(f + 1) * self.Nfp] = ellf.T @ np.diag(wt) @ ellf[:, self.fmask[f]]
        self.Mf = E
        self.LIFT = Minv @ E
        # cubature of degree 3N for the collision term, interpolation and projection
        cr, cs, cw = stroud_rule(cubature_degree(N))
        self.cr, self.cs, self.cw = cr, cs, cw
        self.Nc = cr.size
        self.I = basis.lagrange_at(N, self.r, self.s, cr, cs)      # [Nc, Np]
        self.P = Minv @ self.I.T @ np.diag(cw)                      # [Np, Nc]
        # P1 (vertex) interpolation to the nodes: barycentric coordinates
        self.bary = np.stack([-(self.r + self.s) / 2.0, (1.0 + self.r) / 2.0, (1.0 + self.s) / 2.0], axis=1)
