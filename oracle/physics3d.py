"""3D Galerkin-Boltzmann physics, 10 fields (oracle; test infrastructure only).

Paper, Sec. 2: expanding the phase-space density in Hermite polynomials up to second
order gives n = 6 coefficients in 2D and n = 10 in 3D; the 3D matrices are not printed
(the paper refers to its companion work).  They follow from the same construction as
the printed 2D ones: with the orthonormal Hermite functions of the scaled particle
velocity, xi psi_k = sqrt(k+1) psi_{k+1} + sqrt(k) psi_{k-1} in each direction, so
Atilde_d couples the moment of multi-index alpha with alpha +- e_d (both of total
order <= 2) with weight sqrt(max(alpha_d, beta_d)).  The printed 2D matrices are
exactly this rule on the indices (0,0), (1,0), (0,1), (1,1), (2,0), (0,2).

Field order (reading): q1..q10 = moments (0,0,0); (1,0,0), (0,1,0), (0,0,1);
(1,1,0), (1,0,1), (0,1,1); (2,0,0), (0,2,0), (0,0,2).  Macroscopic maps as in 2D:
rho = q1, rho u = c q2, rho v = c q3, rho w = c q4 (c = sqrt(RT)).

Collision (BGK, Sec. 2 pattern): the second-order moments relax to the moments of the
local Maxwellian, q_(e_i + e_j) -> q_{1+i} q_{1+j} / q1 (i != j) and
q_(2 e_i) -> q_{1+i}^2 / (sqrt2 q1), so N(q) = -(1/tau)(q_alpha - q_alpha^eq) on fields
5..10; Sec. 4 splits it as -Lambda q + Ntilde(q), Lambda = diag(0,0,0,0,1/tau x 6).

Pins (tests/test_oracle_physics3d.py): restricted to the z-free moments the matrices
are the printed 2D ones; Atilde_n has the spectrum {0 x4, +-1 x2, +-sqrt3} for every
unit n (so |Atilde_n| = alpha Atilde_n^2 + beta Atilde_n^4 with the 2D alpha, beta);
the equilibrium moment flux is the Euler flux (p + rho u^2, rho u v, ...); the
collision term vanishes at equilibrium; nu = tau RT (shear-wave decay, solver tests).
"""
import math

import numpy as np

SQ2 = math.sqrt(2.0)
NFIELDS = 10

MULTI_INDEX = ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1),
               (2, 0, 0), (0, 2, 0), (0, 0, 2))


def hermite_matrix(d):
    """Atilde_d (10 x 10) from the Hermite recurrence (module doc)."""
    A = np.zeros((10, 10))
    for i, a in enumerate(MULTI_INDEX):
        for j, b in enumerate(MULTI_INDEX):
            diff = [a[k] - b[k] for k in range(3)]
            if abs(diff[d]) == 1 and all(diff[k] == 0 for k in range(3) if k != d):
                A[i, j] = math.sqrt(max(a[d], b[d]))
    return A


ATX, ATY, ATZ = (hermite_matrix(d) for d in range(3))

# the z-free moments in the 2D order (q1, q2, q3, q4, q5, q6) of Sec. 2
SUBSET_2D = (0, 1, 2, 4, 7, 8)


def abs_normal_matrix(n):
    """|Atilde_n| for unit normals n (..., 3), from the symmetric eigen-decomposition."""
    n = np.asarray(n, dtype=np.float64)
    An = n[..., 0, None, None] * ATX + n[..., 1, None, None] * ATY + n[..., 2, None, None] * ATZ
    lam, R = np.linalg.eigh(An)
    return np.einsum('...ik,...k,...jk->...ij', R, np.abs(lam), R)


def ntilde(q1, q2, q3, q4, tau):
    """Non-stiff collision part for fields 5..10 (Sec. 4 splitting)."""
    r = 1.0 / (tau * q1)
    rs = r / SQ2
    return (q2 * q3 * r, q2 * q4 * r, q3 * q4 * r, q2 * q2 * rs, q3 * q3 * rs, q4 * q4 * rs)


def collision(q, tau):
    """Full BGK collision term, fields on the last axis."""
    q1, q2, q3, q4 = (q[..., k] for k in range(4))
    eq = (q2 * q3 / q1, q2 * q4 / q1, q3 * q4 / q1, q2 * q2 / (SQ2 * q1), q3 * q3 / (SQ2 * q1), q4 * q4 / (SQ2 * q1))
    out = np.zeros_like(q)
    for k in range(6):
        out[..., 4 + k] = -(q[..., 4 + k] - eq[k]) / tau
    return out


def equilibrium_state(rho, u, v, w, c):
    """q (fields on a new last axis) from (rho, u, v, w) with the second moments at equilibrium."""
    rho = np.asarray(rho, dtype=np.float64)
    q2 = rho * np.asarray(u, dtype=np.float64) / c
    q3 = rho * np.asarray(v, dtype=np.float64) / c
    q4 = rho * np.asarray(w, dtype=np.float64) / c
    return np.stack([rho, q2, q3, q4, q2 * q3 / rho, q2 * q4 / rho, q3 * q4 / rho,
                     q2 * q2 / (SQ2 * rho), q3 * q3 / (SQ2 * rho), q4 * q4 / (SQ2 * rho)], axis=-1)


def macroscopic(q, c):
    """(rho, rho u, rho v, rho w), fields on the last axis."""
    return q[..., 0], c * q[..., 1], c * q[..., 2], c * q[..., 3]
