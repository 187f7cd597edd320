"""2D Galerkin-Boltzmann physics (oracle; test infrastructure only).

Paper, Sec. 2: q = (q1..q6) are Hermite coefficients of the phase-space
density; dq/dt = A_x dq/dx + A_y dq/dy + N(q) with A = -sqrt(RT) Atilde
(Atilde printed in full in Sec. 2) and the BGK collision term
N(q) = -(1/tau) (0, 0, 0, q4 - q2 q3/q1, q5 - q2^2/(sqrt2 q1), q6 - q3^2/(sqrt2 q1)).
Sec. 4 splits N(q) = -Lambda q + Ntilde(q) with Lambda = diag(0,0,0,1/tau,1/tau,1/tau).
Macroscopic maps (Sec. 2): rho = q1, rho u = sqrt(RT) q2, rho v = sqrt(RT) q3,
nu = tau RT.

Reading of (Ma, Re) (the paper only states nu = tau RT): lengths and the
reference velocity are 1 and rho0 = 1, so c = sqrt(RT) = 1/Ma, nu = 1/Re and
tau = nu / RT = Ma^2 / Re.

Reading of the wall condition (paper silent): bounce-back of the particle velocities about
the wall velocity, `wall_ghost`.  Far field (the paper's PML equations are not given):
the free-stream equilibrium as the exterior state of the upwind flux.

Reading of the initial non-equilibrium moments (not stated in the paper): q4..q6
start at their equilibrium values q2 q3/q1, q2^2/(sqrt2 q1), q3^2/(sqrt2 q1).
"""
import math

import numpy as np

SQ2 = math.sqrt(2.0)

ATX = np.array([
    [0, 1, 0, 0, 0, 0],
    [1, 0, 0, 0, SQ2, 0],
    [0, 0, 0, 1, 0, 0],
    [0, 0, 1, 0, 0, 0],
    [0, SQ2, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 0]], dtype=np.float64)

ATY = np.array([
    [0, 0, 1, 0, 0, 0],
    [0, 0, 0, 1, 0, 0],
    [1, 0, 0, 0, 0, SQ2],
    [0, 1, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 0],
    [0, 0, SQ2, 0, 0, 0]], dtype=np.float64)

NFIELDS = 6


def sound_speed_and_tau(Ma, Re):
    """(c, tau) = (1/Ma, Ma^2/Re) under the non-dimensional reading in the module doc."""
    c = 1.0 / Ma
    tau = Ma * Ma / Re
    return c, tau


def flux_matrices(c):
    """A_x = -c Atilde_x, A_y = -c Atilde_y (Sec. 2)."""
    return -c * ATX, -c * ATY


def abs_normal_matrix(nx, ny):
    """|Atilde_n| for Atilde_n = nx Atilde_x + ny Atilde_y, batched over normals.

    Computed from the symmetric eigen-decomposition R |Lambda| R^T (the paper's
    diagonalisation F_S = R Lambda R^-1, Sec. 3, upwind flux).
    """
    nx = np.asarray(nx, dtype=np.float64)
    ny = np.asarray(ny, dtype=np.float64)
    An = nx[..., None, None] * ATX + ny[..., None, None] * ATY
    lam, R = np.linalg.eigh(An)
    return np.einsum('...ik,...k,...jk->...ij', R, np.abs(lam), R)


def ntilde(q1, q2, q3, tau):
    """Non-stiff part of the collision term for fields 4..6 (Sec. 4, time splitting)."""
    return (q2 * q3 / (tau * q1),
            q2 * q2 / (tau * q1 * SQ2),
            q3 * q3 / (tau * q1 * SQ2))


def collision(q, tau):
    """Full BGK collision term N(q) of Sec. 2, fields on the last axis."""
    q1, q2, q3, q4, q5, q6 = [q[..., k] for k in range(6)]
    out = np.zeros_like(q)
    out[..., 3] = -(q4 - q2 * q3 / q1) / tau
    out[..., 4] = -(q5 - q2 * q2 / (q1 * SQ2)) / tau
    out[..., 5] = -(q6 - q3 * q3 / (q1 * SQ2)) / tau
    return out


def equilibrium_state(rho, u, v, c):
    """q from (rho, u, v) with q4..q6 at equilibrium; stacked on a new last axis."""
    rho = np.asarray(rho, dtype=np.float64)
    q1 = rho
    q2 = rho * np.asarray(u, dtype=np.float64) / c
    q3 = rho * np.asarray(v, dtype=np.float64) / c
    return np.stack([q1, q2, q3, q2 * q3 / q1, q2 * q2 / (SQ2 * q1), q3 * q3 / (SQ2 * q1)], axis=-1)


def macroscopic(q, c):
    """(rho, rho u, rho v) from q (fields on the last axis)."""
    return q[..., 0], c * q[..., 1], c * q[..., 2]


def wall_ghost(q, wx, wy):
    """Ghost state of a wall moving with velocity (wx, wy) c (reading; the paper gives no wall
    condition): the particle velocities are reflected about the wall velocity, xi -> 2 u_w - xi
    (bounce-back).  With zeta = xi / c the Hermite moments (Sec. 2 definitions:
    q2 = E[zeta_x], q4 = E[zeta_x zeta_y], q5 = (E[zeta_x^2] - rho)/sqrt2, ...) of the reflected
    density follow in closed form:
      q1+ = q1,  q2+ = 2 wx q1 - q2,  q3+ = 2 wy q1 - q3,
      q4+ = q4 + 4 wx wy q1 - 2 wx q3 - 2 wy q2,
      q5+ = q5 + 2 sqrt2 (wx^2 q1 - wx q2),  q6+ = q6 + 2 sqrt2 (wy^2 q1 - wy q3).
    Fields on the last axis; wx, wy broadcast against q[..., 0]."""
    q1, q2, q3, q4, q5, q6 = (q[..., k] for k in range(6))
    out = np.empty_like(q)
    out[..., 0] = q1
    out[..., 1] = 2.0 * wx * q1 - q2
    out[..., 2] = 2.0 * wy * q1 - q3
    out[..., 3] = q4 + 4.0 * wx * wy * q1 - 2.0 * wx * q3 - 2.0 * wy * q2
    out[..., 4] = q5 + 2.0 * SQ2 * (wx * wx * q1 - wx * q2)
    out[..., 5] = q6 + 2.0 * SQ2 * (wy * wy * q1 - wy * q3)
    return out
