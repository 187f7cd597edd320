"""Initial states for the solver, from macroscopic fields (input preparation, host).

Sec. 2 maps: q1 = rho, q2 = rho u / c, q3 = rho v / c.  The paper does not state
the initial second-order moments; they start at their equilibrium values
q4 = q2 q3 / q1, q5 = q2^2 / (sqrt2 q1), q6 = q3^2 / (sqrt2 q1), where the
collision term of Sec. 2 vanishes.
"""
import math

import numpy as np


def equilibrium_fields(rho, u, v, c):
    """Canonical (K, 6, Np) FP64 fields from nodal rho, u, v of shape (K, Np)."""
    rho = np.asarray(rho, dtype=np.float64)
    q1 = rho
    q2 = rho * u / c
    q3 = rho * v / c
    sq2 = math.sqrt(2.0)
    return np.ascontiguousarray(np.stack([q1, q2, q3, q2 * q3 / q1, q2 * q2 / (sq2 * q1), q3 * q3 / (sq2 * q1)], axis=1))


def equilibrium_fields3(rho, u, v, w, c):
    """Canonical (K, 10, Np) FP64 fields of the 3D system from nodal rho, u, v, w of shape
    (K, Np): moments (0,0,0), (1,0,0), (0,1,0), (0,0,1), (1,1,0), (1,0,1), (0,1,1),
    (2,0,0), (0,2,0), (0,0,2), the second-order ones at equilibrium."""
    rho = np.asarray(rho, dtype=np.float64)
    q2, q3, q4 = rho * u / c, rho * v / c, rho * w / c
    sq2 = math.sqrt(2.0)
    return np.ascontiguousarray(np.stack([rho, q2, q3, q4, q2 * q3 / rho, q2 * q4 / rho, q3 * q4 / rho,
                                          q2 * q2 / (sq2 * rho), q3 * q3 / (sq2 * rho), q4 * q4 / (sq2 * rho)],
                                         axis=1))
