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
