"""Error measures of the GPU parity tests.

`rel_err(a, b)` is the larger of two relative errors of `a` against the reference `b`:
the relative L2 norm over the whole array, and the element-wise bound
max |a - b| / max |b|.  A tolerance written as `rel_err(a, b) <= tol` therefore bounds every
single value, so that one wrong element cannot hide in the norm of a large mesh.

The element-wise scale is the array's largest value, not each field's: the right-hand side
of a field can be a small residual of cancelling terms of size c |grad q| (the density of a
nearly incompressible flow), and its rounding error scales with those terms, whose size the
array's largest value gives, not with the residual.  Per-field relative L2 bounds stay in the
tests that have them.
"""
import numpy as np


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def elem_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / np.abs(b).max())


def rel_err(a, b):
    return max(rel_l2(a, b), elem_err(a, b))
