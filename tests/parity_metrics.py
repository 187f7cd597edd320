"""Error measures of the GPU parity tests.

`rel_err(a, b)` is the larger of two relative errors of `a` against the reference `b`:
the relative L2 norm over the whole array, and the element-wise bound
max |a - b| / max |b| taken field by field when the arrays are (elements, fields, nodes)
(field scale max |b_f|, floored at 1e-3 max |b| so that a field that is identically zero in
the reference does not divide by zero), over the whole array otherwise.  A tolerance written
as `rel_err(a, b) <= tol` therefore bounds every single value, so that one wrong element
cannot hide in the norm of a large mesh.
"""
import numpy as np


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def elem_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    bmax = float(np.abs(b).max())
    if a.ndim == 3:
        d = np.abs(a - b).max(axis=(0, 2))
        s = np.maximum(np.abs(b).max(axis=(0, 2)), 1e-3 * bmax)
        return float((d / s).max())
    return float(np.abs(a - b).max() / bmax)


def rel_err(a, b):
    return max(rel_l2(a, b), elem_err(a, b))
