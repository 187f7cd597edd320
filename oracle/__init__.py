"""Plain FP64 CPU oracle for the ALE discontinuous Galerkin Galerkin-Boltzmann method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: it is used by ``tests/``, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.

The oracle follows the paper (arXiv 2607.00199) step by step, in plain numpy
loops and library primitives (matrix products, ``numpy.linalg``,
``scipy.special`` Gauss-Jacobi rules, ``mpmath``).  It shares no code with the
CUDA library in ``paper_2607_00199_b300/``: every operator, connectivity map
and coefficient is rebuilt here from the mathematics.

Modules
-------
basis      Jacobi polynomials, Gauss-Lobatto points, Warp & Blend nodes, the
           orthonormal simplex basis (Sec. 3).
operators  mass, stiffness, differentiation, lift, cubature interpolation and
           projection operators on the reference triangle (Sec. 3).
physics    the 2D Galerkin-Boltzmann flux matrices, the collision term and the
           macroscopic maps (Sec. 2), plus the (Ma, Re) -> (c, tau) reading.
sark       semi-analytic Runge-Kutta coefficients (Sec. 4).
solver     the ALE right-hand side and the SARK step on a moving periodic
           triangle mesh (Secs. 2-5).
tet        Warp & Blend nodes and the reference operators of the tetrahedron
           (Sec. 3 in three dimensions; monomial route, exact rules).
physics3d  the 10-moment 3D Galerkin-Boltzmann system (Sec. 2 construction).
solver3d   the ALE right-hand side and SARK step on a moving periodic
           tetrahedral mesh.
pml        the perfectly matched layer of the airfoil case (a reading: complex
           stretching along the layer's direction with auxiliary fields).

Parity status of each function is stated in its docstring; functions with no
independent pin say "parity unpinned".
"""
