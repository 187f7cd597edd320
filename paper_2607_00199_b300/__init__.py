"""B300-native ALE discontinuous Galerkin solver for the Galerkin-Boltzmann equations.

The compute path lives in the CUDA library ``libgb.so`` (sources in ``csrc/``,
C ABI declared in ``include/gb.h``); ``gb.py`` is its thin ctypes binding.
``inputs.py`` holds the seeded synthetic input generators.  Importing this
package does not load the library; ``paper_2607_00199_b300.gb`` does.
"""
