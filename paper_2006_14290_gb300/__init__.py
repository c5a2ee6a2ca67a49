"""GB300-native sparse-solver hot path: CSR/ELL/COO/hybrid SpMV and CG,
BiCGSTAB, GMRES on it, behind the C ABI in ``include/gko.h``.

``gko``      thin ctypes binding of the C ABI (the CUDA library does the work)
``inputs``   seeded synthetic matrices and vectors
``build``    nvcc build of ``libgko_gb300.so`` for sm_103a
"""
