"""Nested-mesh convolution potential solver for GB300 (sm_103a).

The solver computes the gravitational potential on a nested Cartesian mesh with
the convolution method of Vorobyov et al. (2023): per level, zero-padded FFT
convolution of the cell masses with the isolated inverse-distance kernel, then
cross-level interpolation and summation (Eq. 14), optionally with the pairwise
dipole correction (Eqs. 15, B.1-B.2).  All arithmetic runs in the CUDA library
``libnestconv.so`` behind a C ABI (``include/nm.h``); this package only
marshals arguments to it.

``workloads`` (seeded synthetic densities) imports nothing else, so it can be
used without the CUDA library.  The binding (``nm``) is imported lazily.
"""

def __getattr__(name):
    if name in ("nm", "serve"):
        import importlib
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
