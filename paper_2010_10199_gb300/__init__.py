"""GB300 grouped Fourier transform, LSQR and FISTA for ANOVA approximation.

Submodules:
* ``gft``    -- ctypes binding of the C ABI (``include/anova_gft.h``); all
               computation happens in ``libanova_gft.so`` (CUDA, sm_103a)
* ``build``  -- in-tree nvcc build of that library
* ``inputs`` -- seeded synthetic workloads (no method arithmetic)

Importing the package does not load the CUDA library; ``gft.load()`` does,
and raises if the library has not been built.
"""

__all__ = ["gft", "build", "inputs"]
