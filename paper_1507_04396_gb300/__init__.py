"""GB300 (sm_103a) implementation of parallel Multiresolution Matrix Factorization.

The compute path lives in the CUDA library ``_lib/libpmmf.so`` (built by
``build.build()``); ``pmmf`` is its ctypes binding and ``inputs`` holds the
seeded synthetic workload generators.
"""

__all__ = ["build", "inputs", "pmmf"]
