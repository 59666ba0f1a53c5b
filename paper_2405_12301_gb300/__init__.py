"""GB300-native WENO5-JS residual for the compressible Euler equations.

The compute path lives in the CUDA library ``_lib/libweno_gb300.so`` (built
from ``csrc/``) and is reached through the ctypes binding in ``weno``.
Importing the package itself loads nothing; ``inputs`` holds the seeded
synthetic workloads.
"""
