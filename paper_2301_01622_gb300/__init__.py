"""GB300-native moment-only ("lightweight") lattice Boltzmann (arXiv 2301.01622).

The compute path is the C-ABI library ``libllb.so`` (CUDA, sm_103a) built
from ``csrc/`` by ``build.py``; ``llb`` is its thin ctypes binding with the
same function names as ``include/llb.h``.  ``inputs`` generates the seeded
synthetic initial fields.

Importing the package does not load the library; the first call into
``llb`` does, and raises if the library has not been built.
"""
__all__ = ["llb", "inputs", "build"]
