"""GB300-native linear lattice-Boltzmann acoustic solver (arXiv:1704.03172).

The solver lives in a CUDA shared library behind a C ABI (``include/lbac.h``);
``paper_1704_03172_gb300.lbac`` is its ctypes binding and ``paper_1704_03172_gb300.sim``
the PyTorch-facing wrappers.  Importing this package does not load the library.
"""
__version__ = "0.1.0"
