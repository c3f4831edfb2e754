"""GB300-native semi-implicit step of the 1D3V electron Boltzmann equation (arXiv 2502.16555).

The compute path lives in ``csrc/`` (host assembly in C++, kernels in CUDA for sm_103a) and is
reached through the C ABI declared in ``include/bte.h``; ``paper_2502_16555_gb300.bte`` is the thin
ctypes binding to it.  ``workloads`` holds the synthetic workload descriptions and seeded draws.

Importing the package loads nothing; the shared library is opened on first use of ``bte``.
"""
__version__ = "0.1.0"
