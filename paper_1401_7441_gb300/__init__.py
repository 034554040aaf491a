"""GB300 (sm_103a) localized Hamiltonian application and sparse H/S build for
Daubechies-wavelet linear-scaling DFT (arXiv 1401.7441).

The product is the C-ABI library ``liblsw.so`` (include/lsw.h, sources in ``csrc/``);
``lsw`` is its ctypes binding, ``build`` compiles it in-tree, ``inputs`` generates the
seeded synthetic workloads.  Importing the package loads nothing: the library is
loaded on first use and its absence is an error (there is no fallback path).
"""
__all__ = ["build", "inputs", "lsw"]
