"""GB300-native two-colour D2Q9 chromodynamic MRT lattice Boltzmann (arXiv 2005.04642).

The compute path is the CUDA library ``libcmrt`` (C ABI, ``include/cmrt.h``);
:mod:`paper_2005_04642_gb300.cmrt` is its thin ctypes binding and
:mod:`paper_2005_04642_gb300.inputs` builds seeded synthetic inputs.
Importing the package loads nothing; the library is loaded on first use.
"""
__all__ = ["inputs"]
