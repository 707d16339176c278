"""GB300-native hybrid lattice-Boltzmann for the integral nonlinear Maxwell fluid (arXiv:1504.06123).

The compute path is the CUDA library ``_build/liblbve.so`` (C ABI in ``include/lbve.h``); the Python
modules only marshal arguments.  There is no CPU fallback: importing :mod:`.lbve` raises when the
library is missing.
"""
__all__ = ["lbve", "inputs", "configs"]
