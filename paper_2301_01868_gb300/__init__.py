"""GB300 library for the volumetric lattice Boltzmann method in general
curvilinear coordinates (arXiv:2301.01868): a C-ABI CUDA library
(``libclbm.so``, include/clbm.h) and its Python binding ``clbm``."""
from . import clbm  # noqa: F401
from .clbm import Grid, ClbmError, UnstableError  # noqa: F401
