"""GB300 (sm_103a) sub-sampled Fourier SAFT reconstruction: the operator
A = S F H of arXiv 2012.04534, its adjoint and FISTA, behind the C ABI of
include/sfs.h (libsfs.so).  ``sfs`` is the ctypes binding; ``build`` compiles
the library in-tree with nvcc."""
from . import sfs  # noqa: F401
from .sfs import Geometry, Operator, SfsError  # noqa: F401
