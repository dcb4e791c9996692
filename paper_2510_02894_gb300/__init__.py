"""GB300 (sm_103a) implementation of the 3D shape-feature hot path of
PyRadiomics-cuda (arXiv 2510.02894): marching cubes with mesh volume and
surface area, and the maximum 3D and planar diameters, as a C-ABI CUDA
library (librad.so, include/rad.h) with a thin ctypes binding (rad.py)."""
from . import rad  # noqa: F401
