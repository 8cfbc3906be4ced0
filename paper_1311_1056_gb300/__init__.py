"""GB300 complex Langevin with adaptive gauge cooling (arXiv:1311.1056).

The compute path is the CUDA library libcl.so (C-ABI in include/cl.h); this
package holds its sources (csrc/), its build step (build.py) and the ctypes
binding (cl.py).
"""
from . import cl  # noqa: F401
from .cl import Lattice, make_cool, make_params  # noqa: F401
