"""GB300 complex Langevin with adaptive gauge cooling (arXiv:1311.1056).

The compute path is the CUDA library libcl.so (C-ABI in include/cl.h); this
package holds its sources (csrc/), its build step (build.py), the ctypes
binding (cl.py: lattices, step graphs, batches, the request server, the SU(2)
Polyakov chains), the seeded synthetic workloads (workloads.py) and the
studies of Sec. 3-5 run on the kernels (studies.py).
"""
from . import cl  # noqa: F401
from .cl import Batch, Lattice, PolyakovChains, Server, make_cool, make_params, make_request  # noqa: F401
