"""FP64 CPU oracle of the Chebyshev-collocation diffusion solver.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls, links
or runs this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (no kernels, headers, tables or helpers); both sides
take their inputs from the ``workloads`` generators only.

It computes the plain definition the method reaches, with dense matrices:
dense Chebyshev-Gauss-Lobatto differentiation matrices applied along each axis
(Kronecker structure, Sec. 2 "Extension to the three-dimensional setting"),
boundary rows replaced by the boundary conditions, a direct solve on tiny grids
and restarted GMRES otherwise.  No DCT appears here: the CUDA path's transform
route (Alg. 1 semantics) has to reproduce this dense definition.

Every function is pinned by ``tests/test_oracle.py`` against closed forms,
brute force or the paper's manufactured solutions; see ``PINS`` below for the
map.  Functions without an independent pin say "parity unpinned".
"""
from .core import *  # noqa: F401,F403
from .core import __all__  # noqa: F401
from .precond import (FDMPreconditioner, adjoint_solve_preconditioned,  # noqa: F401,E402
                      geometric_mean, solve_hierarchy, solve_preconditioned)
