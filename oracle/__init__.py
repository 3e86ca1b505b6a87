"""FP64 CPU oracle of the periodic vertex model.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import anything here; the
CUDA library and its Python binding never do.  The oracle shares no code with
the CUDA path: it uses Qhull (scipy) for the periodic Voronoi tessellation,
plain numpy for energy, forces and the explicitly assembled Hessian, and a
dense factorisation for the adjoint.
"""
from . import mesh, model, solvers  # noqa: F401
