"""Plain FP64 CPU oracle for the CutFEM multigrid of Cui & Kanschat (arXiv 2508.11608).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.

It computes, slowly and by the plain definitions:

* classification of background cells against the level set (Sec. 2.1),
* Q_p finite element spaces with a Gauss-Lobatto nodal basis on active cells
  (eq. "spaces"),
* cut-cell quadrature by dimension reduction (the algorithm cited in Sec. 3),
* the assembled Nitsche + ghost-penalty matrix A_l (eqs. "cutfem_nitsche",
  "cutfem-ghost"), as a scipy CSR matrix,
* the embedding prolongation and its transpose (Sec. 2.2),
* the vertex patches, their colours, A_{l,j} = A_l[I_j, I_j] and the
  partitioned multiplicative smoother (eqs. "local-solver", "smoother",
  "smoother-split"),
* the V-cycle with an exact coarsest solve, and CG preconditioned by it.

It shares no code with the CUDA path.  Parity pins live in ``tests/``.
"""

from .levelset import Sphere, Plane, make_levelset  # noqa: F401
from .basis import Basis1D, gll_nodes  # noqa: F401
from .quadrature import cut_cell_rule, gauss01  # noqa: F401
from .fem import Level, assemble_level  # noqa: F401
from .multigrid import Hierarchy  # noqa: F401
