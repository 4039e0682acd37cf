"""Plain FP64 CPU oracle for GCA-H^2 compression (Boerm & Christophersen,
"GCA-H^2 matrix compression for electrostatic simulations").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library (no kernels, headers, helpers, tables or constant generators); the
only module both sides use is ``synth`` (seeded meshes and right-hand sides),
which holds none of the method's arithmetic.

The oracle is deliberately slow and literal: it follows the paper's steps
in the paper's order, in float64, with numpy / scipy primitives as single
steps and no blocking or fusion.  Module map:

* ``rules``     quadrature rules: Gauss-Legendre, the 7-point triangle
                rule, the Gauss rule on the faces of the box omega (Sect. 2)
* ``sauter``    Sauter-Schwab transformations for touching triangle pairs
                (Sect. 8: identical / common edge / common vertex)
* ``galerkin``  the kernel g, its normal derivative and the Galerkin
                entries g_ij of Eq. (1); the dense matrix G for small n
* ``cluster``   cluster tree, bounding boxes, admissibility, block tree
                (Sect. 2)
* ``gca``       Green quadrature matrices (Sect. 2), cross approximation
                with complete pivoting (Sect. 3), nested bases and
                transfer matrices, coupling and near-field blocks (Sect. 4)
* ``h2``        H^2 matrix-vector products (fast recursion and explicit
                bases), transposes, dense reconstruction, error estimates

Parity status per function is stated in each module header; every function
listed there is pinned by a ``-m "not gpu"`` test unless marked
"parity unpinned".
"""

from .params import Params  # noqa: F401
