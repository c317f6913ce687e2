"""Plain, slow FP64 CPU oracle for the RBF-FD Poisson pipeline.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  The CUDA library never calls it and
shares no code with it; both sides read their inputs from `fixtures`.

Each stage is the plain definition of what the method computes, written with
numpy/scipy primitives and no blocking or reordering beyond that definition:

* `knn`       -- n nearest nodes by brute force, ties broken by index (Sec. II,
                 the support set N(x) of Eq. 1).
* `weights`   -- RBF-FD Laplacian weights from the PHS r^3 + monomial augmented
                 system, one dense LU solve per stencil (Sec. II Eq. 1, Sec. V).
* `assemble`  -- the discrete Poisson operator with Dirichlet rows and its
                 right-hand side (Sec. IV, Eqs. 2-4 at steady state).
* `solve`     -- the sparse linear system solved directly (Sec. VI, the
                 implicit solve), plus the adjoint gradient.
* `explicit`  -- the paper's explicit Euler step (Eq. 4) and its data-size
                 model (Sec. V, Table 1).

Pins that tie each function to the paper or to mathematics live in
tests/test_oracle_*.py.
"""

from .knn import knn, knn_query, knn_grid  # noqa: F401
from .weights import monomial_exponents, n_monomials, local_system, weights, weights_rows  # noqa: F401
from .assemble import assemble, rhs  # noqa: F401
from .solve import solve_direct, solve_refined, residual_extended, gmres_right, adjoint_gradient, poisson_solve  # noqa: F401
from .explicit import explicit_step, l2_estimate_nodes  # noqa: F401
