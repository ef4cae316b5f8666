"""CPU oracle for the finite-difference Poisson iteration of the Dirichlet cavity.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
call it.  It shares no code with the CUDA library (no kernels, headers, tables or
helpers); the only module both sides use is the seeded input generator, which holds
none of the method's arithmetic.

Modules
-------
``fd``         the 2nd-order FD operator, the Dirichlet lifting, exact discrete
               solutions (sparse LU and the discrete sine transform) and the closed
               forms (Dirichlet eigenvalues, k_max, the discrete plane wave).
``iteration``  the paper's nested Poisson iteration (Section 2.2 with alpha = k^2,
               p = 0, as discretised in Section 2.4) with exact inner solves, its
               residual / increment histories and the convergence status rule.
``multigrid``  textbook geometric-multigrid components (red-black Gauss-Seidel,
               full weighting, multilinear prolongation, V-cycle) written as plain
               numpy.  The paper prescribes no inner solver; these restate, in the
               simplest form, the operation sequence the CUDA V-cycle performs, so
               that a single sweep or cycle can be checked element by element.

Every floating-point computation here is float64 / complex128.
"""
from . import fd, iteration, multigrid  # noqa: F401
