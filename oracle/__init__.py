"""FP64 CPU oracle for the immersed-boundary acoustic wave method (Caunt et al.).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

It is a plain, slow restatement of the paper, in the paper's order and notation:

* ``taylor``     -- truncated N-D Taylor basis, derivative operators, BC rows and
                    1D Taylor-system stencil weights (sections "Constructing
                    Finite-Difference Approximations", "Approximating Boundary
                    Conditions", free-surface constraints, velocity free surface).
* ``geometry``   -- interior mask, SDF normals, boundary points, eta cut-off
                    (boundary-point placement paragraph of "Approximating
                    Boundary Conditions").
* ``stencils``   -- support regions, the constrained fit A, its Moore-Penrose
                    pseudoinverse, extrapolation B A^+ and the modified operators
                    ("Reconciliation with the Interior Numerical Discretization",
                    multi-field section).
* ``operators``  -- the modified operators assembled as sparse matrices.
* ``propagate``  -- leapfrog and staggered time stepping, sources, receivers and
                    the exact discrete adjoint of the leapfrog map.
* ``images``     -- method-of-images analytic solutions for a flat surface.

On curved geometry the modified stencils are pinned through polynomial
exactness, brute-force checks, and exact solutions on a circle (harmonic fields
that meet every imposed condition there): the truncation of the rows and the
whole-field error converge at the extrapolation order (``tests/test_oracle_*``).
No individual curved-surface weight is compared with an external value: the
paper prints none for a reproducible geometry.
"""
