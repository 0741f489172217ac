"""CPU oracle for the ghost-cell immersed-boundary fractional-step solver.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check of the package
entry point and the CPU-baseline leg of the benchmark may import this
package. The product (the CUDA library and its Python binding) never
imports, links or calls it, and shares no code with it: the two meet only
on the seeded inputs built by ``paper_2505_17287_gb300.synth``.

Layout:
  geom.c / geom.py  exact cell classification and ghost-cell tables
                    (Section 2.2, Eq. 2 and Eq. 3), plain C, FP64.
  flow.py           the discrete operators, the linear systems and one
                    fractional step (Section 2.1), numpy + scipy in FP64;
                    every linear system is solved by a sparse direct LU,
                    which is the plain definition of its solution.

Parity pins: every function is pinned by a test against something other than
itself (brute force with exact rationals, closed forms, separable
eigen-solutions, invariants); see tests/test_oracle_*.py.
"""
