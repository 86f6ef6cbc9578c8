"""Plain, slow CPU oracle for the eHDG method (arXiv 1601.06681).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import or call this
package: only the tests, the smoke check and the CPU-baseline leg of the
benchmark use it. It shares no code with the CUDA library.

Everything is float64 numpy. Modules:
  basis     -- Gauss-Lobatto-Legendre nodes, Gauss rules, 1D Lagrange bases
  local_ops -- element operators of the upwind HDG local equations
               (Sec. 3, transportLocal / transportLocalk1, localSolverDD)
  ehdg      -- the eHDG iteration (Algorithm 1) with backward Euler,
               Crank-Nicolson and steady stepping, and the trace formulas
               (transportLocale; the shallow-water trace of Sec. 3)
  direct    -- direct solve of the monolithic upwind HDG system (local
               equations plus weak conservation on every face, Sec. 3)
  geometry  -- node coordinates of the structured mesh for building inputs

Readings of points the paper leaves open are listed in each function's
docstring; the pins that tie this code to the paper are in tests/test_oracle_*.
"""
