"""Plain, slow CPU oracle for the stage-parallel Radau IIA heat solver.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code,
tables or helpers with the CUDA path (``paper_2209_06700_gb300``), and it
imports nothing from there.

Everything here is FP64 NumPy/SciPy written from the definitions in
arXiv 2209.06700 (Sec. 1 "Introduction": the Runge-Kutta update; Sec. 2:
the linear system M u' + K u = g, the Kronecker stage system, Eq. (irk:A),
Eq. (irk:Ainv), Eq. (irk:P); Sec. 5: the heat problem on the unit cube with
continuous tensor-product Lagrange elements and Gauss quadrature; Sec. 6:
the 2x2 real form and PRESB).  Modules:

* ``tableau`` - Radau IIA (A, b, c), A^{-1}, Crout LU, the real spectral
  factors of L, and the real Jordan form of A^{-1}.
* ``fem``     - GLL nodes, Gauss rules, Lagrange bases, element matrices by
  direct quadrature, assembly to CSR, element-by-element apply.
* ``heat``    - the manufactured problem: source, load vector, initial
  interpolant, exact solution, FE L2 error.
* ``irk``     - stage right-hand side, the full Kronecker stage system
  solved directly, the exact per-mode IRK step by fast diagonalisation, the
  exact semi-discrete solution, and the operator (irk:A) apply.
* ``deformed`` - the same heat problem on a curved mesh of the cube (the
  uniform mesh under a boundary-fixing non-affine map, Sec. 3.4's case of
  mapping data per quadrature point): per-cell matrices by direct
  quadrature with the exact Jacobian, load, initial value, L2 error.
* ``paper_workload`` - the paper's own manufactured solution (Sec. 5).
* ``mg``      - multigrid ingredients written from their definitions:
  Q_k embedding (prolongation), restriction, Jacobi diagonal, Chebyshev
  iteration, dense coarse solve, one V-cycle, PRESB.

Parity status per function is stated in each module header.
"""
