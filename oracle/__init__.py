"""FP64 CPU oracle for the projection-based CHNS scheme on 2:1-balanced octrees.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product (the CUDA library and its Python binding)
never imports, calls or links anything here, and this package imports nothing from the product.

The oracle is the discretisation written out plainly, with assembled sparse matrices, the way the
paper builds its linear systems (Sec. 5.4, "Traversal-based matrix assembly"):

* ``mesh``   - node enumeration, hanging-node detection and the prolongation P (Sec. 5.3),
* ``fem``    - Q1 basis, 2x2x2 Gauss quadrature, element matrices and vectors of the discrete
               Cahn-Hilliard, velocity-prediction, pressure-Poisson and velocity-update problems
               (Sec. 4.1, Defs. of the VMS velocity prediction, pressure Poisson, velocity
               update and discrete Cahn-Hilliard equations), assembled as A = P^T (sum_e A_e) P,
* ``solvers``- plain Jacobi-PCG, Newton, and library direct/GMRES solves,
* ``step``   - the two-block time step of the flowchart (Fig. "flowchart_block").

Parity status per function is stated in each module header; functions without an independent
pin say "parity unpinned".
"""
